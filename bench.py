"""Benchmark of the finite-PEPS hot path on the 8x8 open Heisenberg workload (D=4, chi=16,
N_s=4096 Metropolis chains).

One step = 2 Metropolis exchange sweeps of every chain + psi, E_loc and O of every chain
(boundary MPS) + one MinSR step + the parameter update, all through the C ABI.
value = samples/s = N_s (x ranks) / device time of one step.  The MinSR step time is reported
beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp64] [--ns NS]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Under torchrun (N > 1) every rank runs an independent replica of the workload (weak scaling,
no collective on the data path); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "samples/sec (psi, E_loc, O_k via boundary MPS) & MinSR step s, vs FP64 plain"
WORKLOAD = "heis8x8_D4_chi16"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--ns", type=int, default=None)
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--burnin", type=int, default=20)
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="steps of the plain FP64 GPU path timed after the main run (0: skip)")
    ap.add_argument("--mode", default="step", choices=["step", "learned", "gram", "batch", "complex", "bound", "rotated", "direct"])
    ap.add_argument("--branches", type=int, default=8)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--cpu-samples", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--solve", default=None, choices=["ff", "fp64", "fp32"],
                    help="MinSR Cholesky: float-float factor + FP64 refinement (FP32 default), FP64 "
                         "(FP64 default), or FP32 factor + FP64 refinement")
    ap.add_argument("--gram", default=None, choices=["ff", "fp64", "bf16"],
                    help="MinSR Gram of the step: float-float on the FP32 pipes (default with --prec fp32), "
                         "FP64 (default with --prec fp64), or split-BF16 tcgen05")
    return ap.parse_args()


def _config(w, ns, sweeps):
    # the same for both arms; each line's "dtype" gives the arithmetic it ran in
    return {"workload": f"{w['Lx']}x{w['Ly']} open Heisenberg J=1, D={w['D']}, chi={w['chi']}, "
                        f"N_s={ns} Metropolis exchange chains ({WORKLOAD})",
            "Lx": w["Lx"], "Ly": w["Ly"], "D": w["D"], "chi": w["chi"], "ns": ns,
            "sweeps_per_step": sweeps, "minsr": {"lambda": w["lam"], "rcond": w["rcond"], "tau": w["tau"]},
            "l2": "inputs larger than L2 (environment store and O exceed 129 MB)"}


# --------------------------------------------------------------------------------- CPU oracle
def _oracle_sample_run(nsamp, sweeps, seed_off=0):
    """The oracle as it stands on `nsamp` chains of the workload: `sweeps` sweeps, then
    psi / E_loc / O, then one MinSR step.  Returns seconds."""
    from paper_2503_12557_gb300 import inputs as I
    from oracle import energy, minsr, sampler
    w = I.WORKLOADS[WORKLOAD]
    lat = I.Lattice(w["Lx"], w["Ly"], w["d"], w["D"])
    th = I.peps_random(lat, w["seed_theta"], **w["init"])
    H = I.heisenberg(lat)
    S0 = I.configs_neel(lat, nsamp)
    t = time.perf_counter()
    S, _, _ = sampler.run_chains(th, S0, lat, w["chi"], "exchange", w["seed_chain"], sweeps, sweep0=seed_off)
    res = energy.evaluate(th, S, lat, w["chi"], H=H)
    minsr.minsr(res["O"].real, res["eloc"].real, lam=w["lam"], rcond=w["rcond"], tau=w["tau"])
    return time.perf_counter() - t


def _cpu_procs(nsamp, sweeps, reps=1, nproc=1):
    """Run the oracle in `nproc` concurrent single-threaded processes (each on its own `nsamp`
    chains, `reps` repetitions, chain seeds offset per process); returns, per repetition, the
    slowest process's seconds."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = []
    for p in range(nproc):
        code = ("import sys, json; sys.path.insert(0, %r); import bench; "
                "print(json.dumps([bench._oracle_sample_run(%d, %d, 1000 * %d + k) for k in range(%d)]))"
                % (ROOT, nsamp, sweeps, p, reps))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for pr in procs:
        o, e = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(f"oracle process failed: {e[-2000:]}")
        outs.append(json.loads(o.strip().splitlines()[-1]))
    return [max(o[k] for o in outs) for k in range(reps)]


def _ncores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(nsamp, sweeps):
    """The oracle as it stands on the host: one core, and every core (one single-threaded process
    per core, each on nsamp chains)."""
    one = _cpu_procs(nsamp, sweeps)[0]
    nc = _ncores()
    allc = _cpu_procs(nsamp, sweeps, nproc=nc)[0]
    return {"value": nc * nsamp / allc, "unit": "samples/s", "cores": nc, "kind": "oracle",
            "one_core": {"value": nsamp / one, "unit": "samples/s", "cores": 1},
            "sample": f"{nsamp} chains of the workload per process: {sweeps} sweeps + psi/E_loc/O + MinSR on them; "
                      f"{nc} concurrent single-threaded processes ({allc:.1f} s, the slowest), and one alone "
                      f"({one:.1f} s); nproc = {nc}"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2503_12557_gb300 import inputs as I
    w = I.WORKLOADS[WORKLOAD]
    ns = a.ns or w["ns"]
    nsamp = a.cpu_samples
    nc = _ncores()
    secs = _cpu_procs(nsamp, a.sweeps, reps=a.warmup + a.steps, nproc=nc)[a.warmup:]
    t = float(np.mean(secs))
    v = nc * nsamp / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(w, ns, a.sweeps),
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": nc, "kind": "oracle",
                             "sample": f"each step: {nsamp} chains of the workload ({a.sweeps} sweeps + psi/E_loc/O "
                                       f"+ MinSR) in each of {nc} concurrent single-threaded processes (nproc = {nc})"},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------- GPU
class _Clocks:
    def __init__(self, path):
        self.path = path
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                                       "-i", str(int(os.environ.get("LOCAL_RANK", "0")))],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            # nvidia-smi's start-up (NVML initialisation) can stall the GPU briefly: let it reach
            # its first reading before the timed region starts (at most 5 s)
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.p.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.05)
            time.sleep(0.3)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            self.p.wait()
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], f[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# DRAM bytes (read + write) of one sampler call of 2 sweeps in FP32 (the 31 kernel launches of the
# split sweep), from one ncu capture of such a call at 304 chains, scaled by the chains processed
# (each chain's environment rows and partials are its own traffic); None until such a capture of
# the current kernels exists.  profiles/sampler_split_heis8x8_D4_chi16_ns304.md: 1.192 GB per call
# of 2 sweeps over 304 chains (k_env one-side pass 0.223 GB, 16 k_sweep_moves 0.700 GB, 14
# k_env_row 0.269 GB).
_SAMPLER_CAPTURE = {"bytes": 1.1915e9, "chains": 304, "sweeps": 2}


def _measured_traffic(kernel, ns, sweeps, prec):
    """DRAM traffic of one call of the dominant kernel (set) from its ncu capture, or None where no
    capture of the current kernels at this precision and sweep count exists."""
    from paper_2503_12557_gb300 import peps as P
    c = _SAMPLER_CAPTURE
    if c and kernel == "sample" and prec == P.PREC_FP32 and sweeps == c["sweeps"]:
        return c["bytes"] * ns / c["chains"]
    return None


def _tau_chains(E, c=5.0):
    """Integrated autocorrelation time (1 + 2 sum_t rho(t), Sokal's window W >= c tau) of the
    local energy along the chains: E is steps x chains; the mean over the chains of each step is
    removed first (the parameters move between steps), rho(t) averages over every chain."""
    x = np.asarray(E, dtype=np.float64)
    x = x - x.mean(axis=1, keepdims=True)
    T = x.shape[0]
    var = np.mean(x * x)
    if var == 0.0 or T < 3:
        return 1.0
    rho = [np.mean(x[: T - t] * x[t:]) / var for t in range(T // 2 + 1)]
    tau = 1.0
    for W in range(1, len(rho)):
        tau = 1.0 + 2.0 * float(np.sum(rho[1:W + 1]))
        if W >= c * tau:
            break
    return max(tau, 1.0)


HEIS_BOUNDS = (-0.75, 0.25)  # the eigenvalues of S_i . S_j for one bond


def run_gpu(a):
    import tempfile

    import torch
    import torch.distributed as dist
    from paper_2503_12557_gb300 import build, costmodel, inputs as I, peps as P
    from paper_2503_12557_gb300.dist import CudaMinSROps, sharded_minsr
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(lrank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    w = I.WORKLOADS[WORKLOAD]
    lat = I.Lattice(w["Lx"], w["Ly"], w["d"], w["D"])
    ns = a.ns or w["ns"]                        # chains of this process (weak scaling)
    prec = P.PREC_FP32 if a.prec == "fp32" else P.PREC_FP64
    H = I.heisenberg(lat)
    nbonds = len(H["terms"])
    theta0 = I.peps_random(lat, w["seed_theta"], **w["init"])
    S0 = I.configs_neel(lat, ns)
    gram = {"fp64": 0, "bf16": 1, "ff": 2}[a.gram or ("ff" if a.prec == "fp32" else "fp64")]
    solve = {"fp64": 0, "fp32": 1, "ff": 2}[a.solve or ("ff" if a.prec == "fp32" else "fp64")]
    mask = P.ST_ZERO_NORM | P.ST_NONFINITE | P.ST_NOCONV   # samples left out of E_loc and MinSR
    seed = w["seed_chain"] + 7919 * rank                    # every process its own chains

    def make(prec_, ns_, gram_, solve_=0):
        h_ = P.PEPS(lat.Lx, lat.Ly, lat.d, lat.D, w["chi"], prec=prec_, max_samples=ns_, gram=gram_, solve=solve_)
        th_ = torch.as_tensor(theta0).cuda()
        h_.set_params(th_)
        h_.set_env_reuse(True)  # the evaluation takes the sampler's last environments (cached, unchanged S)
        return h_, th_

    h, theta = make(prec, ns, gram, solve)
    S = torch.as_tensor(S0).cuda()
    acc = torch.zeros(ns, dtype=torch.int64, device="cuda")
    O = torch.empty(ns, h.Np, dtype=h.odtype, device="cuda")
    stream = torch.cuda.current_stream()
    sweep_ctr = [0]
    info_hist = []
    ops = CudaMinSROps(h) if world > 1 else None

    def step(hh=h, th=theta, SS=S, accd=acc, O_out=O, ctr=sweep_ctr, hist=info_hist, ops_=ops):
        hh.sample(SS, P.MOVE_EXCHANGE, a.sweeps, seed=seed, sweep0=ctr[0], accepted=accd)
        ctr[0] += a.sweeps
        r = hh.evaluate(H, SS, O_out=O_out)
        wts = hh.status_weights(r["status"], mask)
        if ops_ is not None:
            dth, info = sharded_minsr(ops_, r["O"], r["eloc"], wts, lam=w["lam"], rcond=w["rcond"], tau=w["tau"])
        else:
            dth, info = hh.minsr_step(r["O"], r["eloc"], w=wts, lam=w["lam"], rcond=w["rcond"], tau=w["tau"])
        hh.apply_update(th, dth)
        hist.append(info)
        return r, dth

    # burn-in sweeps from the Neel start, untimed
    h.sample(S, P.MOVE_EXCHANGE, a.burnin, seed=seed, sweep0=0, accepted=acc)
    sweep_ctr[0] = a.burnin
    for i in range(a.warmup):
        if i == a.warmup - 1:
            h.timing(True)  # the library's event pool and counters come up outside the timed region
        r, _ = step()
        # the timed loop's reductions too: torch loads their kernels on first use
        eloc_warm = (r["eloc"][:, 0] * (r["status"] & mask == 0)).sum()
    torch.cuda.synchronize()
    h.last_status()
    # ---- timed region (device events on the launching stream)
    h.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    clk_path = os.path.join(tempfile.gettempdir(), f"peps_bench_clocks_rank{rank}.csv")
    with _Clocks(clk_path) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
        e0.record(stream)
        for k in range(a.steps):
            r, _ = step()
            res.append((r["eloc"], r["status"]))  # fresh tensors every step: no copy in the timed region
            marks[k].record(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms_total = e0.elapsed_time(e1)
    word = h.last_status()
    # full one-side environment passes of the timed sampler calls: sweeps alternate direction
    # (even ids down, odd up); a downward sweep, and an upward one that opens a call, need one
    s0 = a.burnin + a.warmup * a.sweeps
    sampler_passes = sum(1 for k in range(a.steps) for t in range(a.sweeps)
                         if (s0 + k * a.sweeps + t) % 2 == 0 or t == 0)
    step_ms = [e0.elapsed_time(marks[0])] + [marks[k - 1].elapsed_time(marks[k]) for k in range(1, a.steps)]
    ms_cls, launches, ctr = h.timing_read()
    h.timing(False)
    # ---- energies of the timed steps: flagged samples left out (as from MinSR), per-site means
    E = np.stack([e[:, 0].cpu().numpy() for e, _ in res])            # steps x chains
    ST = np.stack([st.cpu().numpy() for _, st in res])
    ok = (ST & mask) == 0
    e_site = [float(E[k][ok[k]].mean()) / lat.nsites for k in range(a.steps)]
    lo_b, hi_b = HEIS_BOUNDS[0] * nbonds / lat.nsites, HEIS_BOUNDS[1] * nbonds / lat.nsites
    tau = _tau_chains(E)
    # the last timed step's MinSR update against an FP64 Gram of the same O and E_loc
    dtheta_check = None
    if gram != 0 and world == 1:
        wl = h.status_weights(r["status"], mask)
        dth_last = h.minsr_step(r["O"], r["eloc"], w=wl, lam=w["lam"], rcond=w["rcond"], tau=w["tau"])[0].clone()
        h64g = P.PEPS(lat.Lx, lat.Ly, lat.d, lat.D, w["chi"], prec=prec, max_samples=2, gram=0, solve=0)
        dth64 = h64g.minsr_step(r["O"], r["eloc"], w=wl, lam=w["lam"], rcond=w["rcond"], tau=w["tau"])[0]
        dtheta_check = float((dth_last - dth64).norm() / dth64.norm())
        h64g.close()
    ms_step = ms_total / a.steps
    if world > 1:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = ns * world / (ms_step / 1e3)
    minsr_s = (ms_cls["minsr_gram"] + ms_cls["minsr_eig"] + ms_cls["minsr_other"]) / a.steps / 1e3
    # ---- roofline of the dominant kernel class
    peaks = _peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_derived = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 FMA pipes at the max SM clock
    # measured CUDA-core FMA peaks of this GPU (project probe, run after the timed region)
    fp32_peak = P.probe_fma(False)
    fp64_peak = P.probe_fma(True)
    alu_peak = fp32_peak if prec == P.PREC_FP32 else fp64_peak
    hwin, vwin = costmodel.heisenberg_windows(lat.Lx, lat.Ly, ns)
    # the Jacobi counters mix the sampler's and the environment kernel's SVDs; split them by SVD count
    # with environment reuse the evaluation contracts one side (the sampler left the other)
    env_sides = 1
    svd_env = a.steps * ns * env_sides * (lat.Lx - 2) * (lat.Ly - 1)
    svd_all = max(1, ctr["svds"])
    fe = min(1.0, svd_env / svd_all)
    flops = {
        "env": costmodel.env_flops(lat.Lx, lat.Ly, w["chi"], w["D"], ns * a.steps, env_sides, ctr["jacobi_sweeps"] * fe,
                                   ctr["jacobi_rotations"] * fe),
        "sample": costmodel.sample_flops(lat.Lx, lat.Ly, w["chi"], w["D"], ns, a.sweeps * a.steps,
                                         ctr["jacobi_sweeps"] * (1 - fe), ctr["jacobi_rotations"] * (1 - fe),
                                         passes=sampler_passes),
        "row": costmodel.row_kernel_flops(lat.Lx, lat.Ly, w["chi"], w["D"], ns * a.steps, True, hwin * a.steps),
        "pair": costmodel.pair_kernel_flops(lat.Lx, lat.Ly, w["chi"], w["D"], ns * a.steps, vwin * a.steps),
        "minsr_gram": costmodel.gram_flops(ns * world, h.Np) * a.steps / world,
    }
    dom = max(flops, key=lambda k: ms_cls.get(k, 0.0))
    dom_launch_ms = ms_cls[dom] / max(1, launches[dom])
    achieved = flops[dom] / max(1, launches[dom]) / (dom_launch_ms / 1e3) / 1e12
    # a Gram-dominated step: FP64 FMA peak, FP32 pipe peak (float-float) or the BF16 tensor peak
    gram_peak = {0: fp64_peak, 1: peaks.get("bf16_tflops", 1900.0), 2: fp32_peak}[gram]
    peak = gram_peak if dom == "minsr_gram" else alu_peak
    sampler_name = ("sampler call of alternating sweeps (k_env one-side pass where a sweep needs one, then "
                    "k_sweep_moves and k_env_row per row)" if prec == P.PREC_FP32 else "k_sample")
    roof = {"kernel": {"env": "k_env", "sample": sampler_name, "row": "k_row", "pair": "k_pair",
                       "minsr_gram": "k_gram"}[dom],
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            # per launch, as achieved: the call's bytes spread over the launches the call made
            "traffic": (None if _measured_traffic(dom, ns, a.sweeps, prec) is None else
                        _measured_traffic(dom, ns, a.sweeps, prec) * a.steps / max(1, launches[dom])),
            "peak_source": ("measured: peps_probe_fma FP32 (derived 152 SMs x 128 lanes x 2 x max clock = %.1f)"
                            % fp32_derived if peak == fp32_peak else
                            "measured: peps_probe_fma FP64" if peak == fp64_peak else "MEASURED_PEAKS bf16_tflops"),
            "algorithmic_tflop_per_launch": flops[dom] / max(1, launches[dom]) / 1e12,
            "launch_ms": dom_launch_ms,
            "counting": ("the loop nests' flops at the full bond chi (products, QR, sandwiches) plus the Jacobi "
                         "rotations and sweeps the library counted; the kernels skip the exact-zero rows and "
                         "columns near the open edge, so the executed flops are fewer")}
    # library launches per step: the classes' counts plus the memsets of evaluate / minsr
    gpu_launches = int(sum(launches.values())) + 4 * a.steps
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == P.PREC_FP32 else "f64", "data": "synthetic",
            "config": _config(w, ns, a.sweeps), "step_ms": step_ms, "minsr_step_s": minsr_s,
            "minsr": {"gram": {0: "FP64 CUDA cores", 1: "split-BF16 tcgen05",
                               2: "float-float pairs on the FP32 pipes"}[gram],
                      "solve": {0: "FP64 Cholesky", 1: "FP32 Cholesky + FP64 refinement",
                                2: "float-float Cholesky + FP64 refinement"}[solve],
                      "sharded_over_processes": world > 1,
                      "gram_ms": ms_cls["minsr_gram"] / a.steps, "solve_ms": ms_cls["minsr_eig"] / a.steps,
                      "gram_tflops_algorithmic": (flops["minsr_gram"] / a.steps /
                                                  max(1e-9, ms_cls["minsr_gram"] / a.steps / 1e3) / 1e12),
                      "gram_pipe_frac": (costmodel.gram_pipe_flops(ns, h.Np, gram) /
                                         max(1e-9, ms_cls["minsr_gram"] / a.steps / 1e3) / 1e12 / gram_peak),
                      "dtheta_rel_diff_vs_fp64_gram_and_solve": dtheta_check,
                      "last_info": [float(x) for x in info_hist[-1].cpu()]},
            "kernel_ms_per_step": {k: v / a.steps for k, v in ms_cls.items()},
            "jacobi": {"svds": int(ctr["svds"]), "sweeps_per_svd": ctr["jacobi_sweeps"] / svd_all,
                       "rotations_per_svd": ctr["jacobi_rotations"] / svd_all},
            "roofline": roof, "alu_peaks_measured_tflops": {"fp32": fp32_peak, "fp64": fp64_peak},
            "gpu_launches": gpu_launches, "clocks": clk.summary(),
            "acceptance": float(acc.sum().item()) / max(1.0, ns * (sweep_ctr[0]) * (2 * lat.Lx * lat.Ly - lat.Lx - lat.Ly) * 0.5),
            "energy": {"eloc_mean_per_site": e_site,
                       "heisenberg_bounds_per_site": [lo_b, hi_b],
                       "all_steps_within_bounds": bool(all(lo_b <= x <= hi_b for x in e_site)),
                       "samples_left_out_per_step": [int((~ok[k]).sum()) for k in range(a.steps)],
                       "status_word": word,
                       "tau_int_eloc": tau,
                       "tau_convention": "1 + 2 sum_t rho(t) over MinSR steps of 2 sweeps (effective samples = N / tau)"},
            "energy_converged_samples_per_s": value / tau}
    # ---- the plain FP64 GPU path on the same workload and chain count (after the timed region)
    if a.fp64_steps > 0 and prec == P.PREC_FP32 and world == 1:
        line["fp64_plain"] = _fp64_plain(a, P, make, theta, S, H, ns, seed, sweep_ctr[0], mask, tau, value, lat)
    # ---- end to end through the public API with host buffers
    if not a.no_e2e:
        th_host = torch.empty(h.Np, dtype=torch.float64).pin_memory()
        th_host.copy_(theta.cpu())
        S_host = torch.empty(ns, lat.nsites, dtype=torch.uint8).pin_memory()
        S_host.copy_(S.cpu())
        dth_host = torch.empty(h.Np, dtype=torch.float64).pin_memory()
        el_host = torch.empty(ns, 2, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(a.steps):
            theta.copy_(th_host, non_blocking=True)
            S.copy_(S_host, non_blocking=True)
            h.set_params(theta)
            r, dth = step()
            dth_host.copy_(dth, non_blocking=True)
            el_host.copy_(r["eloc"], non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = f0.elapsed_time(f1) / a.steps
        if world > 1:
            t = torch.tensor([e2e_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        line["e2e"] = {"value": ns * world / (e2e_ms / 1e3), "unit": "samples/s",
                       "h2d_bytes_per_step": h.Np * 8 + ns * lat.nsites,
                       "d2h_bytes_per_step": h.Np * 8 + ns * 16}
    if rank == 0 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a.cpu_samples, a.sweeps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


def _fp64_plain(a, P, make, theta, S_fp32, H, ns, seed, sweep0, mask, tau, value32, lat):
    """The plain FP64 GPU path (FP64 contractions, FP64 Gram, FP64 Cholesky) at the same chain count,
    from the FP32 run's parameters and configurations: samples/s of a.fp64_steps steps (CUDA
    events), and the per-site energy of the FP32 and FP64 evaluations of the same configurations
    at the same parameters (equal energy error: within the 1e-4 per site gate, so both reach the
    same error with the same samples)."""
    import torch
    w = I_workload()
    h64, th64 = make(P.PREC_FP64, ns, 0)
    h32e, th32 = make(P.PREC_FP32, ns, 2)
    th64.copy_(theta)
    th32.copy_(theta)
    h64.set_params(th64)
    h32e.set_params(th32)
    S = S_fp32.clone()
    # the same configurations through both precisions (no parameter update in between)
    r32 = h32e.evaluate(H, S)
    r64 = h64.evaluate(H, S)
    ok = ((r32["status"] & mask) == 0) & ((r64["status"] & mask) == 0)
    # O rows: largest |O32 - O64| over each row's largest |O64|
    dO_all = ((r32["O"].double() - r64["O"]).abs().amax(dim=1) /
              r64["O"].abs().amax(dim=1).clamp_min(1e-300))[ok].cpu().numpy()
    del r32["O"], r64["O"]
    d_e = float(((r32["eloc"][:, 0] - r64["eloc"][:, 0])[ok]).mean().abs()) / lat.nsites
    dl_all = (r32["logabs"] - r64["logabs"])[ok].abs().double().cpu().numpy()
    de_all = ((r32["eloc"][:, 0] - r64["eloc"][:, 0])[ok].abs() / lat.nsites).double().cpu().numpy()
    d_l = float(dl_all.max())
    h32e.close()
    acc = torch.zeros(ns, dtype=torch.int64, device="cuda")
    O = torch.empty(ns, h64.Np, dtype=torch.float64, device="cuda")
    ctr = [sweep0]

    def step():
        h64.sample(S, P.MOVE_EXCHANGE, a.sweeps, seed=seed, sweep0=ctr[0], accepted=acc)
        ctr[0] += a.sweeps
        r = h64.evaluate(H, S, O_out=O)
        wts = h64.status_weights(r["status"], mask)
        dth, _ = h64.minsr_step(r["O"], r["eloc"], w=wts, lam=w["lam"], rcond=w["rcond"], tau=w["tau"])
        h64.apply_update(th64, dth)

    # warm-up on a few chains (module load, workspaces), then the timed steps at full size
    h64.sample(S[:152].clone(), P.MOVE_EXCHANGE, 1, seed=seed, sweep0=0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.fp64_steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.fp64_steps
    v64 = ns / (ms / 1e3)
    h64.close()
    return {"value": v64, "unit": "samples/s", "ms_per_step": ms, "steps": a.fp64_steps,
            "what": "FP64 contractions, FP64 Gram, FP64 Cholesky, same chains and step",
            "energy_converged_samples_per_s": v64 / tau,
            "fp32_vs_fp64_same_configs": {"mean_eloc_diff_per_site": d_e, "max_dlogpsi": d_l,
                                          "median_dlogpsi": float(np.median(dl_all)),
                                          "p99_dlogpsi": float(np.quantile(dl_all, 0.99)),
                                          "samples_dlogpsi_over_1e-5": int((dl_all > 1e-5).sum()),
                                          "samples_dlogpsi_over_1e-3": int((dl_all > 1e-3).sum()),
                                          "max_deloc_per_site": float(de_all.max()),
                                          "median_deloc_per_site": float(np.median(de_all)),
                                          "samples_deloc_per_site_over_1e-4": int((de_all > 1e-4).sum()),
                                          "median_dO_row_rel": float(np.median(dO_all)),
                                          "p99_dO_row_rel": float(np.quantile(dO_all, 0.99)),
                                          "max_dO_row_rel": float(dO_all.max()),
                                          "samples": int(ok.sum().item()),
                                          "gate_per_site": 1e-4, "equal_energy_error": d_e <= 1e-4},
            "fp32_over_fp64_energy_converged": value32 / v64}


def I_workload():
    from paper_2503_12557_gb300 import inputs as I
    return I.WORKLOADS[WORKLOAD]


def run_learned(a):
    """12x12 Rydberg array (Omega = 1, R_b = 1.7, V0 / r^6 for r <= 4; D = 4, chi = 24, tensors drawn
    as for the 8x8 workload; FP32 contractions, bf16 network), for every detuning delta in
    {0, 1, 2, 3}: N_s chains thermalised by local flips, the network trained on the sampler's own
    (S_t, S_{t+2}) pairs, then two arms from the same configurations, each followed by psi and
    E_loc of every chain at every step:
      local: one single-flip sweep per step;
      mixed: one single-flip sweep plus one network move per step (learned.run_mixed's kernel).
    Per arm: seconds per step (sampling alone, and with the energy evaluation), tau of E_loc along
    the chains (1 + 2 sum rho), energy-converged samples/s = N_s / (t tau), and the energy error
    at equal wall time, sigma_E sqrt(t tau / (N_s x 1 s)) per site for one second of sampling
    plus evaluation.  The gain of the network is local's error over mixed's (above 1: the
    network helps)."""
    import torch
    from paper_2503_12557_gb300 import build, inputs as I, learned as Lr, peps as P
    build.build()
    w = I.WORKLOADS["rydberg12x12_D4_chi24"]
    lat = I.Lattice(w["Lx"], w["Ly"], w["d"], w["D"])
    ns = a.ns or 4096
    T = max(a.steps, 12)
    theta = torch.as_tensor(I.peps_random(lat, w["seed_theta"], **w["init"])).cuda()
    out = {"mode": "learned", "workload": f"12x12 Rydberg, D=4, chi=24, {ns} chains, {T} steps per arm",
           "deltas": {}}

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, r

    h = P.PEPS(lat.Lx, lat.Ly, 2, lat.D, w["chi"], prec=P.PREC_FP32, max_samples=ns)
    h.set_params(theta)
    for delta in (0.0, 1.0, 2.0, 3.0):
        H = I.rydberg(lat, delta=delta)
        S = torch.zeros(ns, lat.nsites, dtype=torch.uint8, device="cuda")
        S, _, _ = Lr.run_local(h, S, max(a.burnin, 10), seed=w["seed_chain"], sweep0=0)
        S_in, S_out, S = Lr.collect_pairs(h, S, 4, 2, seed=w["seed_chain"] + 1, sweep0=1000)
        prop = P.Proposal(lat.Lx, lat.Ly, I.proposal_init(5), C=16, wprec=1)
        t_train, losses = timed(lambda: Lr.train(prop, S_in, S_out, 200, lr=3e-3, batch=4096))
        res = {"train_s": t_train, "loss_first_last": [losses[0], losses[-1]]}
        for arm in ("local", "mixed"):
            S_arm = S.clone()
            acc_l = torch.zeros(ns, dtype=torch.int64, device="cuda")
            acc_n = torch.zeros(ns, dtype=torch.int64, device="cuda")
            E = []
            t_sample = t_eval = 0.0
            lpsi = h.amplitudes(S_arm)[0] if arm == "mixed" else None
            for t in range(T):
                def samp():
                    h.sample(S_arm, P.MOVE_FLIP, 1, seed=w["seed_chain"] + 2, sweep0=2000 + t, accepted=acc_l)
                    if arm == "mixed":
                        lp, _, _ = h.amplitudes(S_arm)
                        h.sample_learned(prop, S_arm, lp, seed=w["seed_chain"] + 3, step=2000 + t, accepted=acc_n)
                ts, _ = timed(samp)
                te, r = timed(lambda: h.evaluate(H, S_arm, want_O=False))
                t_sample += ts
                t_eval += te
                E.append(r["eloc"][:, 0].cpu().numpy() / lat.nsites)
            E = np.array(E)
            tau = _tau_chains(E)
            ts, te = t_sample / T, t_eval / T
            sig = float(E.std())
            res[arm] = {"s_per_step_sampling": ts, "s_per_step_with_eval": ts + te, "tau_int_eloc": tau,
                        "E_per_site": float(E.mean()), "sigma_E_per_site": sig,
                        "energy_converged_samples_per_s": ns / ((ts + te) * tau),
                        "err_per_site_at_1s": sig * float(np.sqrt((ts + te) * tau / ns)),
                        "local_acceptance": float(acc_l.sum().item()) / (ns * T * lat.nsites)}
            if arm == "mixed":
                res[arm]["network_acceptance"] = float(acc_n.sum().item()) / (ns * T)
        res["gain_err_local_over_mixed"] = res["local"]["err_per_site_at_1s"] / res["mixed"]["err_per_site_at_1s"]
        out["deltas"][str(delta)] = res
        print(json.dumps({"delta": delta, **res}), flush=True)
    h.close()
    print(json.dumps(out), flush=True)


def run_gram(a):
    """MinSR step on a synthetic O (N_s x N_p, entries N(0,1) plus a 0.1 column offset so that
    centring matters) with the FP64 CUDA-core Gram, the split-BF16 tcgen05 Gram and the float-float
    Gram on the FP32 pipes; reports each Gram's time, its pipe rate (3 BF16 products, 13 FP32
    operations per algorithmic multiply-add) and the relative difference of each dtheta from the
    FP64 one."""
    import torch
    from paper_2503_12557_gb300 import build, inputs as I, peps as P
    build.build()
    ns = a.ns or 16384
    lat = I.Lattice(14, 14, 2, 4)  # N_p = 80 000, the smallest square open lattice above 73 728
    peaks = _peaks()
    out = {"mode": "gram", "ns": ns}
    res = {}
    g = torch.Generator(device="cuda").manual_seed(5005)
    for gram, tag in ((1, "tcgen05_split_bf16"), (2, "float_float_fp32"), (0, "fp64_cuda_cores")):
        h = P.PEPS(lat.Lx, lat.Ly, 2, lat.D, lat.D, prec=P.PREC_FP64, max_samples=2, gram=gram)
        out["np"] = h.Np
        g.manual_seed(5005)
        O = torch.randn(ns, h.Np, dtype=torch.float64, device="cuda", generator=g)
        O += 0.1 * torch.randn(h.Np, dtype=torch.float64, device="cuda", generator=g)
        e = torch.zeros(ns, 2, dtype=torch.float64, device="cuda")
        e[:, 0] = torch.randn(ns, dtype=torch.float64, device="cuda", generator=g) - 3.0
        reps = 1 if gram == 0 else 3
        h.minsr_step(O, e, lam=1.0, tau=0.1)  # warm-up (allocations)
        h.timing(True)
        for _ in range(reps):
            dth, info = h.minsr_step(O, e, lam=1.0, tau=0.1)
        h.last_status()
        ms, la, _ = h.timing_read()
        h.timing(False)
        gram_ms = ms["minsr_gram"] / reps
        mac = ns * (ns + 1) / 2 * h.Np  # algorithmic multiply-adds of one triangle
        r = {"gram_ms": gram_ms, "solve_ms": ms["minsr_eig"] / reps, "step_s": sum(ms.values()) / reps / 1e3,
             "lambda": 1.0, "warning": h.last_warning}
        if gram == 1:
            tflops = 3 * 2 * mac / (gram_ms / 1e3) / 1e12
            r["tensor_tflops_bf16"] = tflops
            r["roofline"] = {"bound": "tensor", "achieved": tflops, "peak": peaks.get("bf16_tflops", 1900.0),
                             "unit": "TFLOP/s", "frac": tflops / peaks.get("bf16_tflops", 1900.0)}
        elif gram == 2:
            r["fp32_pipe_tflops"] = 13 * 2 * mac / (gram_ms / 1e3) / 1e12
            r["fp32_pipe_frac_of_measured_fma_peak"] = r["fp32_pipe_tflops"] / P.probe_fma(False)
        else:
            r["fp64_tflops"] = 2 * mac / (gram_ms / 1e3) / 1e12
        res[tag] = dth
        out[tag] = r
        del O
        h.close()
        torch.cuda.empty_cache()
    for tag in ("tcgen05_split_bf16", "float_float_fp32"):
        d = res[tag] - res["fp64_cuda_cores"]
        out[tag]["dtheta_rel_diff"] = float(d.norm() / res["fp64_cuda_cores"].norm())
    print(json.dumps(out), flush=True)


def run_batch(a):
    """Ragged multi-instance batch: 64 independent open Heisenberg PEPS with (L, D) drawn uniformly
    from {6, 8, 10, 12} x {3, 4, 5} (seed 5005), chi = D^2, tensors drawn as for the 8x8 workload,
    N_s configurations each (uniform S^z = 0); psi, E_loc and O of every instance by one
    persistent launch over the (instance, sample) queue, recorded in a CUDA graph.  Reports
    samples/s of the graph replay and of the same evaluations issued one handle after another,
    and (with --autotune) the batch budget the autotuner chose."""
    import torch
    from paper_2503_12557_gb300 import build, inputs as I, peps as P
    build.build()
    ns = a.ns or 256
    rng = np.random.default_rng(5005)
    shapes = [(int(rng.choice([6, 8, 10, 12])), int(rng.choice([3, 4, 5]))) for _ in range(64)]
    prec = P.PREC_FP32 if a.prec == "fp32" else P.PREC_FP64
    items = []
    for k, (L, D) in enumerate(shapes):
        lat = I.Lattice(L, L, 2, D)
        h = P.PEPS(L, L, 2, D, D * D, prec=prec, max_samples=ns)
        h.set_params(torch.as_tensor(I.peps_random(lat, 5005 + k, **I.WORKLOADS[WORKLOAD]["init"])).cuda())
        S = torch.as_tensor(I.configs_uniform_sz0(lat, ns, 6005 + k)).cuda()
        items.append((h, I.heisenberg(lat), S, True))
    out = {"mode": "batch", "instances": 64, "ns_per_instance": ns, "precision": a.prec,
           "shapes": {f"{L}x{L}_D{D}": sum(1 for s in shapes if s == (L, D)) for (L, D) in sorted(set(shapes))}}
    # one instance after another (eager), then the recorded graph
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        outs = [h.evaluate(H, S, want_O=True) for (h, H, S, _) in items]  # warm-up
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            outs = [h.evaluate(H, S, want_O=True) for (h, H, S, _) in items]
        e1.record(stream)
        stream.synchronize()
    eager_ms = e0.elapsed_time(e1) / a.steps
    kb = 0
    if a.autotune:
        # the budget is chosen on the first 32 samples of every instance (the full batch at
        # 2048 samples takes minutes per launch), then used for the full one
        sub = [(h, H, S[:min(32, S.shape[0])].contiguous(), wo) for (h, H, S, wo) in items]
        tb = P.Batch(sub, stream=stream, autotune=True)
        kb = tb.budget_kb
        tb.close()
    batch = P.Batch(items, stream=stream, budget_kb=kb)
    out["batch_budget_kb"] = kb or "default"
    for _ in range(a.warmup):
        batch.launch()
    stream.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(a.steps):
        batch.launch()
    f1.record(stream)
    stream.synchronize()
    graph_ms = f0.elapsed_time(f1) / a.steps
    same = all(torch.equal(o["logabs"], r["logabs"]) and torch.equal(o["eloc"], r["eloc"])
               for o, r in zip(batch.out, outs))
    tot = 64 * ns
    out.update({"graph_ms": graph_ms, "eager_ms": eager_ms, "graph_samples_per_s": tot / (graph_ms / 1e3),
                "eager_samples_per_s": tot / (eager_ms / 1e3),
                "graph_equals_eager": bool(same)})
    print(json.dumps(out), flush=True)


def run_complex(a):
    """10x10 open J1-J2-chiral model (J1 = 1, J2 = 0.5, chiral J_chi = 0.3 on every elementary
    triangle) on a complex PEPS, D = 6, chi = 36, entries complex Gaussian with std 0.3 (real and
    imaginary parts N(0, 0.045); mean-zero tensors, so the truncation error is large: this measures
    throughput and the reduced-precision error, not physics), N_s uniform S^z = 0 configurations:
    one exchange sweep, psi / E_loc / O, and one MinSR step with
    the pseudo-inverse cutoff 1e-8.  complex64 contractions; a complex128 handle on the first 8
    configurations gives the reduced-precision error."""
    import torch
    from paper_2503_12557_gb300 import build, inputs as I, peps as P
    build.build()
    ns = a.ns or 304
    lat = I.Lattice(10, 10, 2, 6)
    th = torch.as_tensor(I.peps_random(lat, 1003, scale=0.3, complex_=True)).cuda()
    H = I.j1j2_chiral(lat)
    S = torch.as_tensor(I.configs_uniform_sz0(lat, ns, 2003)).cuda()
    h = P.PEPS(10, 10, 2, 6, 36, prec=P.PREC_FP32, max_samples=ns, cplx=True)
    h.set_params(th)
    out = {"mode": "complex", "workload": "10x10 J1-J2-chiral, complex PEPS D=6 chi=36", "ns": ns, "np": h.Np}
    r = h.evaluate(H, S[:8])  # warm-up
    torch.cuda.synchronize()
    h.timing(True)
    t0 = time.perf_counter()
    h.sample(S, move=P.MOVE_EXCHANGE, nsweeps=1, seed=3003)
    r = h.evaluate(H, S)
    dth, info = h.minsr_step(r["O"], r["eloc"], lam=0.0, rcond=1e-8, tau=0.05)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms, la, ctr = h.timing_read()
    h.timing(False)
    eval_ms = ms["env"] + ms["row"] + ms["pair"] + ms["combine"]
    out.update({"sweep_ms": ms["sample"], "eval_ms": eval_ms, "minsr_s": (ms["minsr_gram"] + ms["minsr_eig"] + ms["minsr_other"]) / 1e3,
                "eval_samples_per_s": ns / (eval_ms / 1e3), "step_wall_s": wall, "minsr_info": [float(x) for x in info.cpu()],
                "status_nonzero": int((r["status"] != 0).sum().item())})
    h64 = P.PEPS(10, 10, 2, 6, 36, prec=P.PREC_FP64, max_samples=8, cplx=True)
    h64.set_params(th)
    r64 = h64.evaluate(H, S[:8])
    torch.cuda.synchronize()
    dl = (r["logabs"][:8] - r64["logabs"]).abs().max().item()
    e32 = torch.complex(r["eloc"][:8, 0], r["eloc"][:8, 1])
    e64 = torch.complex(r64["eloc"][:, 0], r64["eloc"][:, 1])
    out["complex64_vs_complex128"] = {"max_dlogpsi": dl, "max_deloc_per_site": ((e32 - e64).abs().max().item()) / 100}
    print(json.dumps(out), flush=True)


def run_bound(a):
    """Variational-bound estimator on the bench workload (8x8 open Heisenberg, D=4, chi=16,
    biased Gaussian tensors) with the cut in the middle (i = 4): N_s configurations after
    a.burnin exchange sweeps from the Neel state; the fast estimator (ratios from the
    neighbouring environments) and E_loc^bound on the same configurations, their times, the
    rebuilt row steps per sample, and the elementwise difference <E_bound - E_loc>."""
    import numpy as np
    import torch
    from paper_2503_12557_gb300 import build, inputs as I, peps as P
    build.build()
    w = I.WORKLOADS[WORKLOAD]
    lat = I.Lattice(w["Lx"], w["Ly"], w["d"], w["D"])
    ns = a.ns or 1216
    cut = lat.Lx // 2
    prec = P.PREC_FP32 if a.prec == "fp32" else P.PREC_FP64
    H = I.heisenberg(lat)
    h = P.PEPS(lat.Lx, lat.Ly, lat.d, lat.D, w["chi"], prec=prec, max_samples=ns)
    h.set_params(torch.as_tensor(I.peps_random(lat, w["seed_theta"], **w["init"])).cuda())
    S = torch.as_tensor(I.configs_neel(lat, ns)).cuda()
    h.sample(S, P.MOVE_EXCHANGE, max(a.burnin, 4), seed=w["seed_chain"])
    h.local_energy_bound(H, S[:8], cut)  # warm-up
    torch.cuda.synchronize()
    h.timing(True)
    fast = h.evaluate(H, S, want_O=False)
    b = h.local_energy_bound(H, S, cut)
    torch.cuda.synchronize()
    ms, la, _ = h.timing_read()
    h.timing(False)
    # rebuilt row steps per sample: every antiparallel bond rebuilds the rows between the
    # first row it changes and the cut, on its side of the cut
    Sh = S.cpu().numpy().astype(np.int64)
    steps = np.zeros(ns)
    for sites, _ in H["terms"]:
        i, j = sites
        anti = Sh[:, i] != Sh[:, j]
        ri, rj = i // lat.Ly, j // lat.Ly
        up = [r for r in (ri, rj) if r < cut]
        lo = [r for r in (ri, rj) if r >= cut]
        n = (cut - min(up) if up else 0) + (max(lo) - cut + 1 if lo else 0)
        steps += anti * n
    ef = fast["eloc"][:, 0].double().cpu().numpy()
    eb = b["eloc"][:, 0].double().cpu().numpy()
    diff = eb - ef
    env_ms_per_rowstep = ms["env"] / 2 / (ns * 2 * (lat.Lx - 1))   # two env passes, Lx-1 rows per side
    out = {"mode": "bound", "workload": f"8x8 open Heisenberg, D=4, chi=16, N_s={ns}, cut i={cut}",
           "precision": a.prec, "bound_kernel_ms": ms["bound"], "bound_total_ms": ms["bound"] + ms["env"] / 2 + ms["combine"] / 2,
           "fast_eval_ms": ms["env"] / 2 + ms["row"] + ms["pair"] + ms["combine"] / 2,
           "bound_samples_per_s": ns / ((ms["bound"] + ms["env"] / 2) / 1e3),
           "fast_samples_per_s": ns / ((ms["env"] / 2 + ms["row"] + ms["pair"]) / 1e3),
           "rebuilt_row_steps_per_sample": float(steps.mean()),
           "bound_ms_per_row_step": ms["bound"] / max(1.0, float(steps.sum())),
           "env_ms_per_row_step": env_ms_per_rowstep,
           "E_fast_per_site": float(ef.mean() / lat.nsites), "E_bound_per_site": float(eb.mean() / lat.nsites),
           "mean_diff_bound_minus_fast": float(diff.mean()), "stderr_diff": float(diff.std() / np.sqrt(ns)),
           "status_nonzero": int((b["status"] != 0).sum().item())}
    print(json.dumps(out), flush=True)


def run_rotated(a):
    """Rotated-basis (unbiased) energy estimator on the bench workload's PEPS (8x8 open
    Heisenberg, D=4, chi=16, biased Gaussian tensors): the PEPS rotated into the x, y and z
    eigenbases of the spin (complex handle), N_s flip chains per basis for a.burnin (at least
    10) sweeps, the diagonal part of H averaged per basis; beside it the fast estimator on
    exchange chains of the unrotated PEPS.  Times per basis from CUDA events."""
    import numpy as np
    import torch
    from paper_2503_12557_gb300 import build, estimators, inputs as I, peps as P
    build.build()
    w = I.WORKLOADS[WORKLOAD]
    lat = I.Lattice(w["Lx"], w["Ly"], w["d"], w["D"])
    ns = a.ns or 1216
    sweeps = max(a.burnin, 10)
    prec = P.PREC_FP32 if a.prec == "fp32" else P.PREC_FP64
    th = torch.as_tensor(I.peps_random(lat, w["seed_theta"], **w["init"])).cuda()
    bonds = I.spin_bonds(lat)
    S0 = I.configs_uniform(lat, ns, w["seed_S"])
    hc = P.PEPS(lat.Lx, lat.Ly, 2, lat.D, w["chi"], prec=prec, max_samples=ns, cplx=True)
    estimators.rotated_basis_energy(lat.Lx, lat.Ly, lat.D, w["chi"], th, bonds, S0[:8], burn_in=1, handle=hc)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    e, se, per = estimators.rotated_basis_energy(lat.Lx, lat.Ly, lat.D, w["chi"], th, bonds, S0, burn_in=sweeps,
                                                 seed=w["seed_chain"], handle=hc)
    e1.record()
    torch.cuda.synchronize()
    ms_rot = e0.elapsed_time(e1)
    hr = P.PEPS(lat.Lx, lat.Ly, 2, lat.D, w["chi"], prec=prec, max_samples=ns)
    hr.set_params(th)
    S = torch.as_tensor(I.configs_neel(lat, ns)).cuda()
    hr.sample(S, P.MOVE_EXCHANGE, sweeps, seed=w["seed_chain"])
    r = hr.evaluate(I.heisenberg(lat), S, want_O=False)
    ef = r["eloc"][:, 0].double()
    out = {"mode": "rotated", "workload": f"8x8 open Heisenberg, D=4, chi=16, N_s={ns} flip chains per basis, "
                                          f"{sweeps} sweeps", "precision": a.prec,
           "E_rotated_per_site": e / lat.nsites, "stderr_per_site": se / lat.nsites,
           "per_basis": [{"basis": b, "mean": m, "stderr": s_, "acceptance": acc} for b, (m, s_, acc) in zip("xyz", per)],
           "E_fast_per_site_exchange_chains": float(ef.mean()) / lat.nsites,
           "stderr_fast_per_site": float(ef.std() / np.sqrt(ns)) / lat.nsites,
           "rotated_ms_total": ms_rot, "rotated_samples_per_s": 3 * ns / (ms_rot / 1e3)}
    print(json.dumps(out), flush=True)


def run_direct(a):
    """Direct sampling on the bench workload (8x8 open Heisenberg, D=4, chi=16, biased Gaussian
    tensors): double-layer environments at chi_d = D = 4 (the paper's D_c^double ~ D), N_s
    independent configurations drawn row by row, then psi and E_loc of the drawn
    configurations; the importance-weighted energy with weights |psi|^2 / p, its effective
    sample size, and the times of each part (CUDA events of the library's timing record)."""
    import numpy as np
    import torch
    from paper_2503_12557_gb300 import build, inputs as I, peps as P
    build.build()
    w = I.WORKLOADS[WORKLOAD]
    lat = I.Lattice(w["Lx"], w["Ly"], w["d"], w["D"])
    ns = a.ns or 4096
    chid = lat.D
    prec = P.PREC_FP32 if a.prec == "fp32" else P.PREC_FP64
    H = I.heisenberg(lat)
    h = P.PEPS(lat.Lx, lat.Ly, lat.d, lat.D, w["chi"], prec=prec, max_samples=ns)
    h.set_params(torch.as_tensor(I.peps_random(lat, w["seed_theta"], **w["init"])).cuda())
    h.direct_prepare(chid)
    h.direct_sample(min(ns, 8), seed=w["seed_chain"], draw=0)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    h.direct_prepare(chid)
    e1.record()
    torch.cuda.synchronize()
    prep_ms = e0.elapsed_time(e1)
    h.timing(True)
    S, lp, st = h.direct_sample(ns, seed=w["seed_chain"], draw=1)
    r = h.evaluate(H, S, want_O=False)
    torch.cuda.synchronize()
    ms, la, _ = h.timing_read()
    h.timing(False)
    lw = (2 * r["logabs"] - lp).cpu().numpy()
    e = r["eloc"][:, 0].cpu().numpy()
    wt = np.exp(lw - lw.max())
    wt /= wt.sum()
    est = float(np.sum(wt * e))
    ess = float(1.0 / np.sum(wt ** 2))
    out = {"mode": "direct", "workload": f"8x8 open Heisenberg, D=4, chi=16, chi_d={chid}, N_s={ns}",
           "precision": a.prec, "double_layer_prepare_ms": prep_ms, "direct_sample_ms": ms["direct"], "eval_ms": ms["env"] + ms["row"] + ms["pair"] + ms["combine"],
           "direct_samples_per_s": ns / (ms["direct"] / 1e3), "launches": {"direct": la["direct"]},
           "E_weighted_per_site": est / lat.nsites,
           "stderr_per_site": float(np.sqrt(np.sum(wt ** 2 * (e - est) ** 2))) / lat.nsites,
           "ess": ess, "ess_fraction": ess / ns, "ess_per_s": ess / ((ms["direct"] + ms["env"] + ms["row"] + ms["pair"]) / 1e3),
           "status_nonzero": int((st != 0).sum().item()), "distinct_configurations": int(len(set(map(bytes, S.cpu().numpy()))))}
    print(json.dumps(out), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode == "learned":
        run_learned(a)
    elif a.mode == "gram":
        run_gram(a)
    elif a.mode == "batch":
        run_batch(a)
    elif a.mode == "complex":
        run_complex(a)
    elif a.mode == "bound":
        run_bound(a)
    elif a.mode == "rotated":
        run_rotated(a)
    elif a.mode == "direct":
        run_direct(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
