"""Variational optimisation loop around the C library: Metropolis sweeps, psi / E_loc / O of every
chain, one MinSR step and the parameter update per iteration (the paper's imaginary-time
evolution with the minimum-step stochastic reconfiguration, Eq. (tdvp_fast)), with per-step
metrics written as JSON lines and checkpoints that resume the same trajectory.

Every random number the chains draw comes from the counter-based generator inside the sampler
kernel, keyed by (seed, sweep id, chain), so a resumed run that restores theta, the chain
configurations and the sweep counter repeats the uninterrupted run exactly.

sampler="direct" replaces the chains by the paper's direct sampling (Sec. "On Direct
Sampling"): every step rebuilds the double-layer environments for the current parameters,
draws N_s independent configurations (draw round = step number), and weights them by
|psi(S)|^2 / p(S) in the energy and in the MinSR step (self-normalised importance sampling).
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import peps as P
from .learned import tau_int


class VMC:
    """One optimisation: a handle, its parameters and N_s Metropolis chains on the device."""

    def __init__(self, Lx, Ly, d, D, chi, H, theta0, S0, prec=P.PREC_FP64, move=P.MOVE_EXCHANGE, seed=1,
                 lam=1e-4, rcond=0.0, tau=0.05, sweeps_per_step=2, gram=0, solve=0, sampler="metropolis", chi_double=None):
        if sampler not in ("metropolis", "direct"):
            raise ValueError("sampler must be 'metropolis' or 'direct'")
        self.cfg = dict(Lx=Lx, Ly=Ly, d=d, D=D, chi=chi, prec=prec, move=move, seed=seed, lam=lam, rcond=rcond,
                        tau=tau, sweeps_per_step=sweeps_per_step, gram=gram, solve=solve, sampler=sampler,
                        chi_double=int(chi_double if chi_double is not None else D))
        self.H = H
        self.h = P.PEPS(Lx, Ly, d, D, chi, prec=prec, max_samples=len(S0), gram=gram, solve=solve)
        self.theta = torch.as_tensor(np.asarray(theta0, dtype=np.float64)).cuda().contiguous()
        self.h.set_params(self.theta)
        self.h.set_env_reuse(True)  # evaluate() follows sample() on the same, unmodified chains
        self.S = torch.as_tensor(np.asarray(S0, dtype=np.uint8)).cuda().contiguous()
        self.acc = torch.zeros(len(S0), dtype=torch.int64, device="cuda")
        self.sweep = 0
        self.step_no = 0
        self.history = []

    @property
    def nsites(self):
        return self.cfg["Lx"] * self.cfg["Ly"]

    def burn_in(self, nsweeps):
        if self.cfg["sampler"] == "direct":
            return  # independent draws need no burn-in
        self.h.sample(self.S, self.cfg["move"], nsweeps, seed=self.cfg["seed"], sweep0=self.sweep, accepted=self.acc)
        self.sweep += nsweeps

    def step(self):
        """One iteration; returns its metrics (energy per site, its variance and standard error,
        acceptance of the sweeps, MinSR info, status counts)."""
        c = self.cfg
        direct = c["sampler"] == "direct"
        acc0 = self.acc.clone()
        wts = None
        if direct:
            self.h.direct_prepare(c["chi_double"])
            _, lp, _ = self.h.direct_sample(self.S.shape[0], seed=c["seed"], draw=self.step_no, S_out=self.S)
        else:
            self.h.sample(self.S, c["move"], c["sweeps_per_step"], seed=c["seed"], sweep0=self.sweep,
                          accepted=self.acc)
            self.sweep += c["sweeps_per_step"]
        r = self.h.evaluate(self.H, self.S)
        if direct:
            lw = 2.0 * r["logabs"] - lp
            wts = torch.exp(lw - lw.max())
            wts = (wts / wts.sum()).contiguous()
        dth, info = self.h.minsr_step(r["O"], r["eloc"], w=wts, lam=c["lam"], rcond=c["rcond"], tau=c["tau"])
        self.h.last_status()  # synchronises and reads the step's warning
        warn = self.h.last_warning
        self.h.apply_update(self.theta, dth)
        e = r["eloc"][:, 0].double()
        ns = e.numel()
        if direct:
            mean = float((wts * e).sum())
            err = float(torch.sqrt((wts ** 2 * (e - mean) ** 2).sum()))
            var = float((wts * (e - mean) ** 2).sum())
            acc_rate = None
        else:
            mean, err, var = float(e.mean()), float(e.std() / np.sqrt(ns)), float(e.var())
            moves = (2 * c["Lx"] * c["Ly"] - c["Lx"] - c["Ly"]) if c["move"] == P.MOVE_EXCHANGE else c["Lx"] * c["Ly"]
            acc_rate = float((self.acc - acc0).sum()) / (ns * moves * c["sweeps_per_step"])
        m = {"step": self.step_no, "energy_per_site": mean / self.nsites,
             "variance": var, "stderr_per_site": err / self.nsites,
             "acceptance": acc_rate,
             "status_nonzero": int((r["status"] != 0).sum()), "minsr_info": [float(x) for x in info.cpu()],
             "dtheta_norm": float(dth.norm()), "numeric_warning": warn}
        if direct:
            m["ess_fraction"] = float(1.0 / (wts ** 2).sum()) / ns
        self.step_no += 1
        self.history.append(m)
        return m

    def run(self, nsteps, log_path=None):
        for _ in range(nsteps):
            m = self.step()
            if log_path:
                with open(log_path, "a") as f:
                    f.write(json.dumps(m) + "\n")
        return self.history[-nsteps:]

    def energy_tau_int(self):
        """Integrated autocorrelation time of the per-step energy (Sokal window, c = 5)."""
        return tau_int(np.array([m["energy_per_site"] for m in self.history]))

    # ---- checkpoints: theta, chains and counters (raw arrays) + a JSON header
    def save(self, path):
        torch.cuda.synchronize()
        np.savez(path, theta=self.theta.cpu().numpy(), S=self.S.cpu().numpy(), acc=self.acc.cpu().numpy(),
                 header=json.dumps({"cfg": self.cfg, "sweep": self.sweep, "step": self.step_no}))

    @classmethod
    def load(cls, path, H):
        z = np.load(path if path.endswith(".npz") else path + ".npz")
        hdr = json.loads(str(z["header"]))
        c = hdr["cfg"]
        v = cls(c["Lx"], c["Ly"], c["d"], c["D"], c["chi"], H, z["theta"], z["S"], prec=c["prec"], move=c["move"],
                seed=c["seed"], lam=c["lam"], rcond=c["rcond"], tau=c["tau"], sweeps_per_step=c["sweeps_per_step"],
                gram=c["gram"], solve=c["solve"], sampler=c.get("sampler", "metropolis"),
                chi_double=c.get("chi_double"))
        v.acc.copy_(torch.as_tensor(z["acc"]).cuda())
        v.sweep, v.step_no = hdr["sweep"], hdr["step"]
        return v

    def close(self):
        self.h.close()
