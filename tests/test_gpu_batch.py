"""Multi-instance batches (C ABI peps_batch_*: one persistent kernel launch per precision over a
work queue of (instance, sample) items, recorded in a CUDA graph) and the autotuners
(peps_autotune, peps_batch_autotune): results equal the per-handle calls bit for bit, and every
instance of a ragged FP64 batch matches the oracle, for instances with different lattices, D,
chi, precisions and sample counts."""
import numpy as np
import pytest
import torch

from paper_2503_12557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2503_12557_gb300 import build, peps
    build.build()
    return peps


def _instance(P, Lx, Ly, D, prec, ns, seed, ham="heis", chi=None):
    lat = I.Lattice(Lx, Ly, 2, D)
    h = P.PEPS(Lx, Ly, 2, D, chi or D * D, prec=prec, max_samples=ns)
    h.set_params(torch.as_tensor(I.peps_random(lat, seed, scale=0.5, bias=1.0)).cuda())
    S = torch.as_tensor(I.configs_uniform_sz0(lat, ns, seed + 1)).cuda()
    H = I.heisenberg(lat) if ham == "heis" else I.rydberg(lat, delta=1.0)
    return h, H, S, lat


def _eager(h, H, S, want_O):
    r = h.evaluate(H, S, want_O=want_O)
    torch.cuda.synchronize()
    return {k: (v.clone() if v is not None else None) for k, v in r.items()}


def test_batch_graph_equals_individual_calls(P):
    specs = [(4, 4, 2, 0, 37, 11, "heis", True), (5, 6, 3, 1, 64, 12, "heis", True), (4, 5, 2, 0, 21, 13, "ryd", False),
             (6, 6, 3, 1, 50, 14, "heis", False), (6, 6, 4, 1, 40, 15, "heis", True)]
    inst = [_instance(P, Lx, Ly, D, prec, ns, seed, ham) + (wo,) for (Lx, Ly, D, prec, ns, seed, ham, wo) in specs]
    ref = [_eager(h, H, S, wo) for (h, H, S, lat, wo) in inst]
    batch = P.Batch([(h, H, S, wo) for (h, H, S, lat, wo) in inst], nbranch=3)
    batch.launch()
    batch.stream.synchronize()
    for o, r in zip(batch.out, ref):
        for k in ("logabs", "phase", "eloc", "O", "status"):
            if o.get(k) is not None:
                assert torch.equal(o[k], r[k]), k
    # new configurations written into the recorded input buffers: the replay sees them
    for (h, H, S, lat, wo), o in zip(inst, batch.out):
        o["S"].copy_(torch.as_tensor(I.configs_uniform_sz0(lat, S.shape[0], 99)).cuda())
    torch.cuda.synchronize()
    ref2 = [_eager(h, H, o["S"], wo) for (h, H, S, lat, wo), o in zip(inst, batch.out)]
    batch.launch()
    batch.stream.synchronize()
    for o, r in zip(batch.out, ref2):
        for k in ("logabs", "eloc", "O"):
            if o.get(k) is not None:
                assert torch.equal(o[k], r[k]), k
    batch.close()


def test_ragged_fp64_batch_matches_the_oracle(P):
    # every instance of one persistent FP64 launch against the oracle (1e-10, samples whose
    # truncation hit a near-degenerate cut excluded on both sides, as in the parity tests)
    from oracle import energy
    specs = [(4, 4, 2, 4, 9, 31), (5, 6, 3, 5, 12, 32), (6, 4, 2, 3, 7, 33), (4, 5, 3, 9, 10, 34)]
    inst = []
    for (Lx, Ly, D, chi, ns, seed) in specs:
        lat = I.Lattice(Lx, Ly, 2, D)
        th = I.peps_random(lat, seed, scale=0.5, bias=1.0)
        h = P.PEPS(Lx, Ly, 2, D, chi, prec=0, max_samples=ns)
        h.set_params(torch.as_tensor(th).cuda())
        S = I.configs_uniform_sz0(lat, ns, seed + 100)
        inst.append((h, I.heisenberg(lat), torch.as_tensor(S).cuda(), lat, th, chi, S))
    batch = P.Batch([(h, H, Sd, True) for (h, H, Sd, lat, th, chi, S) in inst])
    # new configurations after recording: the launch reads them
    for (h, H, Sd, lat, th, chi, S), o in zip(inst, batch.out):
        o["S"].copy_(torch.as_tensor(S).cuda())
    batch.launch()
    batch.stream.synchronize()
    for (h, H, Sd, lat, th, chi, S), o in zip(inst, batch.out):
        ref = energy.evaluate(th, S, lat, chi, H=H, want_O=True)
        st = o["status"].cpu().numpy()
        ok = ((st & 1) == 0) & ((ref["status"] & 1) == 0)
        assert ok.sum() >= int(0.7 * len(S))
        assert np.max(np.abs(o["logabs"].cpu().numpy() - ref["logabs"])[ok]) <= 1e-10
        el = o["eloc"].cpu().numpy()[:, 0]
        assert np.max((np.abs(el - ref["eloc"].real) / np.maximum(1.0, np.abs(ref["eloc"])))[ok]) <= 1e-10
        O = o["O"].cpu().numpy()
        dO = np.max(np.abs(O - ref["O"].real), axis=1) / np.maximum(1.0, np.max(np.abs(ref["O"]), axis=1))
        assert np.max(dO[ok]) <= 1e-10
    batch.close()


def test_batch_autotune_keeps_results(P):
    specs = [(5, 5, 2, 1, 30, 41, "heis", True), (6, 6, 3, 1, 24, 42, "heis", True), (4, 6, 3, 1, 16, 43, "ryd", False)]
    inst = [_instance(P, Lx, Ly, D, prec, ns, seed, ham) + (wo,) for (Lx, Ly, D, prec, ns, seed, ham, wo) in specs]
    ref = [_eager(h, H, S, wo) for (h, H, S, lat, wo) in inst]
    batch = P.Batch([(h, H, S, wo) for (h, H, S, lat, wo) in inst], autotune=True)
    assert batch.budget_kb in (56, 72, 110, 220)
    batch.launch()
    batch.stream.synchronize()
    for o, r in zip(batch.out, ref):
        for k in ("logabs", "eloc", "O", "status"):
            if o.get(k) is not None:
                assert torch.equal(o[k], r[k]), k
    batch.close()


def test_batch_rejects_repeated_handle(P):
    h, H, S, lat = _instance(P, 4, 4, 2, 0, 8, 3)
    with pytest.raises(RuntimeError):
        P.Batch([(h, H, S, False), (h, H, S, False)])


@pytest.mark.parametrize("Lx,Ly,D,prec,ns", [(6, 6, 3, 1, 96), (8, 8, 4, 1, 128), (5, 5, 2, 0, 40)])
def test_autotune_keeps_results(P, Lx, Ly, D, prec, ns):
    h, H, S, lat = _instance(P, Lx, Ly, D, prec, ns, 21)
    before = _eager(h, H, S, True)
    kb = h.autotune(S, H)
    cands = {72, 110, 220} if prec == 1 else {100, 210}
    assert len(kb) == 4 and all(k in cands for k in kb), kb
    after = _eager(h, H, S, True)
    for k in ("logabs", "eloc", "O"):
        assert torch.equal(before[k], after[k]), k
    # the sampler under the tuned plan: same chains as an untuned handle
    h2, _, _, _ = _instance(P, Lx, Ly, D, prec, ns, 21)
    S1, S2 = S.clone(), S.clone()
    h.sample(S1, move=P.MOVE_EXCHANGE, nsweeps=1, seed=4)
    h2.sample(S2, move=P.MOVE_EXCHANGE, nsweeps=1, seed=4)
    torch.cuda.synchronize()
    assert torch.equal(S1, S2)
