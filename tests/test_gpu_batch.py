"""Multi-instance batches in one CUDA graph and the shared-memory autotuner (C ABI
peps_batch_* and peps_autotune): results equal the per-handle calls bit for bit, for ragged
instances (different lattices, D, chi = D^2, precisions and sample counts)."""
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


def _instance(P, Lx, Ly, D, prec, ns, seed, ham="heis"):
    lat = I.Lattice(Lx, Ly, 2, D)
    h = P.PEPS(Lx, Ly, 2, D, D * D, prec=prec, max_samples=ns)
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
             (6, 6, 3, 1, 50, 14, "heis", False)]
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
