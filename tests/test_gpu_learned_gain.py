"""What the trained proposal network gains over local moves alone.

On a 6x6 Rydberg-shaped PEPS close to a polarised product state (weak correlations), chains
that use only local single-flip sweeps are compared with chains that make trained network moves
(MH with exact PEPS ratios, so both sample |psi|^2).  The figure of merit is effective samples
per second: chains x steps / (2 tau_int x device time), with tau_int of the Rydberg density by
Sokal's window.  Both runs start from the same burnt-in configurations and sample the same
distribution, so their mean densities must agree within the statistical error.
"""
import numpy as np
import pytest
import torch

from paper_2503_12557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_trained_network_gains_effective_samples_per_second():
    from paper_2503_12557_gb300 import build, learned as Lr, peps as P
    build.build()
    lat = I.Lattice(6, 6, 2, 2)
    chi, nc = 4, 1024
    theta = torch.as_tensor(I.peps_near_product(lat, 7, amp=0.3, noise=0.05)).cuda()
    h = P.PEPS(lat.Lx, lat.Ly, 2, lat.D, chi, prec=P.PREC_FP32, max_samples=nc)
    h.set_params(theta)
    S = torch.zeros(nc, lat.nsites, dtype=torch.uint8, device="cuda")
    S, _, _ = Lr.run_local(h, S, 10, seed=11, sweep0=0)
    S_in, S_out, S = Lr.collect_pairs(h, S, 6, 2, seed=12, sweep0=100)
    prop = P.Proposal(lat.Lx, lat.Ly, I.proposal_init(3), C=16, wprec=1)
    losses = Lr.train(prop, S_in, S_out, 150, lr=3e-3, batch=2048)
    assert losses[-1] < losses[0]
    density = lambda s: s.float().mean(dim=1).cpu().numpy()  # noqa: E731
    steps = 80
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    SA = S.clone()
    ev[0].record()
    SA, obsA, accA = Lr.run_local(h, SA, steps, seed=21, sweep0=1000, observe=density)
    ev[1].record()
    SB = S.clone()
    lpsi, _, _ = h.amplitudes(SB)
    accB = torch.zeros(nc, dtype=torch.int64, device="cuda")
    obsB = []
    ev[2].record()
    for t in range(steps):
        h.sample_learned(prop, SB, lpsi, seed=31, step=t, accepted=accB)
        obsB.append(density(SB))
    ev[3].record()
    torch.cuda.synchronize()
    tA, tB = ev[0].elapsed_time(ev[1]) / 1e3, ev[2].elapsed_time(ev[3]) / 1e3
    tauA, tauB = Lr.tau_int(np.array(obsA)), Lr.tau_int(np.array(obsB))
    essA = nc * steps / (2 * tauA * tA)
    essB = nc * steps / (2 * tauB * tB)
    accept = accB.sum().item() / (nc * steps)
    mA, mB = np.mean(obsA), np.mean(obsB)
    err = 3 * np.sqrt(np.var(np.array(obsA)) * 2 * tauA / (nc * steps) + np.var(np.array(obsB)) * 2 * tauB / (nc * steps))
    print(f"local: tau {tauA:.2f} time {tA:.3f}s ESS/s {essA:.3g}; network: tau {tauB:.2f} time {tB:.3f}s "
          f"ESS/s {essB:.3g}, acceptance {accept:.3f}; densities {mA:.4f} {mB:.4f} +- {err:.4f}")
    assert accept > 0.05
    assert abs(mA - mB) < err + 1e-3
    assert essB > essA
