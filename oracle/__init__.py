"""Plain CPU FP64 oracle for the sampling-based finite-PEPS hot path (arXiv:2503.12557).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The CUDA library never calls it, and it shares no code
with the CUDA path: the two meet only in ``paper_2503_12557_gb300.inputs`` (seeded generators
and Hamiltonian term lists, no arithmetic of the method).

Every routine here is written for a reader to check against the paper by eye: plain numpy in
float64 / complex128, library primitives (QR, SVD, eigh, solve) used as single steps, and no
blocking, fusion or reordering beyond what the definition states.

Modules
-------
philox   Philox4x32-10 counter-based generator (Salmon et al., SC'11), from its published
         definition; the sampler's random numbers.
tn       projection of the PEPS on a configuration, boundary MPS with truncation (Sec. "On the
         boundary MPS method", Eq. (boundary_MPS_approx)), per-tensor log normalisation (Sec. "On
         Numerical Stability"), one- and two-row sandwiches.
energy   local energy (Eq. (local_estimator), Eq. (local_obs)) and log-derivatives O (Sec.
         "Reformulation of the imaginary-time Schroedinger equation").
minsr    MinSR update (Eq. (tdvp_fast)) and the SR pseudo-inverse it reduces to (Eq. (tdvp_slow)).
exact    exact references used to pin the above: dense contraction, state vectors, sparse H.
sampler  Metropolis exchange / flip sweeps with environment reuse.
proposal learned convolutional proposal network: forward, backward, MH acceptance.
"""
