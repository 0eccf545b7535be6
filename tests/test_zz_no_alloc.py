"""The allocation-free entry point against the library's grouped run.

mrsim_adc_grouped_noalloc serves host programs that cannot allocate device
memory while they run: programs whose device memory is held by another
allocator (a caching pool or fixed arena reserving nearly all of HBM, so a
new cudaMalloc fails or forces the pool to release memory) and acquisition /
reconstruction loops that forbid cudaMalloc / cudaFree after start-up because
those calls can block until the device is idle.  It keeps its block sums in
a static device array instead of allocating them.

The test computes one Gx-only with-ADC window both ways: mrsim_run in grouped
mode (which allocates its scratch) and the allocation-free call fed with the
same magnetization, group ids and group parameters.  Two calls in a row must
each match within the FP32 tolerance of the other GPU tests (signal rel-L2
1e-4); the second call also shows that the shared array is cleared between
calls.  This file runs last so that a failure here cannot hide another one.
"""

import numpy as np
import pytest

from mrsim_inputs import SeqBuilder, configs

pytestmark = pytest.mark.gpu

GAMMA_BAR = 42.577478518e6


def test_noalloc_window_signal_matches_grouped_run_on_two_calls(mrsim):
    import torch

    ph = configs.small_phantom(24, 20, 5)
    K = ph.K
    rng = np.random.default_rng(21)
    ph.M_init = rng.uniform(-0.6, 0.6, (3, K)).astype(np.float32)
    n_s, dwell, gx = 48, 10e-6, 9.17e-3
    b = SeqBuilder()
    b.add(dwell, n_s, g=(gx, 0.0, 0.0), adc=True)
    seq = b.build()

    with mrsim.Context(0) as ctx:
        hp = ctx.phantom(ph)
        hs = ctx.sequence(seq)
        hg = ctx.group(hp, hs)
        ref, _ = ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32)
        G, gid = mrsim.mrsim_group_info(hg, mrsim.G_X, K)

    _, first = np.unique(gid, return_index=True)  # first member of each group
    assert len(first) == G
    dev = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(
        device="cuda", dtype=dt)
    mx, my = dev(ph.M_init[0]), dev(ph.M_init[1])
    d_gid = dev(gid, torch.int32)
    gpos, gdB0, gT2 = dev(ph.x[first]), dev(ph.dB0[first]), dev(ph.T2[first])
    tau = (np.arange(n_s) + 1) * dwell
    kmom = GAMMA_BAR * np.float64(seq.gx[0]) * tau
    d_tau, d_k = dev(tau, torch.float64), dev(kmom, torch.float64)
    sig = torch.empty(2 * n_s, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()

    for _ in range(2):
        sig.fill_(1e30)  # anything left in the output would show up
        rc = mrsim.mrsim_adc_grouped_noalloc(K, mx, my, d_gid, G, gpos, gdB0, gT2, n_s, d_tau,
                                             d_k, sig, stream)
        assert rc == mrsim.OK
        out = sig.cpu().numpy().view(np.complex128)
        err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert err <= 1e-4, err

    too_many = mrsim.NOALLOC_MAX_GROUPS + 1
    rc = mrsim.mrsim_adc_grouped_noalloc(K, mx, my, d_gid, too_many, gpos, gdB0, gT2, n_s, d_tau,
                                         d_k, sig, stream)
    assert rc == mrsim.EINVAL
