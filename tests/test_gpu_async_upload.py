"""Phantom uploads queued without waiting (MRSIM_PHANTOM_ASYNC).

The call returns once the copies and the value checks are on the context's
stream; host work of the next calls overlaps the transfer.  A valid phantom
gives the bits of a waited upload (reproducible sums, so the comparison is
exact); a phantom with a NaN or a T2 <= 0 is accepted by mrsim_phantom and
rejected with MRSIM_EINVAL by every later call that uses it, and the context
keeps working for other phantoms."""

import numpy as np
import pytest
import torch

from mrsim_inputs import configs
from mrsim_inputs.sequence import fse_2d

pytestmark = pytest.mark.gpu


@pytest.fixture
def ctx(mrsim):
    c = mrsim.Context(0)
    yield c
    c.close()


def pinned(ph):
    """The phantom's seven arrays as pinned host tensors (kept alive by the
    caller until the next call on the context has returned)."""
    return [torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
            for a in (ph.x, ph.y, ph.z, ph.T1, ph.T2, ph.dB0, ph.M0)]


def grouped_signal(mrsim, ctx, hp, seq, K):
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    sig, M = ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32, K=K, want_M=True)
    ctx.free("grp", hg)
    ctx.free("seq", hs)
    return sig, M


def test_async_upload_gives_the_waited_bits(mrsim, ctx):
    ph = configs.small_phantom(64, 64, 8)
    seq = fse_2d(n_ro=16, n_pe=16, etl=4, n_shots=1)
    host = pinned(ph)
    mrsim.mrsim_set_reproducible(ctx.h, 1)
    try:
        h_wait = mrsim.mrsim_phantom(ctx.h, ph.K, *host)
        h_async = mrsim.mrsim_phantom(ctx.h, ph.K, *host, flags=mrsim.PHANTOM_ASYNC)
        ref = grouped_signal(mrsim, ctx, h_wait, seq, ph.K)
        got = grouped_signal(mrsim, ctx, h_async, seq, ph.K)
    finally:
        mrsim.mrsim_set_reproducible(ctx.h, 0)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    back = mrsim.mrsim_phantom_read(ctx.h, h_async, ph.K, fields=("T1", "dB0"))
    assert np.array_equal(back["T1"], ph.T1) and np.array_equal(back["dB0"], ph.dB0)
    for h in (h_wait, h_async):
        mrsim.mrsim_free_phantom(h)


@pytest.mark.parametrize("bad", ["nan_dB0", "zero_T2"])
def test_async_upload_reports_bad_values_at_first_use(mrsim, ctx, bad):
    ph = configs.small_phantom(32, 32, 4)
    seq = fse_2d(n_ro=16, n_pe=16, etl=4, n_shots=1)
    if bad == "nan_dB0":
        ph.dB0 = ph.dB0.copy()
        ph.dB0[ph.K // 3] = np.nan
    else:
        ph.T2 = ph.T2.copy()
        ph.T2[7] = 0.0
    host = pinned(ph)
    with pytest.raises(mrsim.MrsimError) as e:  # the waited upload rejects it at once
        mrsim.mrsim_phantom(ctx.h, ph.K, *host)
    assert e.value.code == mrsim.EINVAL
    hp = mrsim.mrsim_phantom(ctx.h, ph.K, *host, flags=mrsim.PHANTOM_ASYNC)
    hs = ctx.sequence(seq)
    for call in (lambda: mrsim.mrsim_group(ctx.h, hp, hs),
                 lambda: ctx.run(hp, hs, None, mrsim.PLAIN, mrsim.FP32),
                 lambda: mrsim.mrsim_phantom_read(ctx.h, hp, ph.K)):
        with pytest.raises(mrsim.MrsimError) as e:
            call()
        assert e.value.code == mrsim.EINVAL
    mrsim.mrsim_free_phantom(hp)
    # the context still serves a valid phantom
    good = configs.small_phantom(32, 32, 4)
    good_host = pinned(good)
    hg = mrsim.mrsim_phantom(ctx.h, good.K, *good_host, flags=mrsim.PHANTOM_ASYNC)
    sig, _ = ctx.run(hg, hs, None, mrsim.PLAIN, mrsim.FP32)
    assert np.all(np.isfinite(sig)) and np.abs(sig).max() > 0
    ctx.free("seq", hs)
    mrsim.mrsim_free_phantom(hg)
