"""Full-size parity: 27,525,120 isochromats, FSE and EPI, in the launch
configuration the benchmark times (grouped FP32, autotuned launch parameters).

The expected signals come from the FP64 oracle through
tests/golden/make_fullsize_reference.py and are tied to the exact inputs by
SHA-256 digests.  Final magnetizations are checked on a sample of isochromats
that the oracle recomputes one by one.
"""

import os

import numpy as np
import pytest

import oracle
from mrsim_inputs import configs, phantom_digest, sequence_digest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name, ph, seq):
    path = os.path.join(GOLDEN, f"{name}_27m_oracle.npz")
    assert os.path.exists(path), f"{path} missing: run tests/golden/make_fullsize_reference.py"
    d = np.load(path)
    assert str(d["phantom_digest"]) == phantom_digest(ph), "phantom differs from the stored one"
    assert str(d["sequence_digest"]) == sequence_digest(seq), "sequence differs from the stored one"
    return d["signal"]


@pytest.fixture(scope="module")
def full(mrsim):
    ph = configs.full_phantom()
    ctx = mrsim.Context(0)
    hp = ctx.phantom(ph)
    yield ph, ctx, hp
    ctx.close()


@pytest.mark.parametrize("name", ["fse", "epi"])
def test_fullsize_grouped_signal_and_sampled_magnetization(mrsim, full, name):
    ph, ctx, hp = full
    seq = configs.fse_sequence() if name == "fse" else configs.epi_sequence()
    ref = golden(name, ph, seq)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    mrsim.mrsim_autotune(ctx.h, hp, hs, hg, mrsim.GROUPED, mrsim.FP32, 1)
    sig, M = ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32, K=ph.K, want_M=True)
    err = oracle.rel_l2(sig, ref)
    assert err <= 1e-4, f"{name} grouped rel-L2 {err:.3e}"
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(ph.K, size=192, replace=False))
    _, Mref = oracle.simulate(ph.subset(idx), seq, memo=True, adc_recurrence=True)
    assert np.max(np.abs(M[:, idx] - Mref)) <= 1e-4
    ctx.free("grp", hg)
    ctx.free("seq", hs)


def test_fullsize_group_ids_bit_exact(mrsim, full):
    ph, ctx, hp = full
    seq = configs.fse_sequence()
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    for gt in (mrsim.G_X, mrsim.G_Z):
        n, gid = mrsim.mrsim_group_info(hg, gt, ph.K)
        ref, nref = oracle.group(ph, gt)
        assert n == nref
        assert np.array_equal(gid, ref)
    ctx.free("grp", hg)
    ctx.free("seq", hs)


def test_fullsize_plain_epi_and_plain_cache_fse(mrsim, full):
    ph, ctx, hp = full
    epi = configs.epi_sequence()
    hs = ctx.sequence(epi)
    sig, _ = ctx.run(hp, hs, None, mrsim.PLAIN, mrsim.FP32)
    assert oracle.rel_l2(sig, golden("epi", ph, epi)) <= 1e-4
    ctx.free("seq", hs)
    fse = configs.fse_sequence()
    hs = ctx.sequence(fse)
    sig, _ = ctx.run(hp, hs, None, mrsim.PLAIN_CACHE, mrsim.FP32)
    assert oracle.rel_l2(sig, golden("fse", ph, fse)) <= 1e-4
    ctx.free("seq", hs)
