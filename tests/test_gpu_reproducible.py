"""Reproducible sums (mrsim_set_reproducible): block sums (Eq. 9) and signal
sums (Eqs. 6, 8, 10) formed in 64-bit fixed point, so repeated runs give
identical bits whatever order the atomics take.

Every form of the path is run twice with the setting on and compared bit for
bit: the cell form and the per-isochromat form of the fused kernel, direct
advances (about one group per isochromat), the per-isochromat fallback for
subsequences without a type, receive coils, two-axis types, the plain modes,
FP32 and FP64.  The values stay those of the default path: against the FP64
oracle at the parity tolerances (signal rel-L2 1e-4 FP32 / 1e-10 FP64), and
against a default run at 1e-6 (FP32: the cell form holds 4 isochromats per
thread instead of 8, another summation order) or 1e-12 (FP64: the fixed-point
step is 2^-40 on these phantoms)."""

import dataclasses

import numpy as np
import pytest

import oracle
from mrsim_inputs import coil_maps, configs
from mrsim_inputs.phantom import continuous_phantom
from mrsim_inputs.sequence import epi_2d, fse_2d, radial_2d, spin_echo_2d

from test_gpu_parity import general_type_sequence

pytestmark = pytest.mark.gpu

TOL_ORACLE = {0: 1e-4, 1: 1e-10}
TOL_DEFAULT = {0: 1e-6, 1: 1e-12}


@pytest.fixture(scope="module")
def ctx(mrsim):
    c = mrsim.Context(0)
    yield c
    mrsim.mrsim_set_reproducible(c.h, False)
    c.close()


def run(mrsim, ctx, ph, seq, mode, precision, reproducible, two_axis=1):
    mrsim.mrsim_set_reproducible(ctx.h, reproducible)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, two_axis)
    try:
        hp = ctx.phantom(ph)
        hs = ctx.sequence(seq)
        hg = ctx.group(hp, hs) if mode in (mrsim.GROUPED, mrsim.SURROGATE) else None
        outs = [ctx.run(hp, hs, hg, mode, precision, K=ph.K, want_M=True) for _ in range(2)]
        if hg:
            ctx.free("grp", hg)
        ctx.free("seq", hs)
        ctx.free("ph", hp)
    finally:
        mrsim.mrsim_set_reproducible(ctx.h, False)
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, 1)
    return outs


def cases():
    se = spin_echo_2d(n_ro=32, n_pe=16, n_tr=2)
    return {
        # cell form: many (group, window) sums shared by several CTAs
        "fse_cell": (lambda: configs.small_phantom(64, 64, 8),
                     lambda: fse_2d(n_ro=64, n_pe=16, etl=4), 1),
        "epi_cell": (lambda: configs.small_phantom(64, 64, 4), lambda: epi_2d(n_ro=32, n_lines=16), 1),
        # one group per isochromat: direct advances
        "direct": (lambda: continuous_phantom(24, 24, 2, 2, seed=31), lambda: se, 1),
        # subsequences without a type: the per-isochromat fallback kernels
        "general": (lambda: configs.small_phantom(32, 32, 4), general_type_sequence, 0),
        # two-axis types
        "radial": (lambda: configs.small_phantom(32, 32, 2),
                   lambda: radial_2d(n_ro=32, n_spokes=8), 1),
        # receive coils (one pass of 3 coils in the cell form)
        "coils": (lambda: configs.small_phantom(32, 32, 4), lambda: se, 1),
    }


CASES = cases()


def phantom_for(name):
    ph = CASES[name][0]()
    if name == "coils":
        ph = dataclasses.replace(ph, coils=coil_maps(ph, 3, seed=5))
    return ph


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_grouped_runs_bit_identical(mrsim, ctx, name, precision):
    ph = phantom_for(name)
    seq = CASES[name][1]()
    two_axis = CASES[name][2]
    (s1, M1), (s2, M2) = run(mrsim, ctx, ph, seq, mrsim.GROUPED, precision, True, two_axis)
    assert np.array_equal(s1, s2)
    assert np.array_equal(M1, M2)
    (d, _), _ = run(mrsim, ctx, ph, seq, mrsim.GROUPED, precision, False, two_axis)
    assert oracle.rel_l2(s1.ravel(), d.ravel()) <= TOL_DEFAULT[precision]


@pytest.mark.parametrize("mode", ["plain", "plain_cache"])
@pytest.mark.parametrize("precision", [0, 1])
def test_plain_runs_bit_identical(mrsim, ctx, mode, precision):
    m = {"plain": mrsim.PLAIN, "plain_cache": mrsim.PLAIN_CACHE}[mode]
    ph = phantom_for("coils")
    seq = spin_echo_2d(n_ro=32, n_pe=16, n_tr=2)
    (s1, _), (s2, _) = run(mrsim, ctx, ph, seq, m, precision, True)
    assert np.array_equal(s1, s2)
    (d, _), _ = run(mrsim, ctx, ph, seq, m, precision, False)
    assert oracle.rel_l2(s1.ravel(), d.ravel()) <= TOL_DEFAULT[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_reproducible_against_oracle(mrsim, ctx, precision):
    ph = configs.small_phantom(32, 32, 4)
    seq = fse_2d(n_ro=32, n_pe=8, etl=4)
    (sig, M), _ = run(mrsim, ctx, ph, seq, mrsim.GROUPED, precision, True)
    ref, Mref = oracle.simulate(ph, seq)
    assert oracle.rel_l2(sig, ref) <= TOL_ORACLE[precision]
    assert float(np.max(np.abs(M - Mref))) <= (1e-7 if precision else 1e-4)


def test_setting(mrsim, ctx):
    assert mrsim.mrsim_get_reproducible(ctx.h) is False
    mrsim.mrsim_set_reproducible(ctx.h, True)
    assert mrsim.mrsim_get_reproducible(ctx.h) is True
    mrsim.mrsim_set_reproducible(ctx.h, False)
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_set_reproducible(ctx.h, 2)
    assert e.value.code == mrsim.EINVAL
