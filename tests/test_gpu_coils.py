"""Receive coils (Eq. 6 with P coils): every mode and precision of the CUDA
path against the FP64 oracle, coil by coil.

Tolerances are those of the single-coil parity tests: signal rel-L2 1e-4 for
FP32 runs and 1e-10 for FP64 runs, per coil.  A unit sensitivity (S = 1)
multiplies every term by (1, 0) exactly, so it must reproduce the run without
coils up to the order in which atomics add the block sums and the signal
(FP32 and FP64 atomics, which differ from run to run in the last bits):
rel-L2 1e-6."""

import dataclasses

import numpy as np
import pytest

import oracle
from mrsim_inputs import coil_maps, configs
from mrsim_inputs.phantom import continuous_phantom
from mrsim_inputs.sequence import fse_2d, spin_echo_2d

from test_gpu_parity import general_type_sequence

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}


@pytest.fixture(scope="module")
def ctx(mrsim):
    c = mrsim.Context(0)
    yield c
    c.close()


def with_coils(ph, n, seed):
    return dataclasses.replace(ph, coils=coil_maps(ph, n, seed))


def run(mrsim, ctx, ph, seq, mode, precision, want_M=False):
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs) if mode in (mrsim.GROUPED, mrsim.SURROGATE) else None
    out = ctx.run(hp, hs, hg, mode, precision, K=ph.K, want_M=want_M)
    if hg:
        ctx.free("grp", hg)
    ctx.free("seq", hs)
    ctx.free("ph", hp)
    return out


def check_coils(sig, ref, precision):
    assert sig.shape == ref.shape
    for p in range(ref.shape[0]):
        e = oracle.rel_l2(sig[p], ref[p])
        assert e <= TOL[precision], f"coil {p}: signal rel-L2 {e:.3e}"


@pytest.mark.parametrize("mode", ["plain", "plain_cache", "grouped"])
@pytest.mark.parametrize("precision", [0, 1])
def test_coils_match_oracle(mrsim, ctx, mode, precision):
    ph = with_coils(configs.small_phantom(24, 20, 3), 3, seed=41)
    seq = spin_echo_2d(n_ro=16, n_pe=8, n_tr=2)
    ref, Mref = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
    m = {"plain": mrsim.PLAIN, "plain_cache": mrsim.PLAIN_CACHE, "grouped": mrsim.GROUPED}[mode]
    sig, M = run(mrsim, ctx, ph, seq, m, precision, want_M=True)
    check_coils(sig, ref, precision)
    assert float(np.max(np.abs(M - Mref))) <= (1e-7 if precision else 1e-4)


@pytest.mark.parametrize("ni", [1, 4])
def test_coils_grouped_fse_every_register_block(mrsim, ctx, ni):
    ph = with_coils(configs.small_phantom(32, 32, 4), 4, seed=43)
    seq = fse_2d(n_ro=32, n_pe=32, etl=4, rf_dur=2e-3, rf_dt=10e-6, dwell=10e-6, esp=10e-3,
                 tr=1.0, n_shots=2)
    ref, _ = oracle.simulate(ph, seq, memo=True, adc_recurrence=True, want_M=False)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_FUSED_NI, ni)
    try:
        sig, _ = run(mrsim, ctx, ph, seq, mrsim.GROUPED, 0)
    finally:
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_FUSED_NI, 4)
    check_coils(sig, ref, 0)


def test_coils_direct_mode_one_group_per_isochromat(mrsim, ctx):
    """Per-isochromat dB0 and b1: the fused kernel advances every isochromat
    from its own parameters (direct mode)."""
    ph = with_coils(continuous_phantom(16, 16, 2, 3, seed=47), 2, seed=44)
    seq = spin_echo_2d(n_ro=16, n_pe=8, n_tr=2)
    ref, _ = oracle.simulate(ph, seq, memo=True, adc_recurrence=True, want_M=False)
    for precision in (0, 1):
        sig, _ = run(mrsim, ctx, ph, seq, mrsim.GROUPED, precision)
        check_coils(sig, ref, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_coils_with_fallback_spans_and_initial_state(mrsim, ctx, precision):
    """Every coil pass restarts the whole span chain (fused spans and plain
    fallbacks) from the initial state."""
    ph = with_coils(configs.small_phantom(16, 16, 3), 3, seed=45)
    rng = np.random.default_rng(12)
    ph.M_init = rng.uniform(-0.5, 0.5, (3, ph.K)).astype(np.float32)
    seq = general_type_sequence()
    ref, Mref = oracle.simulate(ph, seq)
    for mode in (mrsim.GROUPED, mrsim.PLAIN):
        sig, M = run(mrsim, ctx, ph, seq, mode, precision, want_M=True)
        check_coils(sig, ref, precision)
        assert float(np.max(np.abs(M - Mref))) <= (1e-7 if precision else 1e-4)


@pytest.mark.parametrize("reproducible", [False, True])
def test_unit_coil_equals_no_coil(mrsim, ctx, reproducible):
    """With reproducible sums the order of the atomics no longer matters and
    a unit coil gives exactly the signal of none; otherwise up to 1e-6."""
    ph = configs.small_phantom(16, 16, 2)
    seq = spin_echo_2d(n_ro=16, n_pe=8, n_tr=2)
    unit = np.zeros((1, 2, ph.K), np.float32)
    unit[0, 0] = 1.0
    mrsim.mrsim_set_reproducible(ctx.h, reproducible)
    try:
        for mode in (mrsim.GROUPED, mrsim.PLAIN):
            for precision in (0, 1):
                single, _ = run(mrsim, ctx, ph, seq, mode, precision)
                coil, _ = run(mrsim, ctx, dataclasses.replace(ph, coils=unit), seq, mode,
                              precision)
                assert coil.shape == (1, seq.n_samples)
                if reproducible:
                    assert np.array_equal(coil[0], single), (mode, precision)
                else:
                    assert oracle.rel_l2(coil[0], single) <= 1e-6
    finally:
        mrsim.mrsim_set_reproducible(ctx.h, False)


def test_coil_errors(mrsim, ctx):
    ph = configs.small_phantom(8, 8, 2)
    seq = spin_echo_2d(n_ro=8, n_pe=8, n_tr=1)
    hp = ctx.phantom(ph)
    too_many = np.zeros((mrsim.MAX_COILS + 1, 2, ph.K), np.float32)
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_coils(ctx.h, hp, too_many)
    assert e.value.code == mrsim.EINVAL
    bad = np.ones((2, 2, ph.K), np.float32)
    bad[1, 0, 5] = np.inf
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_coils(ctx.h, hp, bad)
    assert e.value.code == mrsim.EINVAL
    # a phantom with coils is batched: one signal per coil, in coil order
    mrsim.mrsim_coils(ctx.h, hp, coil_maps(ph, 2, seed=3))
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    two = np.zeros(2 * 2 * seq.n_samples)
    mrsim.mrsim_run_batch(ctx.h, [hp], [hs], [hg], [two])
    ref2, _ = oracle.simulate(dataclasses.replace(ph, coils=coil_maps(ph, 2, seed=3)), seq,
                              want_M=False)
    check_coils(two.view(np.complex128).reshape(2, seq.n_samples), ref2, 0)
    # detached again: one coil, S = 1
    mrsim.mrsim_coils(ctx.h, hp, None)
    sig = np.zeros(2 * seq.n_samples)
    mrsim.mrsim_run(ctx.h, hp, hs, hg, mrsim.GROUPED, mrsim.FP32, sig)
    ref, _ = oracle.simulate(ph, seq, want_M=False)
    assert oracle.rel_l2(sig.view(np.complex128), ref) <= 1e-4


@pytest.mark.parametrize("n_coils", [1, 2, 3, 5, 8])
def test_coils_cell_form_takes_several_coils_per_pass(mrsim, ctx, n_coils):
    """The cell form of the fused kernel takes up to four coils per pass over
    the sequence (passes of 4, 2 and 1 coils); every coil's signal matches the
    oracle with the cell form on and off, and the coil kernel ran."""
    ph = with_coils(configs.small_phantom(24, 24, 4), n_coils, seed=50 + n_coils)
    seq = fse_2d(n_ro=32, n_pe=32, etl=4, rf_dur=2e-3, rf_dt=10e-6, dwell=10e-6, esp=10e-3,
                 tr=1.0, n_shots=2)
    ref, _ = oracle.simulate(ph, seq, memo=True, adc_recurrence=True, want_M=False)
    for cell in (8, 0):
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_NI, cell)
        mrsim.mrsim_profile_reset(ctx.h)
        mrsim.mrsim_profile_enable(ctx.h, True)
        try:
            sig, _ = run(mrsim, ctx, ph, seq, mrsim.GROUPED, 0)
            prof = mrsim.mrsim_profile_get(ctx.h)
        finally:
            mrsim.mrsim_profile_enable(ctx.h, False)
            mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_NI, 8)
        check_coils(sig, ref, 0)
        ran = {k for k, v in prof.items() if k.startswith("fused") and v[0] > 0}
        assert ran == ({"fused_cell_coils_f32"} if cell else {"fused_grouped_f32"}), ran
