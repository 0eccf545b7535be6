"""Cell form of the fused grouped kernel against the FP64 oracle.

In the cell form every thread holds isochromats of one (with-ADC group,
with-RF group) cell and applies one combined row C = T Adv per cell to each
with-RF subsequence (Sec. 2.3 update step; Eqs. 4-5 and 7), and sums the
free-axis-rotated transverse magnetization for each with-ADC window (Eq. 9).
Every case runs at 4 and 8 isochromats per thread, with the combined rows read
from a table and formed by each thread, and with the form off, at the FP32 bar
(signal rel-L2 1e-4, M_final max error 1e-4 of max M0), and checks from the
per-kernel profile which form actually ran.
"""

import numpy as np
import pytest

import oracle
from mrsim_inputs import SeqBuilder, configs
from mrsim_inputs.phantom import mapped_phantom
from mrsim_inputs.sequence import epi_2d, fse_2d, gre_2d, spin_echo_2d

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def ctx(mrsim):
    c = mrsim.Context(0)
    yield c
    c.close()


def run_cell(mrsim, ctx, ph, seq, cell_ni, rows=0):
    """Grouped FP32 run with the cell form set to cell_ni and the combined
    rows to `rows` (0 automatic, 1 table, 2 per thread); returns the signal,
    M_final and the names of the fused kernels that ran."""
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_NI, cell_ni)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_ROWS, rows)
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    try:
        mrsim.mrsim_profile_reset(ctx.h)
        mrsim.mrsim_profile_enable(ctx.h, True)
        sig, M = ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32, K=ph.K, want_M=True)
        prof = mrsim.mrsim_profile_get(ctx.h)
    finally:
        mrsim.mrsim_profile_enable(ctx.h, False)
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_NI, 8)
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_ROWS, 0)
        ctx.free("grp", hg)
        ctx.free("seq", hs)
        ctx.free("ph", hp)
    return sig, M, {k for k, v in prof.items() if k.startswith("fused") and v[0] > 0}


def check(sig, M, ref, Mref, M0max):
    e = oracle.rel_l2(sig, ref)
    assert e <= TOL, f"signal rel-L2 {e:.3e}"
    em = float(np.max(np.abs(M - Mref))) / M0max
    assert em <= TOL, f"M_final max error {em:.3e}"
    return e


def mixed_rf_sequence():
    """Slice-selective sinc excitations (Gz-only, the more frequent with-RF
    type) and non-selective hard refocusing pulses (no gradients) in one
    sequence, Gx readouts with Gy phase encodes: the with-RF groups of the
    hard pulses (T1, T2, dB0) are constant inside every cell as well."""
    b = SeqBuilder()
    for p in range(3):
        b.rf_sinc(90, "x", 1e-3, 10e-6, 4.0, 0.01)
        b.add(1e-3, 1, g=(-2e-3, (p - 1) * 1e-3, -2.5e-3))
        if p < 2:
            b.rf_hard(180, "y", 200e-6, 10e-6)
        b.add(1e-3, 1, g=(0, 0, 0))
        b.readout(16, 10e-6, (4e-3, 0.0, 0.0))
        b.add(20e-3, 1)
    return b.build()


def nonselective_sequence():
    """Hard pulses only (no with-RF gradient type besides no-grads): two free
    axes per isochromat in the cell form."""
    b = SeqBuilder()
    for p in range(4):
        b.rf_hard(30, "x", 100e-6, 10e-6)
        b.add(1e-3, 1, g=(-2e-3, (p - 2) * 1e-3, 1.5e-3))
        b.readout(16, 10e-6, (4e-3, 0.0, 0.0))
        b.add(5e-3, 1, g=(0, 0, 3e-3))
    return b.build()


def fallback_span_sequence():
    """Gz-only sinc pulses and Gx readouts around an unclassifiable with-RF
    subsequence (Gx and Gz during RF) and an unclassifiable with-ADC window
    (Gx and Gy): three spans of the fused kernel with the per-isochromat
    fallback kernels between them, plus a window without gradients."""
    b = SeqBuilder()
    b.rf_sinc(90, "x", 1e-3, 10e-6, 4.0, 0.01)
    b.add(1e-3, 1, g=(-2e-3, 1e-3, -2.5e-3))
    b.readout(16, 10e-6, (4e-3, 0.0, 0.0))
    b.add(1e-3, 1)
    for _ in range(50):
        b.add(10e-6, 1, b1=(2e-6, 0.5e-6), g=(1e-3, 0.0, 2e-3))
    b.add(2e-3, 1, g=(0.0, 1e-3, 0.0))
    b.add(10e-6, 16, g=(5e-3, 2e-3, 0.0), adc=True)
    b.add(1e-3, 1)
    b.readout(16, 10e-6, (4e-3, 0.0, 0.0))
    b.rf_sinc(180, "y", 1e-3, 10e-6, 4.0, 0.01)
    b.add(1e-3, 1, g=(0.0, 0.0, 2e-3))
    b.readout(16, 10e-6, (-4e-3, 0.0, 0.0))
    b.add(10e-6, 8, adc=True)
    b.add(5e-3, 1)
    return b.build()


def cases():
    se_ph, se_seq = configs.se_32()
    small = configs.small_phantom(24, 20, 5)
    return {
        "se_32": (se_ph, se_seq),
        "fse": (small, fse_2d(n_ro=32, n_pe=32, etl=8, rf_dur=2e-3, rf_dt=10e-6, dwell=10e-6,
                             esp=10e-3, tr=0.5, n_shots=2)),
        "epi": (small, epi_2d(n_ro=32, n_lines=24, rf_dur=2e-3, rf_dt=5e-6)),
        "gre": (configs.small_phantom(16, 16, 3), gre_2d(n_ro=16, n_pe=8)),
        "mapped_tiny_cells": (mapped_phantom(24, 24, 6, 6, seed=5), spin_echo_2d(n_ro=16, n_pe=16,
                                                                                  n_tr=3)),
        "mixed_rf_types": (configs.small_phantom(16, 12, 4), mixed_rf_sequence()),
        "two_free_axes": (configs.small_phantom(16, 12, 4), nonselective_sequence()),
    }


@pytest.mark.parametrize("name", ["se_32", "fse", "epi", "gre", "mapped_tiny_cells",
                                  "mixed_rf_types", "two_free_axes"])
def test_cell_form_against_oracle(mrsim, ctx, name):
    ph, seq = cases()[name]
    ref, Mref = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
    M0max = float(np.max(ph.M0))
    sigs = {}
    for ni, rows in ((4, 1), (8, 1), (4, 2), (8, 2), (0, 0)):
        sig, M, ran = run_cell(mrsim, ctx, ph, seq, ni, rows)
        check(sig, M, ref, Mref, M0max)
        assert ran == ({"fused_cell_f32"} if ni else {"fused_grouped_f32"}), ran
        sigs[ni, rows] = sig
    # every form computes the same sums up to FP32 rounding order
    for key in ((4, 1), (8, 1), (4, 2), (8, 2)):
        assert oracle.rel_l2(sigs[key], sigs[0, 0]) <= 1e-5, key


@pytest.mark.parametrize("K", [1, 5, 130, 1025, 1700, 2323])
def test_cell_form_ragged_phantoms(mrsim, ctx, K):
    """Subsets of a phantom leave cells of every size from one isochromat
    up, so most threads hold fewer isochromats than their width.  Below
    about one with-ADC group per four isochromats the per-isochromat
    ("direct") advance runs instead, so the three smallest cases check
    parity only."""
    rng = np.random.default_rng(100 + K)
    full = configs.small_phantom(32, 32, 4)
    inside = np.flatnonzero(full.M0 > 0)
    ph = full.subset(np.sort(rng.choice(inside, size=K, replace=False)))
    seq = spin_echo_2d(n_ro=16, n_pe=16, n_tr=3)
    ref, Mref = oracle.simulate(ph, seq)
    for ni, rows in ((4, 1), (8, 1), (8, 2)):
        sig, M, ran = run_cell(mrsim, ctx, ph, seq, ni, rows)
        if K >= 1000:
            assert ran == {"fused_cell_f32"}
        check(sig, M, ref, Mref, float(np.max(ph.M0)))


def test_cell_form_initial_state_b1_and_fallback_spans(mrsim, ctx):
    """A given initial state (the kernel reads the state instead of
    starting from equilibrium), RF scales, infinite T1 / T2 and a sequence
    with unclassifiable subsequences between the spans (state written and
    read back around the per-isochromat fallback kernels)."""
    ph = configs.small_phantom(16, 16, 3)
    rng = np.random.default_rng(12)
    ph.M_init = rng.uniform(-0.5, 0.5, (3, ph.K)).astype(np.float32)
    ph.b1 = rng.choice(np.array([0.9, 1.0, 1.1], np.float32), ph.K)
    ph.T1 = np.where(ph.labels == 1, np.inf, ph.T1).astype(np.float32)
    ph.T2 = np.where(ph.labels == 2, np.inf, ph.T2).astype(np.float32)
    # general (not two-axis) typing keeps the unclassifiable subsequences
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, 0)
    try:
        for seq in (spin_echo_2d(n_ro=16, n_pe=16, n_tr=2), fallback_span_sequence()):
            ref, Mref = oracle.simulate(ph, seq)
            for ni, rows in ((4, 1), (8, 1), (4, 2), (8, 2)):
                sig, M, ran = run_cell(mrsim, ctx, ph, seq, ni, rows)
                assert "fused_cell_f32" in ran
                check(sig, M, ref, Mref, float(np.max(ph.M0)))
    finally:
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, 1)


def test_cell_tuning_values(mrsim, ctx):
    for bad in (1, 2, 16, -4):
        with pytest.raises(mrsim.MrsimError):
            mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_NI, bad)
    for v in (0, 4, 8):
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_NI, v)
        assert mrsim.mrsim_get_tuning(ctx.h, mrsim.TUNE_CELL_NI) == v
    for bad in (3, -1):
        with pytest.raises(mrsim.MrsimError):
            mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_ROWS, bad)
    for v in (1, 2, 0):
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_ROWS, v)
        assert mrsim.mrsim_get_tuning(ctx.h, mrsim.TUNE_CELL_ROWS) == v


def test_clustered_phantom_runs_the_cell_form(mrsim, ctx):
    """A clustered parameter-mapping phantom has many small cells (position
    pairs times clusters): the automatic choice forms the rows per thread
    instead of building a table several times the size of the state."""
    from oracle import cluster as oc
    base = mapped_phantom(32, 32, 8, 6, seed=21)
    ph = oc.cluster_phantom(base, 24).phantom
    seq = fse_2d(n_ro=32, n_pe=16, etl=4, rf_dur=2e-3, rf_dt=10e-6, dwell=10e-6, esp=10e-3,
                 tr=0.5, n_shots=2)
    ref, Mref = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    try:
        mrsim.mrsim_profile_reset(ctx.h)
        mrsim.mrsim_profile_enable(ctx.h, True)
        sig, M = ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32, K=ph.K, want_M=True)
        prof = {k for k, v in mrsim.mrsim_profile_get(ctx.h).items() if v[0] > 0}
    finally:
        mrsim.mrsim_profile_enable(ctx.h, False)
        ctx.free("grp", hg)
        ctx.free("seq", hs)
        ctx.free("ph", hp)
    assert "fused_cell_f32" in prof and "cell_rows" not in prof, prof
    check(sig, M, ref, Mref, float(np.max(ph.M0)))
