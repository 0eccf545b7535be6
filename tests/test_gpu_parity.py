"""GPU library vs FP64 oracle, through the C ABI.

Tolerances (signal rel-L2 over all complex samples, M_final max abs error
relative to max M0):
  FP64 per-isochromat arithmetic  signal 1e-10 (same formulas, different
                                  rounding order and closed-form shortcuts);
                                  M_final 1e-7, because the ABI returns M_final
                                  as float32 (half an ulp of |M| <= 1 is 6e-8)
  FP32 per-isochromat arithmetic  1e-4 for both (the target for FP32 paths)
Classification and group ids are compared bit-exactly.
"""

import numpy as np
import pytest

import oracle
from mrsim_inputs import Phantom, SeqBuilder, Sequence, configs
from mrsim_inputs.sequence import epi_2d, fse_2d, gre_2d, spin_echo_2d

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}  # by precision (FP32, FP64)


@pytest.fixture(scope="module")
def ctx(mrsim):
    c = mrsim.Context(0)
    yield c
    c.close()


def run_both(mrsim, ctx, ph, seq, mode, precision, want_M=True):
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs) if mode in (mrsim.GROUPED, mrsim.SURROGATE) else None
    sig, M = ctx.run(hp, hs, hg, mode, precision, K=ph.K, want_M=want_M)
    ctx.free("grp", hg) if hg else None
    ctx.free("seq", hs)
    ctx.free("ph", hp)
    return sig, M


def check(sig, M, ref, Mref, precision, M0max=1.0):
    e = oracle.rel_l2(sig, ref)
    assert e <= TOL[precision], f"signal rel-L2 {e:.3e}"
    if M is not None:
        em = float(np.max(np.abs(M - Mref))) / M0max
        tolM = 1e-7 if precision == 1 else 1e-4
        assert em <= tolM, f"M_final max error {em:.3e}"
    return e


SE = None


def se():
    global SE
    if SE is None:
        ph, seq = configs.se_32()
        SE = (ph, seq, *oracle.simulate(ph, seq, memo=True, adc_recurrence=True))
    return SE


@pytest.mark.parametrize("mode", ["plain", "plain_cache", "grouped"])
@pytest.mark.parametrize("precision", [0, 1])
def test_spin_echo_32x32x4_all_modes(mrsim, ctx, mode, precision):
    ph, seq, ref, Mref = se()
    m = {"plain": mrsim.PLAIN, "plain_cache": mrsim.PLAIN_CACHE, "grouped": mrsim.GROUPED}[mode]
    sig, M = run_both(mrsim, ctx, ph, seq, m, precision)
    check(sig, M, ref, Mref, precision)


@pytest.mark.parametrize("two_axis", [1, 0])
def test_classification_bit_exact(mrsim, ctx, two_axis):
    """Subsequence split and gradient types of the library's sequences equal
    the oracle's classifier, with two-axis typing on (the default) and off."""
    from mrsim_inputs.sequence import radial_2d
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, two_axis)
    try:
        for seq in (configs.se_32()[1], fse_2d(n_ro=32, n_pe=32, etl=8, n_shots=1),
                    epi_2d(n_ro=32, n_lines=16), gre_2d(n_ro=16, n_pe=4),
                    radial_2d(n_ro=16, n_spokes=6, oblique_deg=20.0)):
            hs = ctx.sequence(seq)
            info = mrsim.mrsim_seq_info(hs)
            ctx.free("seq", hs)
            q = oracle.classify(seq, two_axis=bool(two_axis))
            for k in ("type", "gtype", "seg_begin", "seg_end"):
                assert np.array_equal(info[k], q[k].astype(info[k].dtype)), k
            assert info["n_samples_total"] == int(q["n_samples"].sum())
    finally:
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, 1)


@pytest.mark.parametrize("shape", [(32, 32, 4), (16, 24, 3), (64, 64, 8)])
def test_group_ids_bit_exact(mrsim, ctx, shape):
    ph = configs.small_phantom(*shape)
    seq = fse_2d(n_ro=16, n_pe=16, etl=4, n_shots=1)
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    for gt in (mrsim.G_X, mrsim.G_Z):
        n, gid = mrsim.mrsim_group_info(hg, gt, ph.K)
        ref, nref = oracle.group(ph, gt)
        assert n == nref
        assert np.array_equal(gid, ref)
    with pytest.raises(mrsim.MrsimError):
        mrsim.mrsim_group_info(hg, mrsim.G_Y, ph.K)  # not needed by this sequence
    ctx.free("grp", hg)
    ctx.free("seq", hs)
    ctx.free("ph", hp)


@pytest.mark.parametrize("n_distinct", [1_000_000, 1_310_720])
def test_group_ids_bit_exact_many_distinct_keys(mrsim, ctx, n_distinct):
    """Group numbering with about a million distinct keys per type: the group
    build's first hash table takes 2^20 keys and the pass is redone with room
    for every isochromat once more arrive.  Here only dB0 separates the Gz
    groups, so they number exactly n_distinct; the Gx groups (x, dB0) number
    more and take the redo in both cases."""
    ph = configs.small_phantom(128, 128, 80)
    rng = np.random.default_rng(11)
    ph.z = np.zeros(ph.K, np.float32)
    ph.T1 = np.full(ph.K, 1.0, np.float32)
    ph.T2 = np.full(ph.K, 0.1, np.float32)
    ph.dB0 = (rng.permutation(ph.K) % n_distinct).astype(np.float32) * np.float32(0.01)
    seq = fse_2d(n_ro=16, n_pe=16, etl=4, n_shots=1)
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    for gt in (mrsim.G_X, mrsim.G_Z):
        n, gid = mrsim.mrsim_group_info(hg, gt, ph.K)
        ref, nref = oracle.group(ph, gt)
        assert n == nref
        assert np.array_equal(gid, ref)
    assert mrsim.mrsim_group_info(hg, mrsim.G_Z)[0] == n_distinct
    ctx.free("grp", hg)
    ctx.free("seq", hs)
    ctx.free("ph", hp)


@pytest.mark.parametrize("n_db0", [10, 40])
def test_layout_dense_and_hashed_cells(mrsim, ctx, n_db0):
    """The layout's cells come from a flag array over (Gx group, Gz group)
    pairs when there are at most 2^24 pairs (10 dB0 classes: 1,280 x 1,280)
    and from the hashed cell path above that (40 classes: 5,120 x 5,120).
    Either way the grouped FSE signal and final magnetization match the
    per-isochromat GPU form, and reproducible-mode runs are bit-identical
    across group builds (the layout is deterministic)."""
    ph = configs.small_phantom(128, 128, 128)
    rng = np.random.default_rng(17)
    ph.T1 = np.full(ph.K, 0.9, np.float32)
    ph.T2 = np.full(ph.K, 0.08, np.float32)
    ph.dB0 = rng.integers(0, n_db0, ph.K).astype(np.float32) * np.float32(0.5)
    seq = fse_2d(n_ro=16, n_pe=16, etl=4, n_shots=1)
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    assert mrsim.mrsim_group_info(hg := ctx.group(hp, hs), mrsim.G_X)[0] == 128 * n_db0
    assert mrsim.mrsim_group_info(hg, mrsim.G_Z)[0] == 128 * n_db0
    hg2 = ctx.group(hp, hs)
    mrsim.mrsim_set_reproducible(ctx.h, 1)  # fixed-point sums: bit-identical runs
    try:
        sig, M = ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32, K=ph.K, want_M=True)
        sig2, M2 = ctx.run(hp, hs, hg2, mrsim.GROUPED, mrsim.FP32, K=ph.K, want_M=True)
    finally:
        mrsim.mrsim_set_reproducible(ctx.h, 0)
    assert np.array_equal(sig, sig2) and np.array_equal(M, M2)
    ref, Mref = ctx.run(hp, hs, None, mrsim.PLAIN, mrsim.FP32, K=ph.K, want_M=True)
    assert oracle.rel_l2(sig, ref) <= 1e-4
    assert float(np.max(np.abs(M - Mref))) <= 1e-4
    for h in (hg, hg2):
        ctx.free("grp", h)
    ctx.free("seq", hs)
    ctx.free("ph", hp)


@pytest.mark.parametrize("precision", [0, 1])
def test_long_cells_sorted_layout(mrsim, ctx, precision):
    """A tall phantom (8 x 1000 x 2) whose layout cells hold up to 1,000
    isochromats, so every branch of the cell sort runs: warp networks of 32
    to 1,024 members.  A member lost or doubled by the sort would show in the
    final magnetization, which comes back through the layout permutation."""
    ph = configs.small_phantom(8, 1000, 2)
    seq = fse_2d(n_ro=16, n_pe=16, etl=4, n_shots=1)
    ref, Mref = oracle.simulate(ph, seq)
    sig, M = run_both(mrsim, ctx, ph, seq, mrsim.GROUPED, precision)
    check(sig, M, ref, Mref, precision)


def test_group_ids_with_b1_and_negative_zero(mrsim, ctx):
    ph = configs.small_phantom(16, 16, 2)
    rng = np.random.default_rng(3)
    ph.b1 = rng.choice(np.array([0.9, 1.0, 1.1], np.float32), ph.K)
    ph.x = ph.x.copy()
    ph.x[ph.x == 0] = -0.0
    ph.x[:5] = 0.0
    seq = spin_echo_2d(n_ro=8, n_pe=8, n_tr=2)
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    for gt in (mrsim.G_X, mrsim.G_Z):
        n, gid = mrsim.mrsim_group_info(hg, gt, ph.K)
        ref, nref = oracle.group(ph, gt)
        assert n == nref and np.array_equal(gid, ref)
    ref, Mref = oracle.simulate(ph, seq)
    sig, M = ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP64, K=ph.K, want_M=True)
    check(sig, M, ref, Mref, 1)


@pytest.mark.parametrize("precision", [0, 1])
def test_fse_small_grouped_and_plain(mrsim, ctx, precision):
    ph = configs.small_phantom(24, 20, 5)
    seq = fse_2d(n_ro=32, n_pe=32, etl=8, rf_dur=2e-3, rf_dt=10e-6, dwell=10e-6, esp=10e-3,
                 tr=0.5, n_shots=2)
    ref, Mref = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
    for mode in (mrsim.GROUPED, mrsim.PLAIN):
        sig, M = run_both(mrsim, ctx, ph, seq, mode, precision)
        check(sig, M, ref, Mref, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_epi_small_grouped_and_plain(mrsim, ctx, precision):
    ph = configs.small_phantom(24, 20, 5)
    seq = epi_2d(n_ro=32, n_lines=24, rf_dur=2e-3, rf_dt=5e-6)
    ref, Mref = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
    for mode in (mrsim.GROUPED, mrsim.PLAIN):
        sig, M = run_both(mrsim, ctx, ph, seq, mode, precision)
        check(sig, M, ref, Mref, precision)


@pytest.mark.parametrize("K", [1, 7, 255, 1023, 1025, 3001])
def test_ragged_and_tiny_phantoms(mrsim, ctx, K):
    rng = np.random.default_rng(K)
    full = configs.small_phantom(32, 32, 4)
    idx = np.sort(rng.choice(full.K, size=K, replace=False))
    ph = full.subset(idx)
    seq = spin_echo_2d(n_ro=16, n_pe=16, n_tr=3)
    ref, Mref = oracle.simulate(ph, seq)
    for mode in (mrsim.GROUPED, mrsim.PLAIN):
        for prec in (0, 1):
            sig, M = run_both(mrsim, ctx, ph, seq, mode, prec)
            check(sig, M, ref, Mref, prec)


def general_type_sequence():
    """Unclassifiable with-RF (Gx + Gz during RF) and with-ADC (Gx + Gy)
    subsequences between known ones: the conventional fallback path."""
    b = SeqBuilder()
    b.rf_sinc(90, "x", 1e-3, 10e-6, 4.0, 0.01)              # Gz-only
    b.add(1e-3, 1, g=(2e-3, 1e-3, -3e-3))
    for j in range(50):                                       # RF with Gx and Gz
        b.add(10e-6, 1, b1=(2e-6, 0.5e-6), g=(1e-3, 0, 2e-3))
    b.add(2e-3, 1, g=(0, 1e-3, 0))
    b.add(10e-6, 16, g=(5e-3, 2e-3, 0), adc=True)            # ADC with Gx and Gy
    b.add(1e-3, 1)
    b.add(10e-6, 16, g=(5e-3, 0, 0), adc=True)               # Gx-only
    b.add(1e-3, 1, g=(0, 0, 1e-3))
    b.rf_hard(30, "y", 100e-6, 10e-6)                         # no-grads RF
    b.add(10e-6, 8, adc=True)                                 # no-grads ADC
    b.add(5e-3, 1)
    return b.build()


@pytest.mark.parametrize("two_axis", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_general_type_fallback_and_no_grads(mrsim, ctx, precision, two_axis):
    """With two-axis typing off, the Gx+Gz pulse and the Gx+Gy window are
    general subsequences (the per-isochromat fallback between spans); with it
    on they are grouped on two positions.  Both match the oracle."""
    ph = configs.small_phantom(16, 16, 3)
    seq = general_type_sequence()
    q = oracle.classify(seq, two_axis=bool(two_axis))
    kinds = set(q["gtype"][q["type"] != oracle.RELAX])
    assert (4 in kinds) if not two_axis else (oracle.G_XZ in kinds and oracle.G_XY in kinds)
    ref, Mref = oracle.simulate(ph, seq)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, two_axis)
    try:
        for mode in (mrsim.GROUPED, mrsim.PLAIN, mrsim.PLAIN_CACHE):
            sig, M = run_both(mrsim, ctx, ph, seq, mode, precision)
            check(sig, M, ref, Mref, precision)
    finally:
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, 1)


def test_initial_state_b1_scale_and_infinite_relaxation(mrsim, ctx):
    ph = configs.small_phantom(16, 16, 2)
    rng = np.random.default_rng(11)
    ph.M_init = rng.uniform(-0.5, 0.5, (3, ph.K)).astype(np.float32)
    ph.b1 = rng.uniform(0.9, 1.1, ph.K).astype(np.float32)
    ph.T1 = np.where(ph.labels == 1, np.inf, ph.T1).astype(np.float32)
    ph.T2 = np.where(ph.labels == 2, np.inf, ph.T2).astype(np.float32)
    seq = spin_echo_2d(n_ro=16, n_pe=16, n_tr=2)
    ref, Mref = oracle.simulate(ph, seq)
    for mode in (mrsim.GROUPED, mrsim.PLAIN, mrsim.PLAIN_CACHE):
        for prec in (0, 1):
            sig, M = run_both(mrsim, ctx, ph, seq, mode, prec)
            check(sig, M, ref, Mref, prec)


def test_sequence_without_adc_and_without_rf(mrsim, ctx):
    ph = configs.small_phantom(8, 8, 2)
    b = SeqBuilder()
    b.rf_hard(45, "x", 100e-6, 10e-6)
    b.add(3e-3, 1, g=(1e-3, 2e-3, 0))
    seq = b.build()
    _, Mref = oracle.simulate(ph, seq)
    for mode in (mrsim.GROUPED, mrsim.PLAIN):
        hp = ctx.phantom(ph)
        hs = ctx.sequence(seq)
        hg = ctx.group(hp, hs) if mode == mrsim.GROUPED else None
        sig, M = ctx.run(hp, hs, hg, mode, mrsim.FP64, K=ph.K, want_M=True)
        assert sig.size == 0
        assert np.max(np.abs(M - Mref)) < 1e-7
    b = SeqBuilder()
    b.add(2e-3, 1, g=(1e-3, 0, 0))
    b.add(10e-6, 10, g=(2e-3, 0, 0), adc=True)
    seq = b.build()
    ref, Mref = oracle.simulate(ph, seq)
    for mode in (mrsim.GROUPED, mrsim.PLAIN):
        sig, M = run_both(mrsim, ctx, ph, seq, mode, 1)
        assert np.allclose(sig, 0) and np.allclose(ref, 0)
        assert np.max(np.abs(M - Mref)) < 1e-7


def test_errors_are_reported(mrsim, ctx):
    ph = configs.small_phantom(8, 8, 2)
    bad = Phantom(**{**ph.__dict__})
    bad.T2 = ph.T2.copy()
    bad.T2[3] = np.nan
    with pytest.raises(mrsim.MrsimError) as e:
        ctx.phantom(bad)
    assert e.value.code == mrsim.EINVAL
    bad.T2[3] = 0.0
    with pytest.raises(mrsim.MrsimError) as e:
        ctx.phantom(bad)
    assert e.value.code == mrsim.EINVAL
    b = SeqBuilder()
    b.add(1e-6, 1, b1=(1e-6, 0), adc=True)
    with pytest.raises(mrsim.MrsimError) as e:
        ctx.sequence(b.build())
    assert e.value.code == mrsim.EUNSUPPORTED
    b = SeqBuilder()
    b.add(1e-6, 1)
    s = b.build()
    s.repeat[0] = 0
    with pytest.raises(mrsim.MrsimError) as e:
        ctx.sequence(s)
    assert e.value.code == mrsim.EINVAL
    # groups built for another phantom
    seq = spin_echo_2d(n_ro=8, n_pe=8, n_tr=1)
    h1, h2 = ctx.phantom(ph), ctx.phantom(ph)
    hs = ctx.sequence(seq)
    g1 = ctx.group(h1, hs)
    sig = np.zeros(2 * 8)
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_run(ctx.h, h2, hs, g1, mrsim.GROUPED, mrsim.FP32, sig)
    assert e.value.code == mrsim.ESTATE
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_run(ctx.h, h2, hs, None, mrsim.GROUPED, mrsim.FP32, sig)
    assert e.value.code == mrsim.EINVAL


def test_device_pointer_inputs_and_outputs(mrsim, ctx):
    import torch
    ph, seq, ref, Mref = se()
    dev = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()
           for k, v in dict(x=ph.x, y=ph.y, z=ph.z, T1=ph.T1, T2=ph.T2, dB0=ph.dB0,
                            M0=ph.M0).items()}
    hp = ctx.phantom(dev, device_ptrs=True)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    sig = torch.zeros(2 * seq.n_samples, dtype=torch.float64, device="cuda")
    M = torch.zeros(3 * ph.K, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    mrsim.mrsim_run(ctx.h, hp, hs, hg, mrsim.GROUPED, mrsim.FP32, sig, M, mrsim.OUT_DEVICE)
    s = sig.cpu().numpy().view(np.complex128)
    check(s, M.cpu().numpy().reshape(3, -1), ref, Mref, 0)


def test_repeated_runs_are_consistent(mrsim, ctx):
    ph, seq, ref, _ = se()
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    a, _ = ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32)
    b, _ = ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32)
    assert oracle.rel_l2(a, ref) <= 1e-4 and oracle.rel_l2(b, a) <= 1e-6


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32, 128])
@pytest.mark.parametrize("precision", [0, 1])
def test_precompute_lane_counts(mrsim, ctx, lanes, precision):
    """Every lane count of the combined-transition step (shuffle tree inside a
    warp, or shared-memory tree over a CTA) gives the oracle's signal; the
    phantom makes almost every isochromat its own group, with a ragged count
    of groups per warp."""
    from mrsim_inputs.phantom import continuous_phantom
    ph = continuous_phantom(13, 11, 3, 2, seed=77)
    seq = fse_2d(n_ro=16, n_pe=8, etl=4, rf_dur=2e-3, rf_dt=10e-6, dwell=10e-6, esp=10e-3,
                 tr=0.5, n_shots=2)
    ref, Mref = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_PRECOMP_LANES, lanes)
    try:
        sig, M = run_both(mrsim, ctx, ph, seq, mrsim.GROUPED, precision)
    finally:
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_PRECOMP_LANES, 0)
    check(sig, M, ref, Mref, precision, M0max=float(np.max(ph.M0)))


@pytest.mark.parametrize("steps", [1, 2, 4, 8, 16, 32])
def test_precompute_fp32_block_lengths(mrsim, ctx, steps):
    """FP32 runs compose a few sub-steps in FP32 registers before each fold into
    the FP64 combined transition; every allowed block length keeps the FP32
    target, and an FP64 run ignores the setting."""
    from mrsim_inputs.phantom import continuous_phantom
    ph = continuous_phantom(13, 11, 3, 2, seed=78)
    seq = fse_2d(n_ro=16, n_pe=8, etl=4, rf_dur=2e-3, rf_dt=10e-6, dwell=10e-6, esp=10e-3,
                 tr=0.5, n_shots=2)
    ref, Mref = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_PRECOMP_STEPS, steps)
    try:
        for precision in (0, 1):
            sig, M = run_both(mrsim, ctx, ph, seq, mrsim.GROUPED, precision)
            check(sig, M, ref, Mref, precision, M0max=float(np.max(ph.M0)))
    finally:
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_PRECOMP_STEPS, 8)


def test_tuning_parameters_are_validated(mrsim, ctx):
    for param, bad in ((mrsim.TUNE_FUSED_NI, 3), (mrsim.TUNE_PRECOMP_LANES, 64),
                       (mrsim.TUNE_PRECOMP_STEPS, 64), (mrsim.TUNE_CELL_NI, 1),
                       (mrsim.TUNE_TWO_AXIS, 2), (mrsim.TUNE_CELL_ROWS, 3), (8, 1), (-1, 1)):
        with pytest.raises(mrsim.MrsimError):
            mrsim.mrsim_set_tuning(ctx.h, param, bad)
    before = mrsim.mrsim_get_tuning(ctx.h, mrsim.TUNE_PRECOMP_STEPS)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_PRECOMP_STEPS, 8)
    assert mrsim.mrsim_get_tuning(ctx.h, mrsim.TUNE_PRECOMP_STEPS) == 8
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_PRECOMP_STEPS, before)


def cancelling_group_case(ni, n_a):
    """Two x-groups, A (the first n_a isochromats, x = -1 cm) and B (the rest,
    x = +1 cm), in one 1024-isochromat phantom whose initial magnetization is
    (+-1, 0, 0).  With no pulse before the with-ADC windows every block-sum
    term is exactly +-1, so sums are exact in FP32.  B's terms total exactly
    zero, while the part of B that shares the first warp of the fused kernel
    with A sums to +2 and the next warp's part to -2.  A pulse after the
    windows makes z the secondary layout key; one z per 32-isochromat block
    keeps B's blocks in index order in the layout.  20 windows span more
    than one batch of staged windows."""
    K = 1024
    k = np.arange(K)
    w = 32 * ni  # isochromats in one warp of the fused kernel
    sign = np.where(k % 2 == 0, 1.0, -1.0)
    first = np.arange(n_a, w)          # B in the first warp: sum +2
    sign[first] = np.where(np.arange(first.size) < first.size // 2 + 1, 1.0, -1.0)
    second = np.arange(w, 2 * w)       # the next warp: sum -2
    sign[second] = np.where(np.arange(w) < w // 2 - 1, 1.0, -1.0)
    sign[:n_a] = 1.0
    assert sign[n_a:].sum() == 0 and sign[first].sum() == 2 and sign[second].sum() == -2
    f = lambda a: np.ascontiguousarray(a, np.float32)
    ph = Phantom(x=f(np.where(k < n_a, -0.01, 0.01)), y=f(np.zeros(K)),
                 z=f((k // 32 - 16) * 1e-4), T1=f(np.full(K, 1.0)), T2=f(np.full(K, 0.1)),
                 dB0=f(np.zeros(K)), M0=f(np.ones(K)),
                 M_init=f(np.stack([sign, np.zeros(K), np.zeros(K)])))
    b = SeqBuilder()
    for _ in range(40):
        b.add(1e-3, 1)
        b.readout(8, 10e-6, (5e-3, 0.0, 0.0))
    b.add(1e-3, 1)
    b.rf_sinc(30, "x", 1e-3, 10e-6)
    return ph, b.build()


@pytest.mark.parametrize("cell,ni,n_a", [(0, 1, 16), (0, 2, 32), (0, 4, 64), (4, 4, 64),
                                         (8, 8, 128)])
def test_group_sum_cancelling_exactly(mrsim, ctx, cell, ni, n_a):
    """A group whose staged with-ADC partials cancel to exactly zero in one
    window must leave nothing behind for the window that reuses its staging
    slot (a leftover partial once leaked into a later window).  Cells of 32
    isochromats keep the cell form's threads on the same isochromats as the
    per-isochromat form's."""
    ph, seq = cancelling_group_case(ni, n_a)
    ref, Mref = oracle.simulate(ph, seq)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_NI, cell)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_FUSED_NI, min(ni, 4))
    try:
        sig, M = run_both(mrsim, ctx, ph, seq, mrsim.GROUPED, 0)
        check(sig, M, ref, Mref, 0)
    finally:
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_FUSED_NI, 4)
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_NI, 8)
