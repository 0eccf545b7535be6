"""Two-axis gradient types on the GPU (the paper's open problem, Sec. 5).

Subsequences whose gradients use exactly two axes are grouped on both
positions: keys (r_a, r_b, T1, T2, dB0[, b1]) (Sec. 2.4 / Fig. 2 extended by
one word), one combined transition per group (Eq. 7 with both positions in
the phase) and with-ADC phases with both gradient moments (Eq. 10).  Group ids
are compared bit for bit with the oracle's numbering; signals and final
states with the per-isochromat FP64 oracle (FP32 1e-4, FP64 1e-10 signal
rel-L2; M_final 1e-4 / 1e-7 of max M0).
"""

import numpy as np
import pytest

import oracle
from mrsim_inputs import SeqBuilder
from mrsim_inputs.phantom import continuous_phantom, ellipse_phantom
from mrsim_inputs.sequence import radial_2d

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}
TOL_M = {0: 1e-4, 1: 1e-7}


@pytest.fixture(scope="module")
def ctx(mrsim):
    c = mrsim.Context(0)
    yield c
    c.close()


def yz_sequence():
    """A slice tilted from z toward y (the pulse on Gy and Gz, G_YZ), a Gx
    readout and a with-ADC window on Gy and Gz (G_YZ)."""
    b = SeqBuilder()
    for p in range(3):
        gss = b.rf_sinc(60, "x", 1e-3, 10e-6, 4.0, 0.01, direction=(0.0, 0.5, 0.8660254))
        b.add(1e-3, 1, g=(-3e-3, -0.25 * gss, -0.4330127 * gss))
        b.readout(16, 10e-6, (4e-3, 0.0, 0.0))
        b.add(0.5e-3, 1)
        b.readout(12, 10e-6, (0.0, (p - 1) * 2e-3, 3e-3))
        b.add(8e-3, 1, g=(0.0, 0.0, 2e-3))
    return b.build(kind="yz")


def spiral_like_sequence():
    """A hard 90 and one with-ADC window of twelve segments whose (Gx, Gy)
    turns from segment to segment: the with-ADC phase must carry both
    moments across segments."""
    b = SeqBuilder()
    b.rf_hard(90, "x", 0.2e-3, 10e-6)
    b.add(0.5e-3, 1)
    g = 4e-3
    for j in range(12):
        u = (j + 1) / 12
        t = 2.0 * u - 1.0
        c, s = (1 - t * t) / (1 + t * t), 2 * t / (1 + t * t)
        b.add(10e-6, 4, g=(g * u * c, g * u * s, 0.0), adc=True)
    b.add(1e-3, 1)
    return b.build(kind="spiral")


def run(mrsim, ctx, ph, seq, precision, fused_ni=4, cell_ni=8):
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_FUSED_NI, fused_ni)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_NI, cell_ni)
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    try:
        info = mrsim.mrsim_seq_info(hs)
        sig, M = ctx.run(hp, hs, hg, mrsim.GROUPED, precision, K=ph.K, want_M=True)
    finally:
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_FUSED_NI, 4)
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_CELL_NI, 8)
        ctx.free("grp", hg)
        ctx.free("seq", hs)
        ctx.free("ph", hp)
    return sig, M, info


def check(sig, M, ref, Mref, precision, M0max):
    e = oracle.rel_l2(sig, ref)
    assert e <= TOL[precision], f"signal rel-L2 {e:.3e}"
    em = float(np.max(np.abs(M - Mref))) / M0max
    assert em <= TOL_M[precision], f"M_final max error {em:.3e}"


def two_axis_types(info):
    g = info["gtype"][info["type"] != 2]
    return sorted({int(t) for t in g if t >= 5})


@pytest.mark.parametrize("name", ["radial", "radial_oblique", "yz"])
def test_two_axis_group_ids_bit_exact(mrsim, ctx, name):
    seq = {"radial": lambda: radial_2d(n_ro=16, n_spokes=6),
           "radial_oblique": lambda: radial_2d(n_ro=16, n_spokes=6, oblique_deg=20.0),
           "yz": yz_sequence}[name]()
    ph = ellipse_phantom(10, 9, 3, 3, seed=41)
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    types = two_axis_types(mrsim.mrsim_seq_info(hs))
    assert types, "no two-axis subsequence"
    for t in types:
        n, gid = mrsim.mrsim_group_info(hg, t, ph.K)
        ref, nref = oracle.group(ph, t)
        assert n == nref and np.array_equal(gid, ref), t
    ctx.free("grp", hg)
    ctx.free("seq", hs)
    ctx.free("ph", hp)


@pytest.mark.parametrize("oblique", [0.0, 20.0])
@pytest.mark.parametrize("precision", [0, 1])
def test_radial_grouped_on_two_positions(mrsim, ctx, oblique, precision):
    """Radial readouts (Gx + Gy windows) and, with an oblique slice, Gx + Gz
    pulses: z-subvoxels of a pixel share their (x, y) groups."""
    ph = ellipse_phantom(12, 12, 3, 3, seed=8)
    seq = radial_2d(n_ro=16, n_spokes=6, oblique_deg=oblique)
    ref, Mref = oracle.simulate(ph, seq)
    for ni in (1, 4):
        sig, M, info = run(mrsim, ctx, ph, seq, precision, fused_ni=ni)
        assert mrsim.G_XY in two_axis_types(info)
        if oblique:
            assert mrsim.G_XZ in two_axis_types(info)
        check(sig, M, ref, Mref, precision, float(np.max(ph.M0)))


@pytest.mark.parametrize("precision", [0, 1])
def test_two_axis_with_rf_scale_initial_state_and_direct_advance(mrsim, ctx, precision):
    """Per-isochromat dB0 and b1 (about one group per isochromat, so the
    advance is evaluated per isochromat) and a given initial state."""
    ph = continuous_phantom(8, 8, 2, 2, seed=12)
    rng = np.random.default_rng(3)
    ph.M_init = rng.uniform(-0.5, 0.5, (3, ph.K)).astype(np.float32)
    seq = radial_2d(n_ro=8, n_spokes=5, oblique_deg=-15.0)
    ref, Mref = oracle.simulate(ph, seq)
    sig, M, info = run(mrsim, ctx, ph, seq, precision)
    assert two_axis_types(info)
    check(sig, M, ref, Mref, precision, float(np.max(ph.M0)))


@pytest.mark.parametrize("name", ["spiral", "yz"])
@pytest.mark.parametrize("precision", [0, 1])
def test_two_axis_windows_and_pulses(mrsim, ctx, name, precision):
    """A with-ADC window of twelve turning (Gx, Gy) segments (both moments
    carried per sample), and pulses and windows on Gy + Gz next to a Gx
    readout (cells of the layout with a two-axis secondary type)."""
    seq = spiral_like_sequence() if name == "spiral" else yz_sequence()
    ph = ellipse_phantom(10, 10, 4, 3, seed=9)
    ref, Mref = oracle.simulate(ph, seq)
    for cell in (8, 0):
        sig, M, info = run(mrsim, ctx, ph, seq, precision, cell_ni=cell)
        assert two_axis_types(info)
        check(sig, M, ref, Mref, precision, float(np.max(ph.M0)))


def test_radial_benchmark_sequence_on_a_reduced_phantom(mrsim, ctx):
    """The benchmark's radial sequence itself (3 ms pulses at 1 us, 64 spokes
    of 256 samples) on a 64 x 64 x 4 phantom of the same construction."""
    from mrsim_inputs import configs
    seq = configs.radial_sequence()
    ph = configs.small_phantom(64, 64, 4)
    ref, Mref = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
    sig, M, info = run(mrsim, ctx, ph, seq, 0)
    assert mrsim.G_XY in two_axis_types(info)
    check(sig, M, ref, Mref, 0, float(np.max(ph.M0)))
