"""Two-axis gradient types (the paper's open problem, Sec. 5): subsequences
whose gradients use exactly two axes, grouped on both positions.  The oracle's
grouped simulator with these types is pinned to its per-isochromat simulator
(the definition, Eqs. 1-6) and its groups to a brute-force numbering."""

import dataclasses

import numpy as np
import pytest

import oracle
from mrsim_inputs.phantom import continuous_phantom, ellipse_phantom
from mrsim_inputs.sequence import radial_2d


def test_radial_classification():
    """Spokes along x or y are one-axis windows; the others use Gx and Gy
    together and become G_XY only when two-axis types are asked for; an oblique
    slice puts the pulses on Gx and Gz (G_XZ)."""
    seq = radial_2d(n_ro=16, n_spokes=8)
    for two_axis in (False, True):
        q = oracle.classify(seq, two_axis=two_axis)
        adc = q["gtype"][q["type"] == oracle.ADC]
        rf = q["gtype"][q["type"] == oracle.RF]
        assert adc[0] == oracle.G_X and adc[4] == oracle.G_Y
        other = oracle.G_XY if two_axis else oracle.G_GENERAL
        assert all(g == other for i, g in enumerate(adc) if i not in (0, 4))
        assert np.all(rf == oracle.G_Z)
    q = oracle.classify(radial_2d(n_ro=16, n_spokes=4, oblique_deg=20.0), two_axis=True)
    assert np.all(q["gtype"][q["type"] == oracle.RF] == oracle.G_XZ)
    assert np.array_equal(oracle.classify(seq)["gtype"],
                          np.where(oracle.classify(seq, two_axis=True)["gtype"] >= oracle.G_XY,
                                   oracle.G_GENERAL, oracle.classify(seq)["gtype"]))


def brute_ids(keys):
    seen, out = {}, []
    for key in keys:
        out.append(seen.setdefault(key, len(seen)))
    return np.asarray(out)


@pytest.mark.parametrize("gtype,axes", [(oracle.G_XY, ("x", "y")), (oracle.G_XZ, ("x", "z")),
                                        (oracle.G_YZ, ("y", "z"))])
def test_two_axis_group_ids_are_first_occurrence_numbers(gtype, axes):
    ph = continuous_phantom(6, 6, 3, 2, seed=31)
    ph.dB0 = np.round(ph.dB0 / 8.0).astype(np.float32) * 8.0  # repeated values
    ph.b1 = None
    gid, n = oracle.group(ph, gtype)
    a, b = (getattr(ph, n_) for n_ in axes)
    keys = [(a[k].item(), b[k].item(), ph.T1[k].item(), ph.T2[k].item(), ph.dB0[k].item())
            for k in range(ph.K)]
    ref = brute_ids(keys)
    assert n == ref.max() + 1
    assert np.array_equal(gid, ref)


def test_two_axis_groups_share_across_the_third_axis():
    """Keyed on (x, y), the z-subvoxels of a pixel share groups: doubling
    them doubles K and leaves the G_XY count unchanged (cf. the subvoxel
    observation beside Table 4), while the G_XZ count doubles."""
    p1 = ellipse_phantom(16, 16, 4, 3, seed=5)
    p2 = ellipse_phantom(16, 16, 8, 3, seed=5)
    n1 = oracle.group(p1, oracle.G_XY)[1]
    n2 = oracle.group(p2, oracle.G_XY)[1]
    assert p2.K == 2 * p1.K and n1 == n2
    assert n1 == np.unique(np.stack([p1.x, p1.y, p1.T1, p1.T2, p1.dB0]), axis=1).shape[1]
    assert oracle.group(p2, oracle.G_XZ)[1] == 2 * oracle.group(p1, oracle.G_XZ)[1]


@pytest.mark.parametrize("oblique", [0.0, 20.0])
def test_grouped_two_axis_equals_ungrouped(oblique):
    """Grouped on two positions, radial readouts (Gx + Gy) and oblique pulses
    (Gx + Gz) give the per-isochromat signal and final state to rounding."""
    ph = ellipse_phantom(12, 12, 3, 3, seed=8)
    seq = radial_2d(n_ro=16, n_spokes=6, oblique_deg=oblique)
    ref, M_ref = oracle.simulate(ph, seq)
    sig, M = oracle.simulate_grouped(ph, seq, two_axis=True)
    assert oracle.rel_l2(sig, ref) <= 1e-12
    assert float(np.max(np.abs(M - M_ref))) <= 1e-12
    q = oracle.classify(seq, two_axis=True)
    assert np.any(q["gtype"] >= oracle.G_XY)  # the two-axis path was taken


def test_grouped_two_axis_with_rf_scale_and_initial_state():
    ph = continuous_phantom(8, 8, 2, 2, seed=12)
    rng = np.random.default_rng(3)
    ph.M_init = rng.uniform(-0.5, 0.5, (3, ph.K)).astype(np.float32)
    seq = radial_2d(n_ro=8, n_spokes=5, oblique_deg=-15.0)
    ref, M_ref = oracle.simulate(ph, seq)
    sig, M = oracle.simulate_grouped(ph, seq, two_axis=True)
    assert oracle.rel_l2(sig, ref) <= 1e-12
    assert float(np.max(np.abs(M - M_ref))) <= 1e-12


def test_two_axis_phase_needs_both_axes():
    """A phantom that differs from another only in y gives a different radial
    signal (both positions enter the with-ADC phase)."""
    ph = ellipse_phantom(8, 8, 1, 2, seed=4)
    seq = radial_2d(n_ro=8, n_spokes=3)
    s1, _ = oracle.simulate_grouped(ph, seq, two_axis=True, want_M=False)
    ph2 = dataclasses.replace(ph, y=(ph.y * np.float32(0.5)).astype(np.float32))
    s2, _ = oracle.simulate_grouped(ph2, seq, two_axis=True, want_M=False)
    r2, _ = oracle.simulate(ph2, seq, want_M=False)
    assert oracle.rel_l2(s2, r2) <= 1e-12 and oracle.rel_l2(s1, s2) > 1e-3


def spiral_like_sequence(n_turn_segs=12, samples=4, dwell=10e-6):
    """A hard 90 followed by one with-ADC window of several segments whose
    (Gx, Gy) turns from segment to segment (a coarse spiral), so the with-ADC
    phase must carry both gradient moments across segments."""
    from mrsim_inputs.sequence import SeqBuilder
    b = SeqBuilder()
    b.rf_hard(90, "x", 0.2e-3, 10e-6)
    b.add(0.5e-3, 1)
    g = 4e-3
    for j in range(n_turn_segs):
        u = (j + 1) / n_turn_segs
        # direction from a rational parametrisation of the angle 2 atan(t)
        t = 2.0 * u - 1.0
        c, s = (1 - t * t) / (1 + t * t), 2 * t / (1 + t * t)
        b.add(dwell, samples, g=(g * u * c, g * u * s, 0.0), adc=True)
    b.add(1e-3, 1)
    return b.build(kind="spiral")


def test_two_axis_window_of_many_segments():
    ph = ellipse_phantom(10, 10, 2, 3, seed=9)
    seq = spiral_like_sequence()
    q = oracle.classify(seq, two_axis=True)
    assert list(q["gtype"][q["type"] == oracle.ADC]) == [oracle.G_XY]
    ref, M_ref = oracle.simulate(ph, seq)
    sig, M = oracle.simulate_grouped(ph, seq, two_axis=True)
    assert oracle.rel_l2(sig, ref) <= 1e-12
    assert float(np.max(np.abs(M - M_ref))) <= 1e-12
