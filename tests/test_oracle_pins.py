"""Pins of the FP64 oracle against mathematics (not against itself).

Each test names the passage of the paper whose behaviour it fixes.  A
plausible mistake (sign of the rotation, order of D and R, dropped M0 column,
ADC sampled at the wrong instant, wrong gradient sign, transposed operand)
fails at least one of them.
"""

import math

import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

import oracle
from mrsim_inputs import Phantom, SeqBuilder, configs, grid_phantom
from mrsim_inputs.phantom import grid_coords

GB = 42.577478518e6
GAMMA = 2 * math.pi * GB


def make_phantom(x, y, z, T1, T2, dB0, M0, b1=None, M_init=None):
    f = lambda a: np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), np.shape(x)),
                                       dtype=np.float32)
    return Phantom(x=f(x), y=f(y), z=f(z), T1=f(T1), T2=f(T2), dB0=f(dB0), M0=f(M0),
                   b1=None if b1 is None else f(b1),
                   M_init=None if M_init is None else np.ascontiguousarray(M_init, np.float32))


def f32(v):
    return np.float64(np.float32(v))


# ---------------------------------------------------------------- P1 -------
def test_p1_free_precession_step_path_equals_closed_form():
    """Eqs. 4-5: with B1 = 0 (here RF scale b1 = 0 on RF segments, so the
    stepped Eq. A1/A2 path runs), D and R commute and the step product is the
    closed-form precession/relaxation."""
    rng = np.random.default_rng(1)
    K = 16
    x, y, z = rng.uniform(-0.1, 0.1, (3, K))
    T1 = rng.uniform(0.3, 1.5, K)
    T2 = rng.uniform(0.04, 0.2, K)
    dB0 = rng.normal(0, 30, K)
    M0 = rng.uniform(0.5, 1, K)
    Mi = rng.uniform(-1, 1, (3, K))
    ph = make_phantom(x, y, z, T1, T2, dB0, M0, b1=np.zeros(K), M_init=Mi)
    g = (3e-3, -2e-3, 1e-3)
    dt, n = 10e-6, 300
    b = SeqBuilder()
    b.add(dt, n, b1=(1e-6, 0.0), g=g)  # classified with-RF; b1 scale 0 removes B1
    seq = b.build()
    _, M = oracle.simulate(ph, seq)
    t = dt * n
    X, Y, Z, T1_, T2_, dB_, M0_ = (np.float64(a) for a in (ph.x, ph.y, ph.z, ph.T1, ph.T2, ph.dB0, ph.M0))
    gx, gy, gz = (f32(v) for v in g)
    phi = GAMMA * (gx * X + gy * Y + gz * Z) * t + 2 * math.pi * dB_ * t
    mxy0 = np.float64(ph.M_init[0]) + 1j * np.float64(ph.M_init[1])
    mxy = mxy0 * np.exp(-t / T2_) * np.exp(-1j * phi)
    mz = M0_ + (np.float64(ph.M_init[2]) - M0_) * np.exp(-t / T1_)
    assert np.max(np.abs(M[0] - mxy.real)) < 1e-12
    assert np.max(np.abs(M[1] - mxy.imag)) < 1e-12
    assert np.max(np.abs(M[2] - mz)) < 1e-12
    # the relaxation-segment path (no RF) gives the same
    b2 = SeqBuilder()
    b2.add(dt, n, g=g)
    _, M2 = oracle.simulate(ph, b2.build())
    assert np.max(np.abs(M2 - M)) < 1e-12


# ---------------------------------------------------------------- P2 -------
@pytest.mark.parametrize("phase,expect", [("x", lambda a: (0.0, math.sin(a), math.cos(a))),
                                          ("y", lambda a: (-math.sin(a), 0.0, math.cos(a)))])
def test_p2_hard_pulse_flip_angle(phase, expect):
    """Eq. A2 with theta = -gamma |B| dt: a hard pulse along +x flips (0,0,M0)
    to (0, M0 sin a, M0 cos a); along +y to (-M0 sin a, 0, M0 cos a)."""
    ph = make_phantom(np.zeros(1), 0, 0, np.inf, np.inf, 0, 0.8)
    for flip in (10.0, 90.0, 137.0, 180.0, 270.0):
        b = SeqBuilder()
        b.rf_hard(flip, phase, 200e-6, 1e-6)
        seq = b.build()
        _, M = oracle.simulate(ph, seq)
        a = GAMMA * f32(seq.b1re[0] if phase == "x" else seq.b1im[0]) * 1e-6 * 200
        assert abs(a - flip * math.pi / 180) < 1e-6
        e = np.array(expect(a)) * f32(0.8)
        assert np.max(np.abs(M[:, 0] - e)) < 1e-13
        assert abs(np.linalg.norm(M[:, 0]) - f32(0.8)) < 1e-13


def test_p2_off_resonant_rotation_about_effective_field():
    """Constant B: N steps compose to one rotation about B by -gamma|B|N dt
    (scipy rotation as the independent reference)."""
    ph = make_phantom(np.array([0.01]), 0.0, 0.0, np.inf, np.inf, 150.0, 1.0,
                      M_init=np.array([[0.3], [-0.2], [0.9]]))
    b = SeqBuilder()
    b.add(2e-6, 500, b1=(3e-6, 1e-6), g=(4e-3, 0, 0))
    seq = b.build()
    _, M = oracle.simulate(ph, seq)
    B = np.array([f32(3e-6), f32(1e-6),
                  f32(4e-3) * f32(0.01) + 2 * math.pi * f32(150.0) / GAMMA])
    th = -GAMMA * np.linalg.norm(B) * 2e-6 * 500
    Rm = Rotation.from_rotvec(th * B / np.linalg.norm(B)).as_matrix()
    m0 = np.array([f32(0.3), f32(-0.2), f32(0.9)])
    assert np.max(np.abs(M[:, 0] - Rm @ m0)) < 1e-12


# ---------------------------------------------------------------- P3 -------
def test_p3_spin_echo_refocuses_gradient_dephasing_exactly():
    """90x - tau - 180y - tau with dephasing from a gradient lobe and T = inf:
    every isochromat returns to (0, M0, 0) at the echo.  The exact expectation
    is built from scipy rotations: Rz(-phi) Ry(-a180) Rz(-phi) Rx(-a90) e_z,
    with the float32 pulse amplitudes and gradient (Eq. 4, Eq. A2)."""
    K = 64
    x = np.linspace(-0.1, 0.1, K)
    ph = make_phantom(x, 0.0, 0.0, np.inf, np.inf, 0.0, 1.0)
    b = SeqBuilder()
    b.rf_hard(90, "x", 10e-6, 1e-6)
    b.add(1e-3, 1, g=(5e-3, 0, 0))
    b.rf_hard(180, "y", 10e-6, 1e-6)
    b.add(1e-3, 1, g=(5e-3, 0, 0))
    seq = b.build()
    _, M = oracle.simulate(ph, seq)
    a90 = GAMMA * f32(seq.b1re[0]) * 1e-6 * 10
    a180 = GAMMA * f32(seq.b1im[2]) * 1e-6 * 10
    R90 = Rotation.from_rotvec([-a90, 0, 0]).as_matrix()
    R180 = Rotation.from_rotvec([0, -a180, 0]).as_matrix()
    for k in range(K):
        phi = GAMMA * f32(5e-3) * np.float64(ph.x[k]) * 1e-3
        P = Rotation.from_rotvec([0, 0, -phi]).as_matrix()
        ex = P @ R180 @ P @ R90 @ np.array([0.0, 0.0, 1.0])
        assert np.max(np.abs(M[:, k] - ex)) < 1e-12
    # and the echo is (0, M0, 0) up to the float32 flip-angle rounding
    assert np.max(np.abs(M - np.array([[0.0], [1.0], [0.0]]))) < 1e-6


def test_p3_spin_echo_refocuses_off_resonance_with_t2_decay():
    """|M_xy(TE)| = M0 exp(-TE/T2) independent of dB0 (tolerance from the
    finite 1 ns pulses: off-resonance tilt ~ dw * dt)."""
    K = 9
    dB0 = np.linspace(-100, 100, K)
    ph = make_phantom(np.zeros(K), 0.0, 0.0, 0.8, 0.05, dB0, 1.0)
    tau = 10e-3
    b = SeqBuilder()
    b.rf_hard(90, "x", 1e-9, 1e-9)
    b.add(tau, 1)
    b.rf_hard(180, "y", 1e-9, 1e-9)
    b.add(tau, 1)
    _, M = oracle.simulate(ph, b.build())
    mag = np.hypot(M[0], M[1])
    assert np.max(np.abs(mag - math.exp(-2 * tau / f32(0.05)))) < 1e-6
    assert np.max(np.abs(M[0])) < 1e-5  # phase refocused onto +y


# ---------------------------------------------------------------- P4 -------
def _fixed_point(alpha, phi, TR, T1, T2):
    """Steady state of the one-TR map M <- D(TR) Rz(phi) Rx(alpha) M + b M0
    (independent textbook construction with scipy rotations)."""
    Rx = Rotation.from_rotvec([-alpha, 0, 0]).as_matrix()   # theta = -alpha about +x
    Rz = Rotation.from_rotvec([0, 0, -phi]).as_matrix()     # M_xy * exp(-i phi)
    E1, E2 = math.exp(-TR / T1), math.exp(-TR / T2)
    D = np.diag([E2, E2, E1])
    A = D @ Rz @ Rx
    bvec = np.array([0, 0, 1 - E1])
    return np.linalg.solve(np.eye(3) - A, bvec)


@pytest.mark.parametrize("T2,dB0", [(0.05, 13.0), (0.2, -37.0)])
def test_p4_gradient_echo_steady_state_fixed_point(T2, dB0):
    T1, TR, flip = 0.3, 10e-3, 30.0
    ph = make_phantom(np.zeros(1), 0, 0, T1, T2, dB0, 1.0)
    b = SeqBuilder()
    n = 1200
    for _ in range(n):
        b.rf_hard(flip, "x", 1e-9, 1e-9)
        b.add(TR - 1e-9, 1)
    seq = b.build()
    _, M = oracle.simulate(ph, seq, memo=True)
    a = GAMMA * f32(seq.b1re[0]) * 1e-9
    phi = 2 * math.pi * f32(dB0) * (TR - 1e-9)
    Ms = _fixed_point(a, phi, TR - 1e-9, f32(T1), f32(T2))
    assert np.max(np.abs(M[:, 0] - Ms)) < 1e-7


def test_p4_ernst_spoiled_limit():
    """T2 << TR: Mz just before each pulse -> M0 (1-E1)/(1-E1 cos a) (Ernst)."""
    T1, T2, TR, flip = 0.3, 1e-4, 50e-3, 30.0
    ph = make_phantom(np.zeros(1), 0, 0, T1, T2, 0.0, 1.0)
    b = SeqBuilder()
    for _ in range(400):
        b.rf_hard(flip, "x", 1e-9, 1e-9)
        b.add(TR - 1e-9, 1)
    seq = b.build()
    _, M = oracle.simulate(ph, seq, memo=True)
    a = GAMMA * f32(seq.b1re[0]) * 1e-9
    E1 = math.exp(-(TR - 1e-9) / f32(T1))
    assert abs(M[2, 0] - (1 - E1) / (1 - E1 * math.cos(a))) < 1e-8


# ---------------------------------------------------------------- P5 -------
def test_p5_signal_is_centred_dft_of_m0():
    """Eq. 6 with T = inf, dB0 = 0 and M(0) = (0, M0, 0): the Cartesian
    readout samples are i * DFT(M0) with kernel exp(-i 2 pi k.r); compared with
    numpy's FFT.  Fixes the gradient sign, the ADC instant and the signal
    convention M_xy = Mx + i My."""
    n = 16
    fov = 0.256
    rng = np.random.default_rng(5)
    M0map = rng.uniform(0.2, 1.0, (n, n))
    ph = grid_phantom(M0map, nz=1, fov=fov)
    ph.M_init = np.stack([np.zeros(ph.K), ph.M0.astype(np.float64), np.zeros(ph.K)]).astype(np.float32)
    dk = 1.0 / fov
    dwell = 10e-6
    g_ro = dk / (GB * dwell)
    d = 1e-3
    b = SeqBuilder()
    kx = ky = 0.0
    for p in range(n):
        kx_t, ky_t = -(n // 2 + 1) * dk, (p - n // 2) * dk
        b.add(d, 1, g=((kx_t - kx) / GB / d, (ky_t - ky) / GB / d, 0))
        kx, ky = kx_t, ky_t
        b.readout(n, dwell, (g_ro, 0, 0))
        kx += n * dk
    seq = b.build()
    sig, _ = oracle.simulate(ph, seq, want_M=False)
    S = sig.reshape(n, n)  # [line p, sample i]
    M0_32 = ph.M0.astype(np.float64).reshape(n, n)
    ref = 1j * np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(M0_32)))
    # exact k-space positions differ from the nominal grid only by the float32
    # rounding of the gradient amplitudes (relative 6e-8 of phases up to
    # ~30 rad accumulated over the prephaser lobes)
    assert oracle.rel_l2(S, ref) < 1e-5


def test_p5_exact_dft_with_actual_gradient_areas():
    """Same as above but the reference uses the float32 gradient areas that
    the sequence really holds, so the match is to rounding (1e-12)."""
    n = 8
    fov = 0.256
    rng = np.random.default_rng(6)
    ph = grid_phantom(rng.uniform(0.2, 1.0, (n, n)), nz=1, fov=fov)
    ph.M_init = np.stack([np.zeros(ph.K), ph.M0.astype(np.float64), np.zeros(ph.K)]).astype(np.float32)
    dk, dwell = 1.0 / fov, 10e-6
    b = SeqBuilder()
    kx = ky = 0.0
    for p in range(n):
        kx_t, ky_t = -(n // 2 + 1) * dk, (p - n // 2) * dk
        b.add(1e-3, 1, g=((kx_t - kx) / GB / 1e-3, (ky_t - ky) / GB / 1e-3, 0))
        kx, ky = kx_t, ky_t
        b.readout(n, dwell, (dk / (GB * dwell), 0, 0))
        kx += n * dk
    seq = b.build()
    sig, _ = oracle.simulate(ph, seq, want_M=False)
    # moments from the float32 sequence itself
    mx = my = 0.0
    ks = []
    for j in range(seq.n_seg):
        g = (f32(seq.gx[j]), f32(seq.gy[j]))
        for r in range(seq.repeat[j]):
            if seq.adc[j]:
                ks.append((mx + g[0] * seq.dt[j] * (r + 1), my + g[1] * seq.dt[j] * (r + 1)))
        mx += g[0] * seq.dt[j] * seq.repeat[j]
        my += g[1] * seq.dt[j] * seq.repeat[j]
    ks = np.array(ks) * GAMMA
    X, Y, M0 = np.float64(ph.x), np.float64(ph.y), np.float64(ph.M0)
    ref = np.array([1j * np.sum(M0 * np.exp(-1j * (k[0] * X + k[1] * Y))) for k in ks])
    assert oracle.rel_l2(sig, ref) < 1e-12


# ---------------------------------------------------------------- P6 -------
def test_p6_linearity_in_m0():
    ph, seq = configs.se_32()
    seq = _truncate(seq, 3)
    # M0 on a 2^-10 grid so that 3 * M0 is exact in float32 as well
    ph.M0 = (np.round(ph.M0.astype(np.float64) * 1024) / 1024).astype(np.float32)
    s1, M1 = oracle.simulate(ph, seq)
    ph2 = Phantom(**{**ph.__dict__})
    ph2.M0 = ph.M0 * np.float32(2.0)
    s2, M2 = oracle.simulate(ph2, seq)
    assert np.array_equal(s2, 2 * s1)  # power-of-two scaling is exact
    ph3 = Phantom(**{**ph.__dict__})
    ph3.M0 = (ph.M0.astype(np.float64) * 3).astype(np.float32)
    s3, _ = oracle.simulate(ph3, seq)
    assert oracle.rel_l2(s3, 3 * s1) < 1e-13


def _truncate(seq, n_tr):
    """First n_tr TRs of a spin-echo sequence (by its ADC count)."""
    adc_seen = 0
    for j in range(seq.n_seg):
        if seq.adc[j]:
            adc_seen += 1
            if adc_seen == n_tr:
                end = j + 1
                break
    from mrsim_inputs import Sequence
    return Sequence(**{k: v[:end].copy() for k, v in seq.arrays().items()}, meta=dict(seq.meta))


# ---------------------------------------------------------------- P7 -------
def test_p7_transition_composition_is_associative():
    """Eq. 7: T(t0, t2) = T(t1, t2) T(t0, t1) (affine composition, M0 column)."""
    ph, seq = configs.se_32()
    q = oracle.classify(seq)
    i = int(np.nonzero(q["type"] == oracle.RF)[0][0])
    a, c = int(q["seg_begin"][i]), int(q["seg_end"][i])
    bmid = (a + c) // 2 + 7
    kw = dict(x=0.01, y=-0.02, z=0.003, T1=0.9, T2=0.08, dB0=12.0, b1=1.05)
    A, bb = oracle.transition(seq, a, c, **kw)
    A1, b1 = oracle.transition(seq, a, bmid, **kw)
    A2, b2 = oracle.transition(seq, bmid, c, **kw)
    assert np.max(np.abs(A - A2 @ A1)) < 1e-13
    assert np.max(np.abs(bb - (A2 @ b1 + b2))) < 1e-13


def test_p7_transition_applied_equals_stepping():
    ph = make_phantom(np.array([0.01]), -0.02, 0.003, 0.9, 0.08, 12.0, 0.7, b1=1.05,
                      M_init=np.array([[0.1], [0.2], [0.5]]))
    _, seq = configs.se_32()
    q = oracle.classify(seq)
    i = int(np.nonzero(q["type"] == oracle.RF)[0][0])
    a, c = int(q["seg_begin"][i]), int(q["seg_end"][i])
    from mrsim_inputs import Sequence
    sub = Sequence(**{k: v[a:c].copy() for k, v in seq.arrays().items()})
    _, M = oracle.simulate(ph, sub)
    A, bb = oracle.transition(seq, a, c, x=f32(0.01), y=f32(-0.02), z=f32(0.003), T1=f32(0.9),
                              T2=f32(0.08), dB0=f32(12.0), b1=f32(1.05))
    m0 = np.array([f32(0.1), f32(0.2), f32(0.5)])
    assert np.max(np.abs(M[:, 0] - (A @ m0 + bb * f32(0.7)))) < 1e-13


# ---------------------------------------------------------------- P8 -------
@pytest.mark.parametrize("which", ["se", "fse", "epi"])
def test_p8_grouped_equals_ungrouped(which):
    """Sec. 2.3: with shared U inside a group, the grouped with-RF combined
    transitions and the three-step with-ADC method (Eqs. 8-10) reproduce the
    per-isochromat simulation exactly (up to rounding)."""
    if which == "se":
        ph, seq = configs.se_32()
        seq = _truncate(seq, 4)
    elif which == "fse":
        ph = configs.small_phantom(16, 16, 4)
        from mrsim_inputs.sequence import fse_2d
        seq = fse_2d(n_ro=16, n_pe=16, etl=4, rf_dur=1e-3, rf_dt=10e-6, dwell=10e-6,
                     esp=8e-3, tr=0.2, n_shots=2)
    else:
        ph = configs.small_phantom(16, 16, 4)
        from mrsim_inputs.sequence import epi_2d
        seq = epi_2d(n_ro=16, n_lines=16, rf_dur=1e-3, rf_dt=10e-6, ramp=20e-6, raster=5e-6)
    s_u, M_u = oracle.simulate(ph, seq)
    s_g, M_g = oracle.simulate_grouped(ph, seq)
    assert oracle.rel_l2(s_g, s_u) < 1e-12
    assert np.max(np.abs(M_g - M_u)) < 1e-12


def test_p8_group_ids_match_brute_force_numbering():
    ph = configs.small_phantom(16, 16, 4)
    for gtype, pos in ((oracle.G_X, ph.x), (oracle.G_Z, ph.z), (oracle.G_Y, ph.y),
                       (oracle.G_NONE, None)):
        gid, ng = oracle.group(ph, gtype)
        seen = {}
        ref = np.empty(ph.K, np.int32)
        for k in range(ph.K):
            key = ((0.0 if pos is None else float(pos[k]) + 0.0), float(ph.T1[k]),
                   float(ph.T2[k]), float(ph.dB0[k]) + 0.0)
            ref[k] = seen.setdefault(key, len(seen))
        assert ng == len(seen)
        assert np.array_equal(gid, ref)


def test_p8_group_keys_canonicalise_negative_zero_and_reject_nan():
    x = np.array([0.0, -0.0, 1e-3], np.float32)
    ph = make_phantom(x, 0, 0, 1.0, 0.1, 0.0, 1.0)
    ph.x = x
    gid, ng = oracle.group(ph, oracle.G_X)
    assert ng == 2 and gid[0] == gid[1] == 0 and gid[2] == 1
    ph.T2 = np.array([0.1, np.nan, 0.1], np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.group(ph, oracle.G_X)


# ---------------------------------------------------------------- P9 -------
def _label_phantom(lab, nz, sub_x=1):
    """Piecewise-constant phantom from a label map; each pixel split into
    sub_x subvoxels along x."""
    ny, nx = lab.shape
    lab2 = np.repeat(lab, sub_x, axis=1)
    xs, ys, zs = grid_coords(nx * sub_x, ny, nz, 0.256, 0.02)
    T1 = np.array([1.0, 0.5, 0.8, 1.2, 0.6])
    T2 = np.array([0.1, 0.05, 0.08, 0.12, 0.07])
    dB0 = np.array([0.0, 5.0, -3.0, 0.0, 7.5])
    from mrsim_inputs.phantom import _expand
    d = _expand(lab2, xs, ys, zs, (T1, T2, dB0, np.ones(5)))
    return Phantom(**d)


def test_p9_group_counts_of_piecewise_constant_phantom():
    """Group counts follow from the region layout: K_g(x) = sum over x columns
    of the distinct regions in the column, K_g(z) = nz * distinct regions,
    K_g(none) = distinct regions; doubling subvoxels along x doubles K_g(x)
    (Table 4's observation, exact here)."""
    rng = np.random.default_rng(9)
    lab = rng.integers(0, 5, (12, 10))
    lab[3:6, 2:8] = 4
    nz = 3
    ph = _label_phantom(lab, nz)
    _, ngx = oracle.group(ph, oracle.G_X)
    _, ngy = oracle.group(ph, oracle.G_Y)
    _, ngz = oracle.group(ph, oracle.G_Z)
    _, ng0 = oracle.group(ph, oracle.G_NONE)
    assert ngx == sum(len(set(lab[:, i])) for i in range(lab.shape[1]))
    assert ngy == sum(len(set(lab[j, :])) for j in range(lab.shape[0]))
    assert ngz == nz * len(set(lab.ravel()))
    assert ng0 == len(set(lab.ravel()))
    ph2 = _label_phantom(lab, nz, sub_x=2)
    _, ngx2 = oracle.group(ph2, oracle.G_X)
    _, ngz2 = oracle.group(ph2, oracle.G_Z)
    assert ngx2 == 2 * ngx and ngz2 == ngz


# ---------------------------------------------------------------- P10 ------
@pytest.mark.parametrize("name,n_rf,n_adc,n_samples", [("se", 64, 32, 1024),
                                                       ("fse", 272, 256, 65536),
                                                       ("epi", 1, 128, 16384)])
def test_p10_subsequence_counts(name, n_rf, n_adc, n_samples):
    seq = {"se": lambda: configs.se_32()[1], "fse": configs.fse_sequence,
           "epi": configs.epi_sequence}[name]()
    q = oracle.classify(seq)
    assert np.sum(q["type"] == oracle.RF) == n_rf
    assert np.sum(q["type"] == oracle.ADC) == n_adc
    assert int(np.sum(q["n_samples"])) == n_samples
    assert set(q["gtype"][q["type"] == oracle.RF]) == {oracle.G_Z}
    assert set(q["gtype"][q["type"] == oracle.ADC]) == {oracle.G_X}
    # alternation: no two subsequences of the same type are adjacent
    assert np.all(q["type"][1:] != q["type"][:-1])


def test_classification_truth_table():
    b = SeqBuilder()
    b.add(1e-6, 1, b1=(1e-6, 0), g=(0, 0, 1e-3))     # RF, Gz-only
    b.add(1e-6, 2, b1=(0, 1e-6), g=(0, 0, -0.0))     # RF continues; -0 counts as zero
    b.add(1e-3, 1, g=(1e-3, 1e-3, 0))                # relax, general
    b.add(1e-6, 4, g=(0, 2e-3, 0), adc=True)         # ADC, Gy-only
    b.add(1e-3, 1)                                   # relax, no grads
    b.add(1e-6, 3, b1=(1e-6, 0), g=(1e-3, 0, 1e-3))  # RF, general
    b.add(1e-6, 3, adc=True)                         # ADC, no grads
    q = oracle.classify(b.build())
    assert list(q["type"]) == [oracle.RF, oracle.RELAX, oracle.ADC, oracle.RELAX, oracle.RF,
                               oracle.ADC]
    assert list(q["gtype"]) == [oracle.G_Z, oracle.G_GENERAL, oracle.G_Y, oracle.G_NONE,
                                oracle.G_GENERAL, oracle.G_NONE]
    assert list(q["n_samples"]) == [0, 0, 4, 0, 0, 3]
    assert list(q["seg_begin"]) == [0, 2, 3, 4, 5, 6]
    b2 = SeqBuilder()
    b2.add(1e-6, 1, b1=(1e-6, 0), adc=True)
    with pytest.raises(oracle.OracleError):
        oracle.classify(b2.build())


def test_rf_content_ids_follow_exact_equality():
    _, seq = configs.se_32()
    q = oracle.classify(seq)
    rf = q["type"] == oracle.RF
    assert list(q["content_id"][rf][:4]) == [0, 1, 0, 1]  # 90x, 180y alternate


# ---------------------------------------------------------------- P11 ------
def test_p11_splitting_error_is_first_order():
    """App. A uses an asymmetric splitting U = D R.  For constant B the exact
    propagator is the exponential of the 4x4 Bloch generator; the splitting
    error must shrink linearly with dt (it is O(dt), not exact)."""
    T1, T2, dB0 = 0.05, 0.02, 40.0
    B1 = 5e-6
    ph = make_phantom(np.zeros(1), 0, 0, T1, T2, dB0, 1.0)
    t_tot = 2e-3
    errs = []
    for n in (50, 100, 200, 400):
        b = SeqBuilder()
        b.add(t_tot / n, n, b1=(B1, 0))
        _, M = oracle.simulate(ph, b.build())
        wx = GAMMA * f32(B1)
        wz = 2 * math.pi * f32(dB0)
        r1, r2 = 1 / f32(T1), 1 / f32(T2)
        # dM/dt = gamma M x B + relaxation, B = (B1, 0, dB0/gamma_bar)
        Lg = np.array([[-r2, wz, 0, 0],
                       [-wz, -r2, wx, 0],
                       [0, -wx, -r1, r1],
                       [0, 0, 0, 0]])
        ex = scipy.linalg.expm(Lg * t_tot) @ np.array([0, 0, 1.0, 1.0])
        errs.append(np.linalg.norm(M[:, 0] - ex[:3]))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)
    assert errs[-1] < 1e-3


# ------------------------------------------------------- shortcuts ---------
def test_memo_and_adc_recurrence_match_direct_form():
    """The per-isochromat memoised combined transition (dynamic caching,
    Sec. 2.2) and the ADC phasor recurrence are exact rewrites."""
    ph, seq = configs.se_32()
    seq = _truncate(seq, 6)
    s0, M0 = oracle.simulate(ph, seq)
    s1, M1 = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
    assert oracle.rel_l2(s1, s0) < 1e-12
    assert np.max(np.abs(M1 - M0)) < 1e-12


def test_thread_count_does_not_change_result_beyond_rounding():
    ph, seq = configs.se_32()
    seq = _truncate(seq, 2)
    s1, M1 = oracle.simulate(ph, seq, n_threads=1)
    s3, M3 = oracle.simulate(ph, seq, n_threads=3)
    assert oracle.rel_l2(s3, s1) < 1e-14
    assert np.array_equal(M1, M3)


# ---------------------------------------------------------------- P13 coils
# Eq. 6 with P receive coils: A(p, t) = sum_k S(k, p) M_xy(k, t), S complex and
# constant in time.  Pinned by (a) a constant complex sensitivity, which must
# scale the one-coil signal by exactly that complex number (a dropped or
# conjugated term fails), (b) linearity in S, (c) an indicator map, which must
# reproduce the one-coil signal of the selected isochromats alone (weighting by
# the wrong isochromat or coil fails).

def _coil_case():
    from mrsim_inputs.sequence import spin_echo_2d
    ph = configs.small_phantom(8, 8, 2)
    seq = spin_echo_2d(n_ro=8, n_pe=8, n_tr=2)
    return ph, seq


def _with_coils(ph, S):
    import dataclasses
    return dataclasses.replace(ph, coils=np.ascontiguousarray(S, np.float32))


def test_p13_constant_coil_scales_signal():
    ph, seq = _coil_case()
    ref, _ = oracle.simulate(ph, seq, want_M=False)
    s0 = np.array([0.75 + 0.5j, -0.25 + 1.0j])
    S = np.zeros((2, 2, ph.K), np.float32)
    S[:, 0] = s0.real[:, None]
    S[:, 1] = s0.imag[:, None]
    sig, _ = oracle.simulate(_with_coils(ph, S), seq, want_M=False)
    assert sig.shape == (2, seq.n_samples)
    for p in range(2):
        assert oracle.rel_l2(sig[p], s0[p] * ref) <= 1e-14


def test_p13_signal_is_linear_in_sensitivity():
    from mrsim_inputs import coil_maps
    ph, seq = _coil_case()
    # multiples of 2^-12: the sum map S1 + S2 is then exact in float32
    S = np.round(coil_maps(ph, 2, seed=31).astype(np.float64) * 4096.0) / 4096.0
    S3 = np.concatenate([S, (S[0] + S[1])[None]], axis=0)
    sig, _ = oracle.simulate(_with_coils(ph, S3), seq, want_M=False)
    assert oracle.rel_l2(sig[2], sig[0] + sig[1]) <= 1e-12


def test_p13_indicator_coil_selects_isochromats():
    ph, seq = _coil_case()
    rng = np.random.default_rng(5)
    sel = np.sort(rng.choice(ph.K, ph.K // 3, replace=False))
    S = np.zeros((2, 2, ph.K), np.float32)
    S[0, 0, sel] = 1.0                 # coil 0: the selected isochromats
    S[1, 1, :] = 1.0                   # coil 1: S = i everywhere
    sig, _ = oracle.simulate(_with_coils(ph, S), seq, want_M=False)
    sub, _ = oracle.simulate(ph.subset(sel), seq, want_M=False)
    full, _ = oracle.simulate(ph, seq, want_M=False)
    assert oracle.rel_l2(sig[0], sub) <= 1e-12
    assert oracle.rel_l2(sig[1], 1j * full) <= 1e-14


def test_p13_bad_sensitivities_are_rejected():
    ph, seq = _coil_case()
    S = np.ones((1, 2, ph.K), np.float32)
    S[0, 1, 3] = np.nan
    with pytest.raises(RuntimeError):
        oracle.simulate(_with_coils(ph, S), seq, want_M=False)


# ------------------------------------------------------- P14 reconstruction
# Cartesian reconstruction (the paper's FFT reconstruction of SE / FSE data;
# EPI on flat-tops only is Cartesian after line reversal).  Pinned by (a) an
# explicit centred DFT written as matrices (independent of numpy's FFT) whose
# k-space, read out through the layout, must reconstruct to the image, and
# (b) the physics: with T1 = T2 = inf, dB0 = 0 and one z plane every isochromat
# is excited alike, so the image of the simulated SE, FSE and EPI k-space must
# be a constant complex multiple of the M0 map (a row flip, a wrong readout
# direction or a one-column shift fails).

def _centred_dft(n):
    k = np.arange(n) - n // 2
    return np.exp(-2j * np.pi * np.outer(k, k) / n)


def test_p14_reconstruction_inverts_explicit_dft():
    from oracle.recon import recon_cartesian
    from mrsim_inputs.sequence import epi_2d, fse_2d, spin_echo_2d, kspace_layout
    rng = np.random.default_rng(14)
    for seq in (spin_echo_2d(n_ro=8, n_pe=6, n_tr=6), fse_2d(n_ro=8, n_pe=8, etl=4),
                epi_2d(n_ro=8, n_lines=6)):
        L = kspace_layout(seq)
        N, M = L["n_ro"], L["n_pe"]
        img = rng.normal(size=(M, N)) + 1j * rng.normal(size=(M, N))
        K = _centred_dft(M) @ img @ _centred_dft(N).T
        i = np.arange(N)
        sig = np.stack([K[L["row"][a], (L["col0"][a] + L["dir"][a] * i) % N]
                        for a in range(len(L["row"]))])
        assert oracle.rel_l2(recon_cartesian(sig.ravel(), L), img) <= 1e-12


def _split_by_tr(seq, tr, n):
    """The n repetitions of a sequence, each as its own sequence (each then
    starts from equilibrium)."""
    from mrsim_inputs import Sequence
    t0 = np.concatenate([[0.0], np.cumsum(seq.dt * seq.repeat)])[:-1]
    out = []
    for p in range(n):
        sel = (t0 >= p * tr - 1e-12) & (t0 < (p + 1) * tr - 1e-12)
        out.append(Sequence(**{k: np.ascontiguousarray(v[sel]) for k, v in seq.arrays().items()}))
    return out


@pytest.mark.parametrize("kind", ["se", "fse", "epi"])
def test_p14_image_of_simulated_kspace_is_m0_map(kind):
    """T1 = T2 = inf keeps the refocusing exact; the spin echo's repetitions
    are simulated one by one from equilibrium (with infinite T1 the residue of
    one TR would otherwise echo in the next), the FSE uses one shot."""
    from oracle.recon import recon_cartesian
    from mrsim_inputs.sequence import epi_2d, fse_2d, spin_echo_2d, kspace_layout
    n = 16
    rng = np.random.default_rng(15)
    M0map = rng.uniform(0.2, 1.0, (n, n))
    ph = grid_phantom(M0map, nz=1, fov=0.256)
    ph.T1 = np.full(ph.K, np.inf, np.float32)
    ph.T2 = np.full(ph.K, np.inf, np.float32)
    ph.dB0 = np.zeros(ph.K, np.float32)
    seq = {"se": lambda: spin_echo_2d(n_ro=n, n_pe=n),
           "fse": lambda: fse_2d(n_ro=n, n_pe=n, etl=n, rf_dur=2e-3, rf_dt=10e-6, dwell=10e-6,
                                 esp=10e-3, tr=1.0),
           "epi": lambda: epi_2d(n_ro=n, n_lines=n, dwell=10e-6)}[kind]()
    parts = _split_by_tr(seq, seq.meta["tr"], n) if kind == "se" else [seq]
    sig = np.concatenate([oracle.simulate(ph, q, memo=True, adc_recurrence=True,
                                          want_M=False)[0] for q in parts])
    img = recon_cartesian(sig, kspace_layout(seq))
    m = ph.M0.astype(np.float64).reshape(n, n)
    c = np.vdot(m, img) / np.vdot(m, m)   # least-squares complex scale
    assert abs(c) > 0.5
    assert oracle.rel_l2(img, c * m) <= 1e-5
