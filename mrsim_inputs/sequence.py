"""Seeded synthetic pulse sequences as run-length-encoded segments.

The paper treats a pulse sequence as a piecewise-constant field B(t)
(Sec. 2.1, below Eq. 2) split into with-RF, with-ADC and relaxation
subsequences (Fig. 1).  A sequence here is a list of segments; segment j holds
``repeat[j]`` sub-steps of length ``dt[j]`` seconds with constant complex RF
field ``b1re + i b1im`` (tesla), gradient (gx, gy, gz) (T/m) and an ADC flag.
When ``adc[j]`` is set, one sample is taken at the end of every sub-step.

The workloads follow Table 2 (Hamming-windowed sinc RF, SE / FSE / EPI with a
256 mm FOV and a 10 mm slice) resized to the shapes used by the benchmarks.
The sinc and window are evaluated with a fixed polynomial of this module
(sin(pi*y) on |y| <= 1/2) instead of libm, so sequences are bit-identical on
every platform.
"""

from __future__ import annotations

import dataclasses
import hashlib
import math
from typing import List, Optional

import numpy as np

# Gyromagnetic ratio of 1H divided by 2*pi (Hz/T).  Used here only to size
# RF amplitudes and gradient areas of the synthetic sequences.
GAMMA_BAR_HZ_PER_T = 42.577478518e6


@dataclasses.dataclass
class Sequence:
    dt: np.ndarray       # float64 [n_seg], seconds per sub-step
    repeat: np.ndarray   # int32   [n_seg], sub-steps in the segment
    b1re: np.ndarray     # float32 [n_seg], tesla
    b1im: np.ndarray     # float32 [n_seg], tesla
    gx: np.ndarray       # float32 [n_seg], T/m
    gy: np.ndarray
    gz: np.ndarray
    adc: np.ndarray      # uint8   [n_seg], 1 = sample at the end of each sub-step
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_seg(self) -> int:
        return int(self.dt.shape[0])

    @property
    def n_samples(self) -> int:
        return int(np.sum(self.repeat.astype(np.int64) * (self.adc != 0)))

    @property
    def duration(self) -> float:
        return math.fsum((self.dt * self.repeat).tolist())

    def arrays(self):
        return dict(dt=self.dt, repeat=self.repeat, b1re=self.b1re, b1im=self.b1im,
                    gx=self.gx, gy=self.gy, gz=self.gz, adc=self.adc)


def sequence_digest(s: Sequence) -> str:
    h = hashlib.sha256()
    for name, a in s.arrays().items():
        h.update(name.encode())
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _sin_pi(x: np.ndarray) -> np.ndarray:
    """sin(pi*x) from its Maclaurin series after reduction to |y| <= 1/2."""
    x = np.asarray(x, dtype=np.float64)
    n = np.rint(x)
    y = x - n
    t = np.pi * y
    t2 = t * t
    acc = np.zeros_like(t)
    # sum_{k=0}^{12} (-1)^k t^(2k+1) / (2k+1)!, Horner in t^2
    for k in range(12, -1, -1):
        c = (-1.0) ** k / math.factorial(2 * k + 1)
        acc = acc * t2 + c
    s = acc * t
    odd = (np.abs(n) % 2) == 1
    return np.where(odd, -s, s)


def _cos_pi(x: np.ndarray) -> np.ndarray:
    return _sin_pi(np.asarray(x, dtype=np.float64) + 0.5)


def hamming_sinc(n: int, tbw: float) -> np.ndarray:
    """Hamming-windowed sinc sampled at sub-step midpoints.

    t_j = -T/2 + (j + 1/2) T/n; shape w(t) = (0.54 + 0.46 cos(2 pi t/T)) *
    sinc(tbw t / T), sinc(u) = sin(pi u)/(pi u)."""
    j = np.arange(n, dtype=np.float64)
    tau = (j + 0.5) / n - 0.5          # t / T
    win = 0.54 + 0.46 * _cos_pi(2.0 * tau)
    u = tbw * tau
    with np.errstate(invalid="ignore", divide="ignore"):
        sinc = np.where(u == 0.0, 1.0, _sin_pi(u) / (np.pi * u))
    return win * sinc


_PHASES = {"x": (1.0, 0.0), "y": (0.0, 1.0), "-x": (-1.0, 0.0), "-y": (0.0, -1.0)}


class SeqBuilder:
    """Appends segments in time order and tracks the current time."""

    def __init__(self):
        self._seg: List[tuple] = []
        self.t = 0.0
        self.n_rf = 0
        self.n_adc = 0

    def add(self, dt, repeat=1, b1=(0.0, 0.0), g=(0.0, 0.0, 0.0), adc=False):
        if not (dt > 0) or repeat < 1:
            raise ValueError("segment needs dt > 0 and repeat >= 1")
        self._seg.append((float(dt), int(repeat), float(b1[0]), float(b1[1]),
                          float(g[0]), float(g[1]), float(g[2]), 1 if adc else 0))
        self.t += dt * repeat

    def delay_until(self, t_target, g=(0.0, 0.0, 0.0)):
        # sub-step times accumulate rounding; gaps shorter than 1 ns are dropped
        d = t_target - self.t
        if d < -1e-9:
            raise ValueError(f"timing violated: at {self.t}, asked for {t_target}")
        if d > 1e-9:
            self.add(d, 1, g=g)
            self.t = t_target

    def grad(self, dur, g):
        self.add(dur, 1, g=g)

    def ramp(self, g0, g1, dur, raster, extra=(0.0, 0.0, 0.0)):
        """Linear gradient ramp g0 -> g1, one segment per raster step (value at
        the step midpoint), plus a constant ``extra`` gradient (e.g. a blip)."""
        n = int(round(dur / raster))
        for j in range(n):
            f = (j + 0.5) / n
            g = tuple(a + (b - a) * f + e for a, b, e in zip(g0, g1, extra))
            self.add(raster, 1, g=g)

    def rf_sinc(self, flip_deg, phase, dur, dt, tbw=4.0, slice_thk=0.010,
                b1_peak_scale=1.0, direction=None):
        """Slice-selective Hamming sinc along z (or along the unit vector
        ``direction`` for an oblique slice).  Amplitude so that
        gamma * sum_j |B1_j| dt equals the flip angle.  Returns the
        slice-select gradient magnitude (T/m)."""
        n = int(round(dur / dt))
        w = hamming_sinc(n, tbw)
        alpha = flip_deg * np.pi / 180.0
        amp = alpha / (2.0 * np.pi * GAMMA_BAR_HZ_PER_T * dt * math.fsum(w.tolist()))
        amp *= b1_peak_scale
        gss = (tbw / dur) / (GAMMA_BAR_HZ_PER_T * slice_thk) if slice_thk else 0.0
        cr, ci = _PHASES[phase]
        g = (0.0, 0.0, gss) if direction is None else tuple(d * gss for d in direction)
        for j in range(n):
            a = amp * w[j]
            self.add(dt, 1, b1=(a * cr, a * ci), g=g)
        self.n_rf += 1
        return gss

    def rf_hard(self, flip_deg, phase, dur, dt):
        """Rectangular (hard) pulse without gradients."""
        n = int(round(dur / dt))
        amp = (flip_deg * np.pi / 180.0) / (2.0 * np.pi * GAMMA_BAR_HZ_PER_T * dt * n)
        cr, ci = _PHASES[phase]
        self.add(dt, n, b1=(amp * cr, amp * ci))
        self.n_rf += 1

    def readout(self, n, dwell, g):
        self.add(dwell, n, g=g, adc=True)
        self.n_adc += 1

    def build(self, **meta) -> Sequence:
        a = np.array(self._seg, dtype=np.float64).reshape(-1, 8)
        f32 = lambda c: np.ascontiguousarray(c, dtype=np.float32)
        return Sequence(dt=np.ascontiguousarray(a[:, 0]),
                        repeat=np.ascontiguousarray(a[:, 1], dtype=np.int32),
                        b1re=f32(a[:, 2]), b1im=f32(a[:, 3]),
                        gx=f32(a[:, 4]), gy=f32(a[:, 5]), gz=f32(a[:, 6]),
                        adc=np.ascontiguousarray(a[:, 7], dtype=np.uint8),
                        meta=dict(meta, n_rf=self.n_rf, n_adc=self.n_adc))


def _dk(fov):
    return 1.0 / fov


def spin_echo_2d(n_ro=32, n_pe=32, fov=0.256, thk=0.010, rf_dur=2e-3,
                 rf_dt=10e-6, dwell=10e-6, te=20e-3, tr=500e-3, tbw=4.0,
                 n_tr: Optional[int] = None) -> Sequence:
    """2-D spin echo: sinc 90x - TE/2 - sinc 180y - readout on Gx, one phase
    encode (Gy) per TR.  Prephasers share one 1 ms lobe after the 90."""
    b = SeqBuilder()
    gb = GAMMA_BAR_HZ_PER_T
    g_ro = _dk(fov) / (gb * dwell)
    d1 = 1e-3
    n_tr = n_pe if n_tr is None else n_tr
    for p in range(n_tr):
        t0 = p * tr
        b.delay_until(t0)
        gss = b.rf_sinc(90, "x", rf_dur, rf_dt, tbw, thk)
        ky = (p % n_pe - n_pe // 2) * _dk(fov)
        b.grad(d1, ((n_ro // 2) * _dk(fov) / gb / d1, ky / gb / d1,
                    -gss * (rf_dur / 2) / d1))
        b.delay_until(t0 + rf_dur / 2 + te / 2 - rf_dur / 2)
        b.rf_sinc(180, "y", rf_dur, rf_dt, tbw, thk)
        b.delay_until(t0 + rf_dur / 2 + te - (n_ro // 2) * dwell)
        b.readout(n_ro, dwell, (g_ro, 0.0, 0.0))
    b.delay_until(n_tr * tr)
    return b.build(kind="se", n_ro=n_ro, n_pe=n_pe, n_tr=n_tr, tr=tr, te=te)


def fse_2d(n_ro=256, n_pe=256, etl=16, fov=0.256, thk=0.010, rf_dur=3e-3,
           rf_dt=1e-6, dwell=4e-6, esp=8e-3, tr=3.0, tbw=4.0, d_pe=1e-3,
           n_shots: Optional[int] = None) -> Sequence:
    """2-D CPMG fast spin echo, sequential phase-encode ordering
    (line = echo * n_shots + shot)."""
    b = SeqBuilder()
    gb = GAMMA_BAR_HZ_PER_T
    g_ro = _dk(fov) / (gb * dwell)
    shots = n_pe // etl if n_shots is None else n_shots
    d1 = 1e-3
    for s in range(shots):
        t0 = s * tr
        b.delay_until(t0)
        gss = b.rf_sinc(90, "x", rf_dur, rf_dt, tbw, thk)
        b.grad(d1, ((n_ro // 2) * _dk(fov) / gb / d1, 0.0, -gss * (rf_dur / 2) / d1))
        for e in range(1, etl + 1):
            b.delay_until(t0 + rf_dur / 2 + (e - 0.5) * esp - rf_dur / 2)
            b.rf_sinc(180, "y", rf_dur, rf_dt, tbw, thk)
            line = (e - 1) * shots + s
            ky = (line % n_pe - n_pe // 2) * _dk(fov)
            b.grad(d_pe, (0.0, ky / gb / d_pe, 0.0))
            b.delay_until(t0 + rf_dur / 2 + e * esp - (n_ro // 2) * dwell)
            b.readout(n_ro, dwell, (g_ro, 0.0, 0.0))
            b.grad(d_pe, (0.0, -ky / gb / d_pe, 0.0))
        b.delay_until(t0 + tr)
    return b.build(kind="fse", n_ro=n_ro, n_pe=n_pe, etl=etl, shots=shots, tr=tr)


def epi_2d(n_ro=128, n_lines=128, fov=0.256, thk=0.010, rf_dur=3e-3, rf_dt=1e-6,
           dwell=3e-6, ramp=100e-6, raster=1e-6, tbw=4.0) -> Sequence:
    """Single-shot 2-D gradient-echo EPI: sinc 90x, prephasers, then n_lines
    flat-top readouts on alternating-sign Gx trapezoids; Gy blips ride on the
    ramp-down of every line but the last."""
    b = SeqBuilder()
    gb = GAMMA_BAR_HZ_PER_T
    g_ro = _dk(fov) / (gb * dwell)
    d1 = 1e-3
    gss = b.rf_sinc(90, "x", rf_dur, rf_dt, tbw, thk)
    kx_pre = -(n_ro // 2) * _dk(fov) - gb * g_ro * ramp / 2
    ky_pre = -(n_lines // 2) * _dk(fov)
    b.grad(d1, (kx_pre / gb / d1, ky_pre / gb / d1, -gss * (rf_dur / 2) / d1))
    blip = _dk(fov) / gb / ramp
    for l in range(n_lines):
        d = 1.0 if l % 2 == 0 else -1.0
        b.ramp((0.0, 0.0, 0.0), (d * g_ro, 0.0, 0.0), ramp, raster)
        b.readout(n_ro, dwell, (d * g_ro, 0.0, 0.0))
        extra = (0.0, blip, 0.0) if l < n_lines - 1 else (0.0, 0.0, 0.0)
        b.ramp((d * g_ro, 0.0, 0.0), (0.0, 0.0, 0.0), ramp, raster, extra)
    return b.build(kind="epi", n_ro=n_ro, n_lines=n_lines)


def gre_2d(n_ro=64, n_pe=64, fov=0.256, thk=0.010, flip=30.0, rf_dur=2e-3,
           rf_dt=10e-6, dwell=10e-6, te=5e-3, tr=10e-3, tbw=4.0,
           spoil_area_cycles=4.0) -> Sequence:
    """2-D spoiled gradient echo: sinc alpha-x, prephasers, Gx readout centred
    at TE, then a Gz spoiler giving ``spoil_area_cycles`` cycles over the slice."""
    b = SeqBuilder()
    gb = GAMMA_BAR_HZ_PER_T
    g_ro = _dk(fov) / (gb * dwell)
    d1 = 1e-3
    for p in range(n_pe):
        t0 = p * tr
        b.delay_until(t0)
        gss = b.rf_sinc(flip, "x", rf_dur, rf_dt, tbw, thk)
        ky = (p - n_pe // 2) * _dk(fov)
        b.grad(d1, (-(n_ro // 2) * _dk(fov) / gb / d1, ky / gb / d1,
                    -gss * (rf_dur / 2) / d1))
        b.delay_until(t0 + rf_dur / 2 + te - (n_ro // 2) * dwell)
        b.readout(n_ro, dwell, (g_ro, 0.0, 0.0))
        d_sp = 1e-3
        b.grad(d_sp, (0.0, -ky / gb / d_sp, spoil_area_cycles / thk / gb / d_sp))
    b.delay_until(n_pe * tr)
    return b.build(kind="gre", n_ro=n_ro, n_pe=n_pe, tr=tr, flip=flip)


def radial_2d(n_ro=32, n_spokes=16, fov=0.256, thk=0.010, flip=30.0, rf_dur=2e-3,
              rf_dt=10e-6, dwell=10e-6, te=5e-3, tr=10e-3, tbw=4.0, oblique_deg=0.0,
              spoil_area_cycles=4.0) -> Sequence:
    """2-D radial spoiled gradient echo: TR p reads one spoke through the
    k-space centre at angle theta_p = pi p / n_spokes, so the readout has
    Gx = g cos(theta_p) and Gy = g sin(theta_p) both nonzero (a with-ADC
    subsequence on two gradient axes) except on spokes along an axis.
    ``oblique_deg`` tilts the slice normal from z toward x, which puts the
    slice-select and its rephaser on two axes (Gx and Gz) as well.  Cosines and
    sines come from this module's polynomial, so the sequence is the same on
    every platform."""
    b = SeqBuilder()
    gb = GAMMA_BAR_HZ_PER_T
    g_ro = _dk(fov) / (gb * dwell)
    d1 = 1e-3
    ob = float(oblique_deg) / 180.0
    normal = None if oblique_deg == 0.0 else (float(_sin_pi(ob)), 0.0, float(_cos_pi(ob)))
    nrm = (0.0, 0.0, 1.0) if normal is None else normal
    for p in range(n_spokes):
        t0 = p * tr
        b.delay_until(t0)
        gss = b.rf_sinc(flip, "x", rf_dur, rf_dt, tbw, thk, direction=normal)
        th = p / n_spokes
        c, sn = float(_cos_pi(th)), float(_sin_pi(th))
        k0 = -(n_ro // 2) * _dk(fov) / gb / d1
        reph = -gss * (rf_dur / 2) / d1
        b.grad(d1, (k0 * c + reph * nrm[0], k0 * sn + reph * nrm[1], reph * nrm[2]))
        b.delay_until(t0 + rf_dur / 2 + te - (n_ro // 2) * dwell)
        b.readout(n_ro, dwell, (g_ro * c, g_ro * sn, 0.0))
        d_sp = 1e-3
        b.grad(d_sp, (0.0, 0.0, spoil_area_cycles / thk / gb / d_sp))
    b.delay_until(n_spokes * tr)
    return b.build(kind="radial", n_ro=n_ro, n_spokes=n_spokes, tr=tr, flip=flip,
                   oblique_deg=oblique_deg)


def kspace_layout(seq: Sequence) -> dict:
    """Where each acquisition line of a generated Cartesian sequence (SE, FSE,
    EPI) sits in k-space, as the generators build them: line a (in ADC-window
    order) fills grid row ``row[a]`` (ky index, 0..n_pe-1, centre n_pe/2), and
    its sample i the column ``(col0[a] + dir[a] * i) mod n_ro`` (kx index,
    centre n_ro/2).  A sample is taken at the end of its dwell, so forward
    readouts start one column right of -kx_max (col0 = 1), reversed EPI lines
    at n_ro - 1.  The spin echo encodes ky before its 180-degree pulse, which
    negates it: row = (n_pe - p) mod n_pe for TR p."""
    m = seq.meta
    kind = m.get("kind")
    if kind == "se":
        n_ro, n_pe, n_tr = m["n_ro"], m["n_pe"], m["n_tr"]
        rows = [(n_pe - (p % n_pe)) % n_pe for p in range(n_tr)]
        col0 = [1] * n_tr
        dirs = [1] * n_tr
    elif kind == "fse":
        n_ro, n_pe, etl, shots = m["n_ro"], m["n_pe"], m["etl"], m["shots"]
        rows, col0, dirs = [], [], []
        for s in range(shots):
            for e in range(1, etl + 1):
                rows.append(((e - 1) * shots + s) % n_pe)
                col0.append(1)
                dirs.append(1)
    elif kind == "epi":
        n_ro, n_pe = m["n_ro"], m["n_lines"]
        rows = list(range(n_pe))
        col0 = [1 if l % 2 == 0 else n_ro - 1 for l in range(n_pe)]
        dirs = [1 if l % 2 == 0 else -1 for l in range(n_pe)]
    else:
        raise ValueError(f"no Cartesian layout for sequence kind {kind!r}")
    return dict(n_ro=int(n_ro), n_pe=int(n_pe), row=np.array(rows, np.int32),
                col0=np.array(col0, np.int32), dir=np.array(dirs, np.int8))
