"""Seeded synthetic phantoms.

A phantom is a set of K static isochromats, each with a position r(k), T1(k),
T2(k), an off-resonance dB0(k) (Hz) and an equilibrium magnetization M0(k),
as in the paper's problem statement (Sec. 2.1, Eq. 1).  The paper's "circles"
phantom (Sec. 3.2) has one big and nine small circles with constant T1, T2 and
dB0 in each; its geometry is not printed, so the ellipse phantom below is a
seeded stand-in with the same structure: per-region constants painted on an
in-plane grid and repeated over z-subvoxels (Sec. 3.5, subvoxel division).

Only +, -, *, /, sqrt and a seeded numpy Generator are used, so the arrays
are bit-identical on every platform for a given seed.
"""

from __future__ import annotations

import dataclasses
import hashlib
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Phantom:
    """Structure-of-arrays isochromat description (float32, length K).

    Units: metres, seconds, Hz.  ``b1`` (relative RF scale) and ``M_init``
    (shape [3, K], initial magnetization) are optional; when absent the RF
    scale is 1 and the initial state is thermal equilibrium (0, 0, M0).
    ``labels`` (int32, region id per isochromat) is informational.
    ``coils`` (shape [P, 2, K]: real and imaginary part of each receive coil's
    sensitivity S(k, p) at every isochromat) is optional; without it the
    signal is received by one coil with S = 1 (Eq. 6).
    """

    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    T1: np.ndarray
    T2: np.ndarray
    dB0: np.ndarray
    M0: np.ndarray
    b1: Optional[np.ndarray] = None
    M_init: Optional[np.ndarray] = None
    labels: Optional[np.ndarray] = None
    shape: tuple = ()
    coils: Optional[np.ndarray] = None

    @property
    def K(self) -> int:
        return int(self.x.shape[0])

    def arrays(self):
        return dict(x=self.x, y=self.y, z=self.z, T1=self.T1, T2=self.T2,
                    dB0=self.dB0, M0=self.M0, b1=self.b1, M_init=self.M_init)

    def subset(self, idx: np.ndarray) -> "Phantom":
        """Isochromats ``idx`` (in that order) as a new phantom."""
        pick = lambda a: None if a is None else np.ascontiguousarray(a[..., idx])
        return Phantom(x=pick(self.x), y=pick(self.y), z=pick(self.z),
                       T1=pick(self.T1), T2=pick(self.T2), dB0=pick(self.dB0),
                       M0=pick(self.M0), b1=pick(self.b1),
                       M_init=pick(self.M_init), labels=pick(self.labels),
                       shape=(len(idx),), coils=pick(self.coils))


def phantom_digest(p: Phantom) -> str:
    """SHA-256 over every array of the phantom (fixes an input exactly)."""
    h = hashlib.sha256()
    for name, a in p.arrays().items():
        h.update(name.encode())
        if a is None:
            h.update(b"none")
        else:
            h.update(np.ascontiguousarray(a).tobytes())
    if p.coils is not None:
        h.update(b"coils")
        h.update(np.ascontiguousarray(p.coils).tobytes())
    return h.hexdigest()


def grid_coords(nx: int, ny: int, nz: int, fov: float, slab: float):
    """Grid coordinates.  In-plane x_i = (i - nx/2) * fov/nx (so that the grid
    matches the FFT convention), z_k = -slab/2 + (k + 1/2) * slab/nz."""
    dx = fov / nx
    dy = fov / ny
    xs = (np.arange(nx, dtype=np.float64) - nx // 2) * dx
    ys = (np.arange(ny, dtype=np.float64) - ny // 2) * dy
    zs = -slab / 2 + (np.arange(nz, dtype=np.float64) + 0.5) * (slab / nz)
    return xs, ys, zs


def _expand(label_map: np.ndarray, xs, ys, zs, params):
    """Turn an in-plane label map [ny, nx] into per-isochromat arrays.

    Isochromat order: index = (j * nx + i) * nz + k  (y major, z minor)."""
    ny, nx = label_map.shape
    nz = len(zs)
    lab = np.repeat(label_map.reshape(-1), nz).astype(np.int32)
    X = np.repeat(np.tile(xs, ny), nz)
    Y = np.repeat(np.repeat(ys, nx), nz)
    Z = np.tile(zs, nx * ny)
    T1, T2, dB0, M0 = (np.asarray(v, dtype=np.float64)[lab] for v in params)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return dict(x=f32(X), y=f32(Y), z=f32(Z), T1=f32(T1), T2=f32(T2),
                dB0=f32(dB0), M0=f32(M0), labels=lab)


def _unit_direction(rng: np.random.Generator):
    """A uniformly distributed unit vector in the plane (no trigonometry)."""
    while True:
        u, v = rng.normal(size=2)
        n2 = u * u + v * v
        if n2 > 1e-12:
            n = np.sqrt(n2)
            return u / n, v / n


def ellipse_label_map(nx: int, ny: int, n_ellipses: int, fov: float,
                      rng: np.random.Generator) -> np.ndarray:
    """Paint ``n_ellipses`` ellipses on an [ny, nx] grid (0 = background).

    Ellipse 0 is the body: centred, semi-axes 0.45 and 0.40 of the FOV.  The
    others have centres uniform in 0.6 x the body, semi-axes U[0.05, 0.2] x FOV
    and a uniform orientation; later ellipses are painted over earlier ones."""
    xs, ys, _ = grid_coords(nx, ny, 1, fov, 1.0)
    X, Y = np.meshgrid(xs, ys)  # [ny, nx]
    lab = np.zeros((ny, nx), dtype=np.int32)
    A0, B0 = 0.45 * fov, 0.40 * fov
    ell = [(0.0, 0.0, A0, B0, 1.0, 0.0)]
    for _ in range(n_ellipses - 1):
        while True:
            cx, cy = rng.uniform(-1.0, 1.0, size=2)
            if cx * cx + cy * cy <= 1.0:
                break
        cx, cy = 0.6 * A0 * cx, 0.6 * B0 * cy
        a, b = rng.uniform(0.05, 0.2, size=2) * fov
        c, s = _unit_direction(rng)
        ell.append((cx, cy, a, b, c, s))
    for e, (cx, cy, a, b, c, s) in enumerate(ell):
        dx, dy = X - cx, Y - cy
        u = (dx * c + dy * s) / a
        v = (dy * c - dx * s) / b
        lab[u * u + v * v <= 1.0] = e + 1
    return lab


def region_params(n_regions: int, rng: np.random.Generator):
    """Per-region T1 ~ U[300,1500] ms, T2 ~ U[40,200] ms, dB0 ~ N(0, 20 Hz),
    PD ~ U[0.5, 1]; region 0 is background (PD 0, T1 1 s, T2 0.1 s, dB0 0)."""
    T1 = np.empty(n_regions + 1)
    T2 = np.empty(n_regions + 1)
    dB0 = np.empty(n_regions + 1)
    M0 = np.empty(n_regions + 1)
    T1[0], T2[0], dB0[0], M0[0] = 1.0, 0.1, 0.0, 0.0
    for r in range(1, n_regions + 1):
        T1[r] = rng.uniform(0.3, 1.5)
        T2[r] = rng.uniform(0.04, 0.2)
        dB0[r] = 20.0 * rng.normal()
        M0[r] = rng.uniform(0.5, 1.0)
    return T1, T2, dB0, M0


def ellipse_phantom(nx: int, ny: int, nz: int, n_ellipses: int, seed: int,
                    fov: float = 0.256, slab: float = 0.020) -> Phantom:
    """Seeded ellipse phantom: nx * ny in-plane pixels times nz z-subvoxels."""
    rng = np.random.default_rng(seed)
    lab = ellipse_label_map(nx, ny, n_ellipses, fov, rng)
    params = region_params(n_ellipses, rng)
    xs, ys, zs = grid_coords(nx, ny, nz, fov, slab)
    d = _expand(lab, xs, ys, zs, params)
    return Phantom(shape=(ny, nx, nz), **d)


def grid_phantom(M0_map: np.ndarray, nz: int = 1, fov: float = 0.256,
                 slab: float = 0.020, T1: float = np.inf, T2: float = np.inf,
                 dB0: float = 0.0) -> Phantom:
    """One region per pixel with an arbitrary M0 map [ny, nx] and uniform
    relaxation / off-resonance (used by the closed-form tests)."""
    ny, nx = M0_map.shape
    xs, ys, zs = grid_coords(nx, ny, nz, fov, slab)
    lab = np.zeros((ny, nx), dtype=np.int32)
    d = _expand(lab, xs, ys, zs, ([T1], [T2], [dB0], [1.0]))
    d["M0"] = np.ascontiguousarray(np.repeat(M0_map.reshape(-1), nz), dtype=np.float32)
    return Phantom(shape=(ny, nx, nz), **d)


def continuous_phantom(nx: int, ny: int, nz: int, n_ellipses: int, seed: int,
                       fov: float = 0.256, slab: float = 0.020,
                       sigma_hz: float = 20.0, b1_range=(0.8, 1.2)) -> Phantom:
    """Ellipse phantom whose dB0 ~ N(0, sigma) and RF scale b1 ~ U[b1_range]
    are drawn per isochromat, so almost every isochromat is its own group."""
    p = ellipse_phantom(nx, ny, nz, n_ellipses, seed, fov, slab)
    rng = np.random.default_rng(seed + 7919)
    p.dB0 = np.ascontiguousarray(sigma_hz * rng.normal(size=p.K), dtype=np.float32)
    p.b1 = np.ascontiguousarray(rng.uniform(b1_range[0], b1_range[1], size=p.K),
                                dtype=np.float32)
    return p


def coil_maps(p: Phantom, n_coils: int, seed: int, fov: float = 0.256) -> np.ndarray:
    """Smooth complex receive sensitivities of n_coils coils around the field of
    view (float32 [n_coils, 2, K]).  Coil c sits at radius 0.6 fov in direction
    2 atan(t_c), t_c spread evenly over [-2.5, 2.5] (+ a seeded jitter of the
    position); its magnitude falls off as
    1 / (1 + d^2 / w^2) with the distance d to the coil (w = 0.3 fov), and its
    phase is a seeded constant plus a linear ramp along x.  Cosines and sines
    come from rational parametrisations, so the maps are the same on every
    platform."""
    rng = np.random.default_rng(seed)
    K = p.K
    x = p.x.astype(np.float64)
    y = p.y.astype(np.float64)
    out = np.zeros((n_coils, 2, K), np.float32)
    w2 = (0.3 * fov) ** 2

    def unit(t):  # (cos, sin) of the angle 2 atan(t)
        d = 1.0 + t * t
        return (1.0 - t * t) / d, 2.0 * t / d

    for c in range(n_coils):
        # direction of coil c: (cos, sin) of 2 atan(t) for t spread over [-2.5, 2.5]
        # (angles within about +-136 degrees around +x)
        ca, sa = unit(2.5 * (2.0 * (c + 0.5) / n_coils - 1.0))
        jit = rng.uniform(-0.05, 0.05, 2) * fov
        cx, cy = 0.6 * fov * ca + jit[0], 0.6 * fov * sa + jit[1]
        mag = 1.0 / (1.0 + ((x - cx) ** 2 + (y - cy) ** 2) / w2)
        t0 = rng.uniform(-1.0, 1.0)
        ramp = rng.uniform(-2.0, 2.0) * x / fov
        cr, ci = unit(t0 + ramp)
        out[c, 0] = (mag * cr).astype(np.float32)
        out[c, 1] = (mag * ci).astype(np.float32)
    return out


def log_candidates(lo: float, hi: float, n: int) -> np.ndarray:
    """n values spaced evenly in log between lo and hi (the candidate set of a
    parameter-mapping search, Sec. 3.2: 100 values, 10-3000 ms for T1 and
    10-500 ms for T2).  The ratio q = (hi/lo)^(1/(n-1)) is found by Newton's
    method on q^(n-1) = hi/lo with products only, so the values are the same on
    every platform."""
    r = hi / lo
    m = n - 1
    q = 1.0 + 2.0 * (r - 1.0) / m if r < 2.0 else 2.0  # above the root
    for _ in range(200):
        p = 1.0
        for _ in range(m - 1):
            p *= q
        q_new = q - (p * q - r) / (m * p)
        if q_new == q:
            break
        q = q_new
    c = np.empty(n)
    c[0] = lo
    for j in range(1, n):
        c[j] = c[j - 1] * q
    c[-1] = hi
    return c


def _snap(v: np.ndarray, cand: np.ndarray) -> np.ndarray:
    """Nearest candidate in log distance: v goes to c_j when it lies between the
    geometric midpoints sqrt(c_{j-1} c_j) and sqrt(c_j c_{j+1})."""
    mids = np.sqrt(cand[:-1] * cand[1:])
    return cand[np.searchsorted(mids, v, side="right")]


def _smooth_field(X, Y, rng: np.random.Generator, fov: float, n_bumps: int = 3):
    """Sum of seeded rational bumps a_j / (1 + |r - c_j|^2 / w_j^2), |field| <= 1."""
    f = np.zeros_like(X)
    for _ in range(n_bumps):
        a = rng.uniform(-1.0, 1.0) / n_bumps
        cx, cy = rng.uniform(-0.4, 0.4, size=2) * fov
        w = rng.uniform(0.1, 0.3) * fov
        f += a / (1.0 + ((X - cx) ** 2 + (Y - cy) ** 2) / (w * w))
    return f


def mapped_phantom(nx: int, ny: int, nz: int, n_ellipses: int, seed: int,
                   fov: float = 0.256, slab: float = 0.020, n_cand: int = 100,
                   db0_sigma_hz: float = 0.0) -> Phantom:
    """Stand-in for a phantom made by parameter mapping (Sec. 3.2): per-pixel T1
    and T2 maps that vary smoothly inside the ellipse regions (seeded rational
    bumps, +-40 %) with 10 % pixel noise, each snapped to the nearest of
    ``n_cand`` log-spaced candidates (10-3000 ms for T1, 10-500 ms for T2), M0
    per region with a +-5 % smooth variation, and dB0 = 0 as in the paper's
    evaluations (``db0_sigma_hz`` > 0 adds a smooth dB0 field of that scale
    plus N(0, 1 %) noise, which makes almost every tuple distinct).  Such a
    phantom has up to n_cand^2 distinct (T1, T2) pairs, which the clustering
    preprocessing (Fig. 4) reduces."""
    rng = np.random.default_rng(seed)
    lab = ellipse_label_map(nx, ny, n_ellipses, fov, rng)
    T1r, T2r, _, M0r = region_params(n_ellipses, rng)
    xs, ys, zs = grid_coords(nx, ny, nz, fov, slab)
    X, Y = np.meshgrid(xs, ys)  # [ny, nx]
    g1, g2, g3 = (_smooth_field(X, Y, rng, fov) for _ in range(3))
    n1, n2 = rng.normal(size=(2, ny, nx))
    T1 = T1r[lab] * (1.0 + 0.4 * g1) * (1.0 + 0.1 * np.clip(n1, -3.0, 3.0))
    T2 = T2r[lab] * (1.0 + 0.4 * g2) * (1.0 + 0.1 * np.clip(n2, -3.0, 3.0))
    T1 = _snap(T1, log_candidates(0.010, 3.0, n_cand))
    T2 = _snap(T2, log_candidates(0.010, 0.5, n_cand))
    M0 = M0r[lab] * (1.0 + 0.05 * g3)
    dB0 = np.zeros_like(X)
    if db0_sigma_hz > 0.0:
        g4 = _smooth_field(X, Y, rng, fov)
        dB0 = db0_sigma_hz * (g4 + 0.01 * rng.normal(size=(ny, nx)))
    zero = np.zeros(n_ellipses + 1)
    d = _expand(lab, xs, ys, zs, (zero, zero, zero, zero))
    rep = lambda a: np.ascontiguousarray(np.repeat(a.reshape(-1), nz), dtype=np.float32)
    d.update(T1=rep(T1), T2=rep(T2), dB0=rep(dB0), M0=rep(M0))
    return Phantom(shape=(ny, nx, nz), **d)
