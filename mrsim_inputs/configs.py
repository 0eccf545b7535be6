"""Named synthetic workloads (phantom + sequence), with their seeds.

* ``se_32``      2-D spin echo, 32x32 in-plane x 4 z-subvoxels = 4096
                 isochromats, 3 ellipses, 2 ms sinc 90x/180y at 10 us, 32 phase
                 encodes, 32 samples at 10 us, TE 20 ms, TR 500 ms (seed 1001).
* ``fse_27m``    2-D FSE, 512x512 x 105 z-subvoxels = 27,525,120 isochromats,
                 8 ellipses, 3 ms sinc 90x/180y at 1 us, ETL 16, 256 phase
                 encodes in 16 shots, 256 samples at 4 us, ESP 8 ms, TR 3 s
                 (seed 1002).
* ``radial_27m`` radial spoiled gradient echo on the same phantom: 64 spokes
                 of 256 samples at 4 us (Gx and Gy together off the axes),
                 3 ms sinc 30 deg at 1 us, TE 5 ms, TR 10 ms.
* ``epi_27m``    single-shot EPI on the same phantom: 3 ms sinc 90x at 1 us,
                 128 lines x 128 samples at 3 us on alternating Gx trapezoids
                 with 100 us ramps at a 1 us raster, Gy blips on the ramps.
* ``*_small``    the same sequences on reduced phantoms (parity-test sizes).
* ``batch64``    64 jobs of uneven size (4k..2M isochromats, log-uniform),
                 round-robin SE / GRE (TR 10 ms, 30 deg) / FSE (ETL 8).
* ``surrogate_fse`` FSE timing with 2 ms pulses at 10 us on the 32x32x4
                 geometry, per-isochromat dB0 and RF scale (seed 1005).
* ``mapped_27m`` the FSE geometry (512x512 x 105) with T1 / T2 maps of a
                 parameter-mapping stand-in: 16 ellipse regions, smooth +-40 %
                 variation and 10 % noise, each value snapped to one of 100
                 log-spaced candidates, and a smooth dB0 field of scale 20 Hz
                 with 1 % noise (seed 1006); the input of the clustering
                 preprocessing (db0_sigma_hz=0: dB0 = 0 as in the paper's
                 evaluations).
"""

from __future__ import annotations

import math
from typing import Tuple

import numpy as np

from .phantom import Phantom, ellipse_phantom, continuous_phantom, mapped_phantom
from .sequence import Sequence, spin_echo_2d, fse_2d, epi_2d, gre_2d, radial_2d

FULL_NX, FULL_NY, FULL_NZ = 512, 512, 105


def se_32() -> Tuple[Phantom, Sequence]:
    return ellipse_phantom(32, 32, 4, 3, seed=1001), spin_echo_2d()


def fse_sequence(n_shots=None) -> Sequence:
    return fse_2d(n_shots=n_shots)


def epi_sequence() -> Sequence:
    return epi_2d()


def full_phantom() -> Phantom:
    return ellipse_phantom(FULL_NX, FULL_NY, FULL_NZ, 8, seed=1002)


def radial_sequence(n_spokes=64, oblique_deg=0.0) -> Sequence:
    """Radial spoiled gradient echo on the full-size geometry: 3 ms sinc
    30 deg pulses at 1 us, 256 samples per spoke at 4 us, TE 5 ms, TR 10 ms;
    spokes off the x and y axes read on Gx and Gy together."""
    return radial_2d(n_ro=256, n_spokes=n_spokes, rf_dur=3e-3, rf_dt=1e-6, dwell=4e-6,
                     te=5e-3, tr=10e-3, oblique_deg=oblique_deg)


def radial_27m() -> Tuple[Phantom, Sequence]:
    return full_phantom(), radial_sequence()


def fse_27m() -> Tuple[Phantom, Sequence]:
    return full_phantom(), fse_sequence()


def epi_27m() -> Tuple[Phantom, Sequence]:
    return full_phantom(), epi_sequence()


def small_phantom(nx=64, ny=64, nz=8, seed=1002) -> Phantom:
    return ellipse_phantom(nx, ny, nz, 8, seed=seed)


def fse_small(nx=64, ny=64, nz=8, n_shots=2) -> Tuple[Phantom, Sequence]:
    return small_phantom(nx, ny, nz), fse_2d(n_shots=n_shots)


def epi_small(nx=64, ny=64, nz=8) -> Tuple[Phantom, Sequence]:
    return small_phantom(nx, ny, nz), epi_2d()


def batch_sizes(n_jobs=64, kmin=4096, kmax=2_000_000, seed=1004):
    """Log-uniform job sizes (isochromat counts) for the batched workload."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(kmin), math.log(kmax), size=n_jobs)
    return [int(round(math.exp(v))) for v in u]


def batch_job(i: int, K: int):
    """Job i of the batched workload: square-ish in-plane grid x nz with about
    K isochromats, sequence round-robin SE / GRE / FSE(ETL 8)."""
    nz = int(min(105, max(4, round(K / 16384))))
    n_in = max(16, int(round(math.sqrt(K / nz))))
    n_in += n_in % 2
    ph = ellipse_phantom(n_in, n_in, nz, 8, seed=1004 + i)
    kind = ("se", "gre", "fse")[i % 3]
    if kind == "se":
        seq = spin_echo_2d(n_ro=32, n_pe=32, n_tr=8)
    elif kind == "gre":
        seq = gre_2d(n_ro=64, n_pe=64)
    else:
        seq = fse_2d(n_ro=64, n_pe=64, etl=8, rf_dur=2e-3, rf_dt=10e-6,
                     dwell=10e-6, esp=10e-3, tr=1.0, n_shots=2)
    return ph, seq


def batch_job_mixed(i: int, K: int):
    """Job i of the mixed batched workload: batch_job(i, K), then by i mod 4
    unchanged, a given initial state (M_init, seeded), two receive coils, or
    an oblique readout sequence whose with-RF and with-ADC subsequences use all
    three gradient axes (no gradient type: per-isochromat fallback)."""
    import dataclasses
    from .phantom import coil_maps
    from .sequence import SeqBuilder
    ph, seq = batch_job(i, K)
    kind = i % 4
    if kind == 1:
        rng = np.random.default_rng(2000 + i)
        Mi = np.stack([rng.uniform(-0.3, 0.3, ph.K), rng.uniform(-0.3, 0.3, ph.K),
                       rng.uniform(0.2, 1.0, ph.K)]) * ph.M0
        ph = dataclasses.replace(ph, M_init=np.ascontiguousarray(Mi, np.float32))
    elif kind == 2:
        ph = dataclasses.replace(ph, coils=coil_maps(ph, 2, seed=3000 + i))
    elif kind == 3:
        b = SeqBuilder()
        for _ in range(4):
            b.rf_sinc(90, "x", 1e-3, 10e-6, 4.0, 0.01)
            b.add(1e-3, 1, g=(-2e-3, -1e-3, -3e-3))
            for _ in range(20):  # a refocusing block with all three axes on
                b.add(10e-6, 1, b1=(2e-6, 0.5e-6), g=(1e-3, 0.5e-3, 2e-3))
            b.add(10e-6, 64, g=(4e-3, 2e-3, 1e-3), adc=True)  # oblique readout
            b.add(5e-3, 1)
        seq = b.build()
    return ph, seq


def surrogate_fse(nx=32, ny=32, nz=4) -> Tuple[Phantom, Sequence]:
    ph = continuous_phantom(nx, ny, nz, 3, seed=1005)
    seq = fse_2d(n_ro=32, n_pe=32, etl=8, rf_dur=2e-3, rf_dt=10e-6,
                 dwell=10e-6, esp=10e-3, tr=1.0, n_shots=4)
    return ph, seq


def mapped_27m(db0_sigma_hz: float = 20.0) -> Phantom:
    return mapped_phantom(FULL_NX, FULL_NY, FULL_NZ, 16, seed=1006, db0_sigma_hz=db0_sigma_hz)


def mapped_small(nx=64, ny=64, nz=4, db0_sigma_hz: float = 20.0) -> Phantom:
    return mapped_phantom(nx, ny, nz, 16, seed=1006, db0_sigma_hz=db0_sigma_hz)
