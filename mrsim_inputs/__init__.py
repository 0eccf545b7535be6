"""Seeded synthetic inputs (phantoms and pulse sequences) shared by the FP64
oracle and the GPU library.

This package holds no arithmetic of the simulation method: it only builds the
arrays that describe a phantom (isochromat positions, T1, T2, dB0, M0) and a
piecewise-constant pulse sequence (RF, gradients, ADC flags).  Every array is
built from +, -, *, / and sqrt on float64 plus a seeded numpy Generator, so
that the same seed yields bit-identical arrays on x86_64 and aarch64.
"""

from .phantom import (Phantom, coil_maps, ellipse_phantom, grid_phantom, mapped_phantom,
                      phantom_digest)
from .sequence import Sequence, SeqBuilder, sequence_digest, GAMMA_BAR_HZ_PER_T
from . import configs

__all__ = [
    "Phantom", "coil_maps", "ellipse_phantom", "grid_phantom", "mapped_phantom", "phantom_digest",
    "Sequence", "SeqBuilder", "sequence_digest", "GAMMA_BAR_HZ_PER_T",
    "configs",
]
