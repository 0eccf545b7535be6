"""FP64 CPU oracle (ctypes binding of ``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the benchmark's CPU-baseline leg.  The CUDA library and its Python binding
never import it, and it imports nothing from them.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RF, ADC, RELAX = 0, 1, 2
G_NONE, G_X, G_Y, G_Z, G_GENERAL = 0, 1, 2, 3, 4
# two-axis gradient types (grouped on both positions; made only on request)
G_XY, G_XZ, G_YZ = 5, 6, 7


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc (IEEE semantics: no fast-math, no FMA
    contraction) into ``liboracle.so`` next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            lib.or_classify.argtypes = [P] * 8 + [I64, I64] + [P] * 7 + [I]
            lib.or_group.argtypes = [I64] + [P] * 7 + [I, P, P]
            lib.or_simulate.argtypes = [I64] + [P] * 9 + [I64] + [P] * 8 + [I, I, I, I, P, P, P]
            lib.or_simulate_grouped.argtypes = [I64] + [P] * 9 + [I64] + [P] * 8 + [I, P, P]
            lib.or_transition.argtypes = [ctypes.c_double] * 7 + [P] * 7 + [I64, I64, P]
            for f in (lib.or_classify, lib.or_group, lib.or_simulate, lib.or_simulate_grouped,
                      lib.or_transition):
                f.restype = I
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _seq_args(seq):
    return [_p(np.ascontiguousarray(seq.dt, np.float64)), _p(np.ascontiguousarray(seq.repeat, np.int32)),
            _p(_f32(seq.b1re)), _p(_f32(seq.b1im)), _p(_f32(seq.gx)), _p(_f32(seq.gy)),
            _p(_f32(seq.gz)), _p(np.ascontiguousarray(seq.adc, np.uint8))]


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


def classify(seq, two_axis: bool = False):
    """Subsequence split + classification.  Returns a dict of numpy arrays:
    type, gtype, seg_begin, seg_end, n_samples, content_id.  With two_axis, a
    subsequence whose gradients use exactly two axes gets G_XY / G_XZ / G_YZ
    instead of G_GENERAL."""
    lib = _load()
    keep = [np.ascontiguousarray(seq.dt, np.float64), np.ascontiguousarray(seq.repeat, np.int32),
            _f32(seq.b1re), _f32(seq.b1im), _f32(seq.gx), _f32(seq.gy), _f32(seq.gz),
            np.ascontiguousarray(seq.adc, np.uint8)]
    n = ctypes.c_int64(0)
    cap = seq.n_seg
    out = dict(type=np.zeros(cap, np.uint8), gtype=np.zeros(cap, np.uint8),
               seg_begin=np.zeros(cap, np.int64), seg_end=np.zeros(cap, np.int64),
               n_samples=np.zeros(cap, np.int64), content_id=np.zeros(cap, np.int32))
    rc = lib.or_classify(*[_p(a) for a in keep], seq.n_seg, cap, ctypes.byref(n),
                         *[_p(out[k]) for k in ("type", "gtype", "seg_begin", "seg_end",
                                                "n_samples", "content_id")],
                         int(two_axis))
    _check(rc, "or_classify")
    return {k: v[: n.value].copy() for k, v in out.items()}


def group(ph, gtype: int):
    """Group ids (first-occurrence numbering) for one gradient type.
    Returns (gid int32 [K], n_groups)."""
    lib = _load()
    arrs = [_f32(ph.x), _f32(ph.y), _f32(ph.z), _f32(ph.T1), _f32(ph.T2), _f32(ph.dB0), _f32(ph.b1)]
    gid = np.empty(ph.K, np.int32)
    ng = ctypes.c_int64(0)
    rc = lib.or_group(ph.K, *[_p(a) for a in arrs], gtype, _p(gid), ctypes.byref(ng))
    _check(rc, "or_group")
    return gid, ng.value


def _ph_args(ph):
    arrs = [_f32(ph.x), _f32(ph.y), _f32(ph.z), _f32(ph.T1), _f32(ph.T2), _f32(ph.dB0),
            _f32(ph.M0), _f32(ph.b1),
            None if ph.M_init is None else np.ascontiguousarray(ph.M_init, np.float32).reshape(3, -1)]
    return arrs


def simulate(ph, seq, memo: bool = False, adc_recurrence: bool = False,
             n_threads: int = 0, want_M: bool = True):
    """Ungrouped FP64 simulation.  Returns (signal, M_final float64 [3, K] or
    None); the signal is complex128 [n_samples], or [P, n_samples] when the
    phantom carries P receive-coil sensitivities (``ph.coils``)."""
    lib = _load()
    arrs = _ph_args(ph)
    sargs = [np.ascontiguousarray(seq.dt, np.float64), np.ascontiguousarray(seq.repeat, np.int32),
             _f32(seq.b1re), _f32(seq.b1im), _f32(seq.gx), _f32(seq.gy), _f32(seq.gz),
             np.ascontiguousarray(seq.adc, np.uint8)]
    ns = seq.n_samples
    coils = getattr(ph, "coils", None)
    P = 1 if coils is None else int(coils.shape[0])
    sens = None if coils is None else np.ascontiguousarray(coils, np.float32).reshape(P, 2, ph.K)
    sig = np.zeros(2 * ns * P + 1, np.float64)
    M = np.zeros((3, ph.K), np.float64) if want_M else None
    rc = lib.or_simulate(ph.K, *[_p(a) for a in arrs], seq.n_seg, *[_p(a) for a in sargs],
                         int(memo), int(adc_recurrence), int(n_threads), P, _p(sens), _p(sig),
                         _p(M))
    _check(rc, "or_simulate")
    out = sig[: 2 * ns * P].view(np.complex128).copy()
    return (out if coils is None else out.reshape(P, ns)), M


def simulate_grouped(ph, seq, want_M: bool = True, two_axis: bool = False):
    """Grouped FP64 simulation (Eqs. 8-10 and per-group Eq. 7).  With
    two_axis, subsequences on exactly two gradient axes are grouped on both
    positions instead of being simulated per isochromat."""
    lib = _load()
    arrs = _ph_args(ph)
    sargs = [np.ascontiguousarray(seq.dt, np.float64), np.ascontiguousarray(seq.repeat, np.int32),
             _f32(seq.b1re), _f32(seq.b1im), _f32(seq.gx), _f32(seq.gy), _f32(seq.gz),
             np.ascontiguousarray(seq.adc, np.uint8)]
    ns = seq.n_samples
    sig = np.zeros(2 * ns + 1, np.float64)
    M = np.zeros((3, ph.K), np.float64) if want_M else None
    rc = lib.or_simulate_grouped(ph.K, *[_p(a) for a in arrs], seq.n_seg,
                                 *[_p(a) for a in sargs], int(two_axis), _p(sig), _p(M))
    _check(rc, "or_simulate_grouped")
    return sig[: 2 * ns].view(np.complex128).copy(), M


def transition(seq, seg_begin: int, seg_end: int, x=0.0, y=0.0, z=0.0, T1=np.inf,
               T2=np.inf, dB0=0.0, b1=1.0):
    """Combined transition (Eq. 7) of segments [seg_begin, seg_end) for one
    isochromat: returns (A [3, 3], b [3]) with M <- A M + b M0."""
    lib = _load()
    sargs = [np.ascontiguousarray(seq.dt, np.float64), np.ascontiguousarray(seq.repeat, np.int32),
             _f32(seq.b1re), _f32(seq.b1im), _f32(seq.gx), _f32(seq.gy), _f32(seq.gz)]
    T = np.zeros(12, np.float64)
    rc = lib.or_transition(float(x), float(y), float(z), float(T1), float(T2), float(dB0),
                           float(b1), *[_p(a) for a in sargs], int(seg_begin), int(seg_end), _p(T))
    _check(rc, "or_transition")
    T = T.reshape(3, 4)
    return T[:, :3].copy(), T[:, 3].copy()


def rel_l2(a, ref) -> float:
    """||a - ref||_2 / ||ref||_2 over all complex samples."""
    a = np.asarray(a)
    ref = np.asarray(ref)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))
