"""Python binding of libmrsim (C ABI in include/mrsim.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  The functions carry the C names (mrsim_create, mrsim_phantom,
mrsim_sequence, mrsim_group, mrsim_run, ...); the small ``Context`` class
below wraps them with numpy / torch arrays for tests and the benchmark.

The library must be built (``paper_2508_03960_gb300.build``); importing this
module on a machine without it raises instead of falling back to anything.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence as Seq

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmrsim.so")

OK, EINVAL, EUNSUPPORTED, ENOMEM, ECUDA, ETIMEOUT, ESTATE = range(7)
SUB_RF, SUB_ADC, SUB_RELAX = 0, 1, 2
G_NONE, G_X, G_Y, G_Z, G_GENERAL = 0, 1, 2, 3, 4
PLAIN, PLAIN_CACHE, GROUPED, SURROGATE = 0, 1, 2, 3
FP32, FP64 = 0, 1
PTR_DEVICE, OUT_DEVICE, PHANTOM_ASYNC = 1, 2, 4
TUNE_FUSED_NI, TUNE_PLAIN_RF_NI, TUNE_ADC_CTAS_PER_SM, TUNE_PRECOMP_LANES = 0, 1, 2, 3
TUNE_PRECOMP_STEPS = 4
TUNE_CELL_NI = 5
TUNE_TWO_AXIS = 6
TUNE_CELL_ROWS = 7

# every entry point declared in include/mrsim.h
EXPORTS = ["mrsim_create", "mrsim_destroy", "mrsim_last_error", "mrsim_phantom",
           "mrsim_phantom_read", "mrsim_coils", "mrsim_classify",
           "mrsim_sequence", "mrsim_seq_info", "mrsim_group", "mrsim_group_info", "mrsim_run",
           "mrsim_run_batch", "mrsim_recon_cartesian", "mrsim_cluster", "mrsim_profile_enable",
           "mrsim_profile_reset",
           "mrsim_profile_get", "mrsim_launch_count", "mrsim_adc_grouped_noalloc",
           "mrsim_set_tuning", "mrsim_get_tuning", "mrsim_autotune",
           "mrsim_set_reproducible", "mrsim_get_reproducible",
           "mrsim_surrogate_train", "mrsim_surrogate_stats", "mrsim_surrogate_use",
           "mrsim_surrogate_check", "mrsim_surrogate_infer",
           "mrsim_surrogate_eval", "mrsim_free_surrogate",
           "mrsim_free_phantom", "mrsim_free_seq", "mrsim_free_groups"]
NOALLOC_MAX_GROUPS = 65536
MAX_COILS = 64
MAX_CLUSTERS = 4096
MAX_ECHOES = 16
# the paper's T2-weighted scan (Table 1: FSE, TR 4500 ms, TE 20/60/100/140 ms),
# the default model of the M0 refit after clustering
T2W_TE = (0.020, 0.060, 0.100, 0.140)
T2W_TR = 4.5


class MrsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mrsim error {code}: {msg}")
        self.code = code


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libmrsim is not built ({path} missing); run "
                          "python -m paper_2508_03960_gb300.build")
    lib = ctypes.CDLL(path)
    P, I, I64, U = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "mrsim_create": (I, [PP, I, P]),
        "mrsim_destroy": (None, [P]),
        "mrsim_last_error": (ctypes.c_char_p, [P]),
        "mrsim_phantom": (I, [P, I64] + [P] * 9 + [U, PP]),
        "mrsim_sequence": (I, [P, I64] + [P] * 8 + [PP]),
        "mrsim_coils": (I, [P, P, I, P, U]),
        "mrsim_phantom_read": (I, [P] * 9),
        "mrsim_classify": (I, [I64] + [P] * 8 + [U, I64] + [P] * 7),
        "mrsim_seq_info": (I, [P] * 7),
        "mrsim_group": (I, [P, P, P, PP]),
        "mrsim_group_info": (I, [P, I, P, P]),
        "mrsim_run": (I, [P, P, P, P, I, I, P, P, U]),
        "mrsim_run_batch": (I, [P, I, P, P, P, P]),
        "mrsim_recon_cartesian": (I, [P, I, I, I, P, P, P, P, U, P]),
        "mrsim_cluster": (I, [P, P, I, P, I, I, P, ctypes.c_double, P, P, P, PP]),
        "mrsim_profile_enable": (I, [P, I]),
        "mrsim_profile_reset": (I, [P]),
        "mrsim_profile_get": (I, [P, I, P, I, P, P]),
        "mrsim_launch_count": (I64, [P]),
        "mrsim_adc_grouped_noalloc": (I, [I64, P, P, P, ctypes.c_int32, P, P, P, I64, P, P, P, P]),
        "mrsim_set_tuning": (I, [P, I, I]),
        "mrsim_get_tuning": (I, [P, I, P]),
        "mrsim_set_reproducible": (I, [P, I]),
        "mrsim_get_reproducible": (I, [P, P]),
        "mrsim_autotune": (I, [P, P, P, P, I, I, I]),
        "mrsim_surrogate_train": (I, [P, P, P, P, I64, I, I, ctypes.c_double, ctypes.c_uint64,
                                      ctypes.c_double, PP]),
        "mrsim_surrogate_stats": (I, [P, P, P]),
        "mrsim_surrogate_use": (I, [P, P]),
        "mrsim_surrogate_check": (I, [P, P, P, P, P, P]),
        "mrsim_surrogate_infer": (I, [P, P, I64, P, P]),
        "mrsim_surrogate_eval": (I, [P, P, I64, P, P, P, P, P]),
        "mrsim_free_surrogate": (None, [P]),
        "mrsim_free_phantom": (None, [P]),
        "mrsim_free_seq": (None, [P]),
        "mrsim_free_groups": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _ptr(a) -> Optional[int]:
    """Address of a numpy array or torch tensor (None stays NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


# ------------------------------------------------------------------ C names --
def mrsim_create(device: int = 0, stream: Optional[int] = None) -> int:
    h = ctypes.c_void_p()
    rc = lib().mrsim_create(ctypes.byref(h), device, stream)
    if rc:
        raise MrsimError(rc, "mrsim_create failed")
    return h.value


def mrsim_destroy(ctx: int) -> None:
    lib().mrsim_destroy(ctx)


def mrsim_last_error(ctx: int) -> str:
    return (lib().mrsim_last_error(ctx) or b"").decode()


def _check(ctx, rc, what):
    if rc:
        raise MrsimError(rc, f"{what}: {mrsim_last_error(ctx)}")


def mrsim_phantom(ctx, K, x, y, z, T1, T2, dB0, M0, b1=None, M_init=None, flags=0) -> int:
    h = ctypes.c_void_p()
    rc = lib().mrsim_phantom(ctx, int(K), *[_ptr(a) for a in (x, y, z, T1, T2, dB0, M0, b1,
                                                              M_init)],
                             flags, ctypes.byref(h))
    _check(ctx, rc, "mrsim_phantom")
    return h.value


def mrsim_phantom_read(ctx, ph, K, fields=("T1", "T2", "dB0", "M0")):
    """Dict of the requested phantom arrays (float32 [K]) copied to the host."""
    names = ("x", "y", "z", "T1", "T2", "dB0", "M0")
    out = {n: np.empty(K, np.float32) for n in fields}
    _check(ctx, lib().mrsim_phantom_read(ctx, ph, *[_ptr(out.get(n)) for n in names]),
           "mrsim_phantom_read")
    return out


def mrsim_sequence(ctx, n_seg, dt, repeat, b1re, b1im, gx, gy, gz, adc) -> int:
    h = ctypes.c_void_p()
    rc = lib().mrsim_sequence(ctx, int(n_seg), *[_ptr(a) for a in (dt, repeat, b1re, b1im, gx,
                                                                    gy, gz, adc)],
                              ctypes.byref(h))
    _check(ctx, rc, "mrsim_sequence")
    return h.value


CLASSIFY_TWO_AXIS = 1
G_XY, G_XZ, G_YZ = 5, 6, 7


def mrsim_classify(seq, flags=0):
    """Subsequence table of a sequence (numpy arrays; no context, no device):
    dict of type, gtype, seg_begin, seg_end, n_samples, content_id.  flags =
    CLASSIFY_TWO_AXIS types subsequences on exactly two axes G_XY / G_XZ / G_YZ."""
    keep = [np.ascontiguousarray(seq.dt, np.float64), np.ascontiguousarray(seq.repeat, np.int32),
            _f32(seq.b1re), _f32(seq.b1im), _f32(seq.gx), _f32(seq.gy), _f32(seq.gz),
            np.ascontiguousarray(seq.adc, np.uint8)]
    cap = int(seq.n_seg)
    out = dict(type=np.zeros(cap, np.uint8), gtype=np.zeros(cap, np.uint8),
               seg_begin=np.zeros(cap, np.int64), seg_end=np.zeros(cap, np.int64),
               n_samples=np.zeros(cap, np.int64), content_id=np.zeros(cap, np.int32))
    n = ctypes.c_int64(0)
    rc = lib().mrsim_classify(int(seq.n_seg), *[_ptr(a) for a in keep], flags, cap,
                              ctypes.byref(n),
                              *[_ptr(out[k]) for k in ("type", "gtype", "seg_begin", "seg_end",
                                                       "n_samples", "content_id")])
    if rc:
        raise MrsimError(rc, "mrsim_classify")
    return {k: v[: n.value].copy() for k, v in out.items()}


def mrsim_seq_info(seq):
    n = ctypes.c_int64()
    ns = ctypes.c_int64()
    rc = lib().mrsim_seq_info(seq, ctypes.byref(n), None, None, None, None, ctypes.byref(ns))
    if rc:
        raise MrsimError(rc, "mrsim_seq_info")
    N = n.value
    out = dict(type=np.zeros(N, np.uint8), gtype=np.zeros(N, np.uint8),
               seg_begin=np.zeros(N, np.int64), seg_end=np.zeros(N, np.int64))
    rc = lib().mrsim_seq_info(seq, ctypes.byref(n), *[_ptr(out[k]) for k in
                                                      ("type", "gtype", "seg_begin", "seg_end")],
                              ctypes.byref(ns))
    if rc:
        raise MrsimError(rc, "mrsim_seq_info")
    out["n_samples_total"] = ns.value
    return out


def mrsim_group(ctx, ph, seq) -> int:
    h = ctypes.c_void_p()
    rc = lib().mrsim_group(ctx, ph, seq, ctypes.byref(h))
    _check(ctx, rc, "mrsim_group")
    return h.value


def mrsim_group_info(groups, gtype, K=None):
    n = ctypes.c_int64()
    gid = None if K is None else np.empty(K, np.int32)
    rc = lib().mrsim_group_info(groups, gtype, ctypes.byref(n), _ptr(gid))
    if rc:
        raise MrsimError(rc, "mrsim_group_info")
    return n.value, gid


def mrsim_coils(ctx, ph, sens, flags=0):
    """Attach receive-coil sensitivities float32 [P, 2, K] (None: detach)."""
    if sens is None:
        _check(ctx, lib().mrsim_coils(ctx, ph, 0, None, flags), "mrsim_coils")
        return 0
    if isinstance(sens, np.ndarray):
        sens = np.ascontiguousarray(sens, np.float32)
        n = int(sens.shape[0])
    else:  # torch tensor on the device
        n = int(sens.shape[0])
    _check(ctx, lib().mrsim_coils(ctx, ph, n, _ptr(sens), flags), "mrsim_coils")
    return n


def mrsim_run(ctx, ph, seq, groups, mode, precision, signal, M_final=None, out_flags=0):
    rc = lib().mrsim_run(ctx, ph, seq, groups, mode, precision, _ptr(signal), _ptr(M_final),
                         out_flags)
    _check(ctx, rc, "mrsim_run")


def mrsim_run_batch(ctx, phs, seqs, groups, signals):
    n = len(phs)
    A = ctypes.c_void_p * n
    rc = lib().mrsim_run_batch(ctx, n, A(*phs), A(*seqs), A(*groups),
                               A(*[_ptr(s) for s in signals]))
    _check(ctx, rc, "mrsim_run_batch")


def mrsim_recon_cartesian(ctx, signal, layout, image=None, flags=0):
    """Image [n_pe, n_ro] complex128 of one coil's signal (numpy, or torch
    device tensors with flags=PTR_DEVICE) given a k-space layout dict
    (n_ro, n_pe, row, col0, dir as from mrsim_inputs.kspace_layout)."""
    n_ro, n_pe = int(layout["n_ro"]), int(layout["n_pe"])
    row = np.ascontiguousarray(layout["row"], np.int32)
    col0 = np.ascontiguousarray(layout["col0"], np.int32)
    d = np.ascontiguousarray(layout["dir"], np.int8)
    if image is None:
        image = np.zeros((n_pe, 2 * n_ro), np.float64)
    if isinstance(signal, np.ndarray):
        signal = np.ascontiguousarray(signal)
        if signal.dtype == np.complex128:
            signal = signal.view(np.float64)
    _check(ctx, lib().mrsim_recon_cartesian(ctx, len(row), n_ro, n_pe, _ptr(signal), _ptr(row),
                                            _ptr(col0), _ptr(d), flags, _ptr(image)),
           "mrsim_recon_cartesian")
    if isinstance(image, np.ndarray):
        return image.view(np.complex128).reshape(n_pe, n_ro)
    return image


def mrsim_cluster(ctx, ph, K, n_clusters, scale=None, max_iter=300, te=T2W_TE, tr=T2W_TR,
                  want_labels=True):
    """Group-reducing preprocessing of phantom ``ph`` (K isochromats).
    Returns (new phantom handle, number of clusters n, labels int32 [K] or
    None, centres float64 [n, 3] as T1 s, T2 s, dB0 Hz)."""
    labels = np.empty(K, np.int32) if want_labels else None
    centres = np.zeros((max(n_clusters, 1), 3), np.float64)
    sc = None if scale is None else np.ascontiguousarray(scale, np.float64)
    te = np.ascontiguousarray(te, np.float64)
    n = ctypes.c_int(0)
    out = ctypes.c_void_p()
    rc = lib().mrsim_cluster(ctx, ph, n_clusters, _ptr(sc), max_iter, len(te),
                             _ptr(te) if len(te) else None, float(tr), _ptr(labels),
                             _ptr(centres), ctypes.byref(n), ctypes.byref(out))
    _check(ctx, rc, "mrsim_cluster")
    return out.value, n.value, labels, centres[: n.value].copy()


def mrsim_profile_enable(ctx, on=True):
    lib().mrsim_profile_enable(ctx, int(on))


def mrsim_profile_reset(ctx):
    lib().mrsim_profile_reset(ctx)


def mrsim_profile_get(ctx):
    """All per-kernel entries: {name: (launches, ms_total)}."""
    out = {}
    buf = ctypes.create_string_buffer(128)
    i = 0
    while True:
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        rc = lib().mrsim_profile_get(ctx, i, buf, 128, ctypes.byref(n), ctypes.byref(ms))
        if rc:
            break
        out[buf.value.decode()] = (n.value, ms.value)
        i += 1
    return out


def mrsim_launch_count(ctx) -> int:
    return int(lib().mrsim_launch_count(ctx))


def mrsim_set_tuning(ctx, param, value):
    _check(ctx, lib().mrsim_set_tuning(ctx, param, value), "mrsim_set_tuning")


def mrsim_get_tuning(ctx, param) -> int:
    v = ctypes.c_int()
    rc = lib().mrsim_get_tuning(ctx, param, ctypes.byref(v))
    if rc:
        raise MrsimError(rc, "mrsim_get_tuning")
    return v.value


def mrsim_set_reproducible(ctx, on):
    _check(ctx, lib().mrsim_set_reproducible(ctx, int(on)), "mrsim_set_reproducible")


def mrsim_get_reproducible(ctx) -> bool:
    v = ctypes.c_int()
    rc = lib().mrsim_get_reproducible(ctx, ctypes.byref(v))
    if rc:
        raise MrsimError(rc, "mrsim_get_reproducible")
    return bool(v.value)


def mrsim_autotune(ctx, ph, seq, groups, mode, precision, reps=1):
    _check(ctx, lib().mrsim_autotune(ctx, ph, seq, groups, mode, precision, reps),
           "mrsim_autotune")
    return {p: mrsim_get_tuning(ctx, p) for p in (TUNE_FUSED_NI, TUNE_PLAIN_RF_NI,
                                                   TUNE_ADC_CTAS_PER_SM, TUNE_PRECOMP_LANES,
                                                   TUNE_PRECOMP_STEPS, TUNE_CELL_NI,
                                                   TUNE_CELL_ROWS)}


def mrsim_surrogate_train(ctx, seq, lo, hi, n_train=1 << 22, epochs=20, batch=16384, lr=3e-3,
                          seed=1005, bound=1e-3) -> int:
    h = ctypes.c_void_p()
    lo = np.ascontiguousarray(lo, np.float64)
    hi = np.ascontiguousarray(hi, np.float64)
    rc = lib().mrsim_surrogate_train(ctx, seq, _ptr(lo), _ptr(hi), int(n_train), int(epochs),
                                     int(batch), float(lr), int(seed), float(bound),
                                     ctypes.byref(h))
    _check(ctx, rc, "mrsim_surrogate_train")
    return h.value


SURROGATE_STATS = ["networks", "train_loss", "val_max_err", "cells_served", "val_served",
                   "val_served_max_err", "groups_served", "groups_exact"]


def mrsim_surrogate_stats(sur, ctx=None) -> dict:
    out = np.zeros(8)
    rc = lib().mrsim_surrogate_stats(sur, ctx, _ptr(out))
    if rc:
        raise MrsimError(rc, "mrsim_surrogate_stats")
    return dict(zip(SURROGATE_STATS, out.tolist()))


def mrsim_surrogate_check(ctx, sur, seq, groups):
    """Largest entry error of the network's transitions over the groups the
    gate serves in a run, against the exact FP64 transitions; returns
    (max_err, n_served)."""
    e = ctypes.c_double()
    n = ctypes.c_int64()
    _check(ctx, lib().mrsim_surrogate_check(ctx, sur, seq, groups, ctypes.byref(e),
                                            ctypes.byref(n)), "mrsim_surrogate_check")
    return e.value, n.value


def mrsim_surrogate_infer(ctx, params, x):
    """Raw network outputs [n, 12] of the tensor-core inference kernel."""
    p = np.ascontiguousarray(params, np.float32)
    xx = np.ascontiguousarray(x, np.float32)
    n = xx.shape[0]
    y = np.zeros((n, 12), np.float32)
    _check(ctx, lib().mrsim_surrogate_infer(ctx, _ptr(p), n, _ptr(xx), _ptr(y)),
           "mrsim_surrogate_infer")
    return y


def mrsim_surrogate_use(ctx, sur):
    _check(ctx, lib().mrsim_surrogate_use(ctx, sur), "mrsim_surrogate_use")


def mrsim_surrogate_eval(ctx, params, x, t):
    """GPU forward + backward of the network: returns (y, grad, loss)."""
    params = np.ascontiguousarray(params, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    n = x.shape[0]
    y = np.zeros((n, 12), np.float32)
    g = np.zeros(params.size, np.float32)
    L = ctypes.c_double()
    rc = lib().mrsim_surrogate_eval(ctx, _ptr(params), n, _ptr(x), _ptr(t), _ptr(y), _ptr(g),
                                    ctypes.byref(L))
    _check(ctx, rc, "mrsim_surrogate_eval")
    return y, g, L.value


def mrsim_free_surrogate(sur):
    lib().mrsim_free_surrogate(sur)


def mrsim_adc_grouped_noalloc(K, mx, my, gid, n_groups, gpos, gdB0, gT2, n_samples, tau, kmom,
                              signal, stream=None) -> int:
    """Allocation-free grouped with-ADC window signal (device tensors in,
    device signal out).  Returns the status code (0 on success)."""
    return int(lib().mrsim_adc_grouped_noalloc(int(K), _ptr(mx), _ptr(my), _ptr(gid),
                                               int(n_groups), _ptr(gpos), _ptr(gdB0), _ptr(gT2),
                                               int(n_samples), _ptr(tau), _ptr(kmom),
                                               _ptr(signal), stream))


def mrsim_free_phantom(ph):
    lib().mrsim_free_phantom(ph)


def mrsim_free_seq(seq):
    lib().mrsim_free_seq(seq)


def mrsim_free_groups(groups):
    lib().mrsim_free_groups(groups)


# -------------------------------------------------------------- helpers -----
class Context:
    """Owns one mrsim context and the handles created through it."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self.h = mrsim_create(device, stream)
        self._handles = []
        self._coils = {}  # phantom handle -> receive coils attached

    def close(self):
        for kind, h in reversed(self._handles):
            {"ph": mrsim_free_phantom, "seq": mrsim_free_seq, "grp": mrsim_free_groups}[kind](h)
        self._handles = []
        if self.h:
            mrsim_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def phantom(self, p, device_ptrs: bool = False) -> int:
        """Upload an ``mrsim_inputs.Phantom`` (numpy) or a dict of torch
        device tensors (device_ptrs=True)."""
        if device_ptrs:
            a = p
            K = a["x"].numel()
            M_init = a.get("M_init")
            h = mrsim_phantom(self.h, K, a["x"], a["y"], a["z"], a["T1"], a["T2"], a["dB0"],
                              a["M0"], a.get("b1"), M_init, PTR_DEVICE)
        else:
            keep = [_f32(p.x), _f32(p.y), _f32(p.z), _f32(p.T1), _f32(p.T2), _f32(p.dB0),
                    _f32(p.M0), _f32(p.b1),
                    None if p.M_init is None else np.ascontiguousarray(p.M_init, np.float32)]
            h = mrsim_phantom(self.h, p.K, *keep)
            if getattr(p, "coils", None) is not None:
                self._coils[h] = mrsim_coils(self.h, h, p.coils)
        self._handles.append(("ph", h))
        return h

    def cluster(self, ph: int, K: int, n_clusters: int, **kw):
        """mrsim_cluster on an uploaded phantom; the new phantom is owned by
        this context (receive coils carried over)."""
        h, n, labels, centres = mrsim_cluster(self.h, ph, K, n_clusters, **kw)
        self._handles.append(("ph", h))
        if self._coils.get(ph):
            self._coils[h] = self._coils[ph]
        return h, n, labels, centres

    def sequence(self, s) -> int:
        keep = [np.ascontiguousarray(s.dt, np.float64), np.ascontiguousarray(s.repeat, np.int32),
                _f32(s.b1re), _f32(s.b1im), _f32(s.gx), _f32(s.gy), _f32(s.gz),
                np.ascontiguousarray(s.adc, np.uint8)]
        h = mrsim_sequence(self.h, s.n_seg, *keep)
        self._handles.append(("seq", h))
        return h

    def group(self, ph: int, seq: int) -> int:
        h = mrsim_group(self.h, ph, seq)
        self._handles.append(("grp", h))
        return h

    def run(self, ph, seq, groups=None, mode=GROUPED, precision=FP32, n_samples=None,
            K=None, want_M=False):
        """Signal complex128 [n_samples] ([P, n_samples] with P receive
        coils) and, if want_M, the final magnetization [3, K]."""
        if n_samples is None:
            n_samples = mrsim_seq_info(seq)["n_samples_total"]
        P = self._coils.get(ph, 0)
        sig = np.zeros(2 * max(n_samples, 1) * max(P, 1), np.float64)
        M = np.zeros((3, K), np.float32) if want_M else None
        mrsim_run(self.h, ph, seq, groups if groups else None, mode, precision, sig, M)
        out = sig[: 2 * n_samples * max(P, 1)].view(np.complex128).copy()
        return (out.reshape(P, n_samples) if P else out), M

    def free(self, kind: str, h: int):
        self._handles = [(k, x) for (k, x) in self._handles if x != h]
        self._coils.pop(h, None)
        {"ph": mrsim_free_phantom, "seq": mrsim_free_seq, "grp": mrsim_free_groups}[kind](h)
