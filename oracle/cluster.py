"""Group-reducing preprocessing of a phantom (reference for the CUDA path).

TEST INFRASTRUCTURE ONLY: loaded by the tests and the benchmark's CPU leg,
never by the library.

Sec. 3.3 and Fig. 4: when the isochromats' (T1, T2, dB0) take too many values,
the groups of Sec. 2.4 are nearly as many as the isochromats.  The paper then
clusters the parameter maps in the space (T1, T2, dB0) with a bisecting K-means,
gives every isochromat its cluster's centre values, and refits M0 from the
T2-weighted images with those centre values.  The paper gives no settings
beyond "bisecting K-means"; the readings taken here are:

R1  Space.  Feature i of isochromat k is the integer x_i(k) = rint(v_i(k) s_i)
    of its value v = (T1 [s], T2 [s], dB0 [Hz]) times a scale s (default
    64000/s, 64000/s, 64/Hz: T1 and T2 in 1/64 ms, dB0 in 1/64 Hz, so one
    millisecond weighs as much as one hertz).  Integer features make every sum
    below exact, so the result does not depend on summation order.
R2  Strategy.  Start with one cluster (id 0) holding every isochromat.  Split
    the cluster with the largest sum of squared distances to its mean (SSE,
    compared exactly); ties go to the smaller id.  A cluster whose members all
    coincide (SSE 0) is never split; when no cluster can be split, stop with
    fewer clusters than asked.
R3  Initial centres of a split: a = the member farthest from the cluster mean,
    b = the member farthest from a (ties: the smallest isochromat index).
R4  2-means (Lloyd): a member goes to side 1 when it is strictly nearer the
    side-1 centre, else to side 0; the new centres are the sides' means.  Stop
    when the centres repeat exactly, after max_iter passes, or when a side
    would be empty (the previous pass then stands).  Distances to centres are
    ((x0 - c0)^2 + (x1 - c1)^2) + (x2 - c2)^2 in FP64, one rounding per
    operation; centres are FP64 means (exact integer sum / count).
R5  Numbering.  Side 0 keeps the split cluster's id; side 1 takes the next
    free id, so ids are 0..n-1 in order of creation.
R6  Centre values.  Cluster mean / s_i in FP64, stored as float32 in the new
    phantom (on the grid of R1: a singleton's centre is its value rounded to
    1/64 ms or 1/64 Hz).
R7  M0 refit.  The T2-weighted images of the volunteer scan (Table 1: FSE, TR
    4500 ms, TE 20/60/100/140 ms) are modelled from the initial maps as
    I_e(k) = M0(k) f_e(T1(k), T2(k)), f_e(T1, T2) = (1 - exp(-TR/T1))
    exp(-TE_e/T2); the new M0 is their least-squares fit with the centre values,
    M0'(k) = sum_e I_e(k) f_e(c) / sum_e f_e(c)^2 (M0 kept where the
    denominator is 0 or no echo is given).
"""

from __future__ import annotations

import dataclasses
from fractions import Fraction

import numpy as np

DEFAULT_SCALE = (64000.0, 64000.0, 64.0)
T2W_TE = (0.020, 0.060, 0.100, 0.140)
T2W_TR = 4.5
MAX_FEATURE = 1 << 20


def quantize(ph, scale=DEFAULT_SCALE):
    """Integer features [3, K] (R1).  Raises ValueError where a value is not
    finite, |x| > 2^20, or T1 / T2 round below one step."""
    V = np.stack([ph.T1, ph.T2, ph.dB0]).astype(np.float64)
    if not np.all(np.isfinite(V)):
        raise ValueError("non-finite T1, T2 or dB0")
    X = np.rint(V * np.asarray(scale, np.float64)[:, None])
    if np.any(np.abs(X) > MAX_FEATURE):
        raise ValueError("feature outside [-2^20, 2^20]")
    if np.any(X[:2] < 1):
        raise ValueError("T1 or T2 below one clustering step")
    return X.astype(np.int64)


def exact_sum(a) -> int:
    """Exact integer sum of an int64 array (chunks of 2^20 cannot overflow)."""
    a = np.asarray(a, np.int64)
    return sum(int(a[i:i + (1 << 20)].sum()) for i in range(0, a.size, 1 << 20))


def dist2(X, c):
    """R4 distance of the columns of X (int64 [3, m]) to centre c (3 floats)."""
    Xf = X.astype(np.float64)
    return ((Xf[0] - c[0]) ** 2 + (Xf[1] - c[1]) ** 2) + (Xf[2] - c[2]) ** 2


def mean(X):
    n = X.shape[1]
    return np.array([float(exact_sum(X[i])) / float(n) for i in range(3)])


def sse(X) -> Fraction:
    """Exact sum of squared distances of the columns of X to their mean."""
    n = X.shape[1]
    num = 0
    for i in range(3):
        s = exact_sum(X[i])
        num += n * exact_sum(X[i] * X[i]) - s * s
    return Fraction(num, n)


def split(X, max_iter):
    """2-means of the columns of X (R3, R4).  Returns side (bool [m]) and the
    centres of the pass that made it."""
    mu = mean(X)
    a = int(np.argmax(dist2(X, mu)))               # first index at the maximum
    d_a = ((X - X[:, a:a + 1]) ** 2).sum(axis=0)   # exact integers
    b = int(np.argmax(d_a))
    c0 = X[:, a].astype(np.float64)
    c1 = X[:, b].astype(np.float64)
    kept = None
    for _ in range(max_iter):
        side = dist2(X, c1) < dist2(X, c0)
        n1 = int(side.sum())
        if n1 == 0 or n1 == side.size:
            break
        kept = (side, c0, c1)
        m0, m1 = mean(X[:, ~side]), mean(X[:, side])
        if np.array_equal(m0, c0) and np.array_equal(m1, c1):
            break
        c0, c1 = m0, m1
    assert kept is not None  # the first pass puts a on side 0 and b on side 1
    return kept


def bisecting_kmeans(X, n_clusters, max_iter=300):
    """R2-R5 on integer features X [3, K].

    Returns (labels int32 [K], centres float64 [n, 3] in feature units,
    history [(parent, new id)] in split order)."""
    K = X.shape[1]
    labels = np.zeros(K, np.int32)
    members = [np.arange(K)]
    score = [sse(X)]
    history = []
    while len(members) < n_clusters:
        cand = [c for c in range(len(members)) if score[c] > 0]
        if not cand:
            break
        c = max(cand, key=lambda j: (score[j], -j))
        idx = members[c]
        side, _, _ = split(X[:, idx], max_iter)
        new = len(members)
        members[c], moved = idx[~side], idx[side]
        members.append(moved)
        labels[moved] = new
        score[c] = sse(X[:, members[c]])
        score.append(sse(X[:, moved]))
        history.append((c, new))
    centres = np.stack([mean(X[:, m]) for m in members])
    return labels, centres, history


def t2w_weights(T1, T2, te=T2W_TE, tr=T2W_TR):
    """f_e(T1, T2) of R7 for every echo (float64 [n_echo, ...])."""
    T1 = np.asarray(T1, np.float64)
    T2 = np.asarray(T2, np.float64)
    return np.stack([(1.0 - np.exp(-tr / T1)) * np.exp(-t / T2) for t in te])


def refit_M0(M0, T1, T2, T1c, T2c, te=T2W_TE, tr=T2W_TR):
    """R7 in FP64; returns float32."""
    M0 = np.asarray(M0, np.float64)
    if len(te) == 0:
        return M0.astype(np.float32)
    fo = t2w_weights(T1, T2, te, tr)
    fc = t2w_weights(T1c, T2c, te, tr)
    num = (M0 * fo * fc).sum(axis=0)
    den = (fc * fc).sum(axis=0)
    out = np.where(den > 0.0, num / np.where(den > 0.0, den, 1.0), M0)
    return out.astype(np.float32)


@dataclasses.dataclass
class Clustered:
    phantom: object        # the new phantom (positions, b1, M_init, coils kept)
    labels: np.ndarray     # int32 [K], cluster id per isochromat
    centres: np.ndarray    # float64 [n, 3]: T1 (s), T2 (s), dB0 (Hz), R6 before float32
    history: list          # [(parent, new id)] in split order


def cluster_phantom(ph, n_clusters, scale=DEFAULT_SCALE, max_iter=300, te=T2W_TE,
                    tr=T2W_TR) -> Clustered:
    """Fig. 4 on a phantom: R1-R7."""
    if n_clusters < 1 or max_iter < 1:
        raise ValueError("n_clusters and max_iter must be positive")
    X = quantize(ph, scale)
    labels, cq, history = bisecting_kmeans(X, n_clusters, max_iter)
    centres = cq / np.asarray(scale, np.float64)[None, :]
    c32 = centres.astype(np.float32)
    T1n, T2n, dBn = (np.ascontiguousarray(c32[labels, i]) for i in range(3))
    M0n = refit_M0(ph.M0, ph.T1, ph.T2, T1n, T2n, te, tr)
    new = dataclasses.replace(ph, T1=T1n, T2=T2n, dB0=dBn, M0=M0n)
    return Clustered(new, labels, centres, history)
