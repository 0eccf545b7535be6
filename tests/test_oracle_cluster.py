"""Pins of the clustering oracle (Sec. 3.3, Fig. 4) to facts fixed outside it:
exact rational means and SSEs recomputed with Python integers, brute force over
every 2-partition of tiny sets, blob structures whose clustering is known, the
least-squares property of the M0 refit, and the special cases (one cluster,
fewer distinct values than clusters, values already on the feature grid)."""

import dataclasses
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import cluster as oc
from mrsim_inputs.phantom import mapped_phantom


def py_mean(cols):
    """Exact mean (Fractions) of a list of integer 3-vectors."""
    n = len(cols)
    return [Fraction(sum(int(c[i]) for c in cols), n) for i in range(3)]


def py_sse(cols):
    mu = py_mean(cols)
    return sum(sum((int(c[i]) - mu[i]) ** 2 for i in range(3)) for c in cols)


def d2(c, mu):
    return sum((int(c[i]) - mu[i]) ** 2 for i in range(3))


def features(n, rng, lo=1, hi=2000):
    X = rng.integers(lo, hi, size=(3, n)).astype(np.int64)
    X[2] -= hi // 2  # dB0 may be negative
    return X


def test_hierarchical_blobs_are_found_with_exact_means():
    """Eight tight blobs at the corners of a nested arrangement (separations
    20000, 2000, 200 along the three axes, radius 5): every bisection must cut
    between the two halves of one level, so eight clusters are the blobs."""
    rng = np.random.default_rng(3)
    cols, truth = [], []
    for b, (i, j, k) in enumerate(itertools.product(range(2), repeat=3)):
        centre = np.array([1000 + 20000 * i, 1000 + 2000 * j, 200 * k])
        m = int(rng.integers(20, 60))
        cols.append(centre[:, None] + rng.integers(-5, 6, size=(3, m)))
        truth += [b] * m
    X = np.concatenate(cols, axis=1).astype(np.int64)
    perm = rng.permutation(X.shape[1])
    X, truth = X[:, perm], np.asarray(truth)[perm]
    labels, centres, history = oc.bisecting_kmeans(X, 8)
    assert len(centres) == 8 and len(history) == 7
    # the partition is the blob partition
    pairs = set(zip(labels.tolist(), truth.tolist()))
    assert len(pairs) == 8 and len({p[0] for p in pairs}) == 8
    for c in range(8):
        mu = py_mean([X[:, k] for k in np.flatnonzero(labels == c)])
        assert [float(m) for m in mu] == centres[c].tolist()


def test_fewer_distinct_values_than_clusters():
    rng = np.random.default_rng(4)
    base = features(5, rng)
    X = base[:, rng.integers(0, 5, size=300)]
    for n in (5, 9):
        labels, centres, history = oc.bisecting_kmeans(X, n)
        assert len(centres) == 5
        for c in range(5):
            cols = X[:, labels == c]
            assert np.all(cols == cols[:, :1])  # one distinct value per cluster
            assert centres[c].tolist() == cols[:, 0].astype(float).tolist()


def test_one_cluster_is_the_mean():
    rng = np.random.default_rng(5)
    X = features(257, rng)
    labels, centres, history = oc.bisecting_kmeans(X, 1)
    assert history == [] and not labels.any()
    assert centres[0].tolist() == [float(m) for m in py_mean(list(X.T))]


def replay(labels, history):
    """Partitions before each split, recovered by undoing the splits from the
    final labels (last split first)."""
    lab = labels.copy()
    states = []
    for parent, new in reversed(history):
        states.append((parent, new, lab.copy()))
        lab[lab == new] = parent
    return list(reversed(states))


@pytest.mark.parametrize("seed", [6, 7])
def test_split_order_and_fixed_points(seed):
    """Before every split, the split cluster has the largest exact SSE of all
    clusters (ties: smaller id); after it, each side's members are no nearer
    the other side's exact mean (a fixed point of the 2-means step)."""
    rng = np.random.default_rng(seed)
    X = features(400, rng, hi=300)
    labels, centres, history = oc.bisecting_kmeans(X, 10)
    assert len(history) == 9
    cols = list(X.T)
    for parent, new, after in replay(labels, history):
        before = np.where(after == new, parent, after)
        ids = sorted(set(before.tolist()))
        sse = {c: py_sse([cols[k] for k in np.flatnonzero(before == c)]) for c in ids}
        best = max(s for s in sse.values())
        assert sse[parent] == best and parent == min(c for c in ids if sse[c] == best)
        s0 = [cols[k] for k in np.flatnonzero(after == parent)]
        s1 = [cols[k] for k in np.flatnonzero(after == new)]
        m0, m1 = py_mean(s0), py_mean(s1)
        eps = Fraction(1, 10 ** 6)
        assert all(d2(c, m0) <= d2(c, m1) + eps for c in s0)
        assert all(d2(c, m1) <= d2(c, m0) + eps for c in s1)


def test_two_means_matches_brute_force_on_tiny_sets():
    """For tiny sets, the first split is a 2-partition whose sides are no nearer
    the other side's mean (checked against the list of all such partitions);
    for clearly bimodal sets it is the partition of least total SSE."""
    rng = np.random.default_rng(8)
    for trial in range(30):
        m = int(rng.integers(3, 9))
        if trial % 2:
            X = features(m, rng, hi=50)
        else:  # two clumps far apart
            X = np.concatenate([features(m // 2, rng, hi=20),
                                features(m - m // 2, rng, hi=20) + 5000], axis=1)
        cols = list(X.T)
        labels, _, _ = oc.bisecting_kmeans(X, 2)
        got = frozenset(np.flatnonzero(labels == 1).tolist())
        fixed, best, best_sse = [], None, None
        for r in range(1, m):
            for S1 in itertools.combinations(range(m), r):
                S0 = [k for k in range(m) if k not in S1]
                m0 = py_mean([cols[k] for k in S0])
                m1 = py_mean([cols[k] for k in S1])
                if all(d2(cols[k], m0) <= d2(cols[k], m1) for k in S0) and \
                        all(d2(cols[k], m1) < d2(cols[k], m0) for k in S1):
                    fixed.append(frozenset(S1))
                tot = py_sse([cols[k] for k in S0]) + py_sse([cols[k] for k in S1])
                if best_sse is None or tot < best_sse:
                    best, best_sse = {frozenset(S1), frozenset(S0)}, tot
        assert got in fixed
        if trial % 2 == 0:
            assert got in best


def grid_phantom_values(rng, K, D):
    """A mapped phantom whose (T1, T2, dB0) take D distinct values on the
    1/64 ms and 1/64 Hz grid."""
    p = mapped_phantom(16, 16, 1, 3, seed=9)
    t1 = rng.integers(640, 192000, D) / 64000.0
    t2 = rng.integers(640, 32000, D) / 64000.0
    db = rng.integers(-2000, 2000, D) / 64.0
    pick = rng.integers(0, D, p.K)
    f32 = lambda a: np.ascontiguousarray(a[pick], np.float32)
    return dataclasses.replace(p, T1=f32(t1), T2=f32(t2), dB0=f32(db))


def test_values_on_the_grid_are_kept_when_no_clustering_is_needed():
    rng = np.random.default_rng(10)
    p = grid_phantom_values(rng, 256, 12)
    r = oc.cluster_phantom(p, 16)
    assert len(r.centres) == 12
    for name in ("T1", "T2", "dB0", "M0"):
        assert np.array_equal(getattr(r.phantom, name), getattr(p, name)), name


def test_m0_refit_is_the_least_squares_fit():
    """The refitted M0 leaves residuals I_e - M0' f_e(c) orthogonal to f(c)
    (normal equation of the fit); with one echo it reproduces the image."""
    rng = np.random.default_rng(11)
    K = 64
    T1 = rng.uniform(0.2, 2.5, K)
    T2 = rng.uniform(0.02, 0.3, K)
    T1c = T1 * rng.uniform(0.8, 1.2, K)
    T2c = T2 * rng.uniform(0.8, 1.2, K)
    M0 = rng.uniform(0.3, 1.0, K)
    M0n = oc.refit_M0(M0, T1, T2, T1c, T2c).astype(np.float64)
    for k in range(K):
        f = lambda a, b, te: (1.0 - math.exp(-4.5 / a)) * math.exp(-te / b)
        I = [M0[k] * f(T1[k], T2[k], te) for te in oc.T2W_TE]
        fc = [f(T1c[k], T2c[k], te) for te in oc.T2W_TE]
        ls = sum(i * c for i, c in zip(I, fc)) / sum(c * c for c in fc)
        assert abs(M0n[k] - ls) <= 1e-6 * ls  # float32 output
        resid = sum((i - ls * c) * c for i, c in zip(I, fc))
        assert abs(resid) <= 1e-12 * sum(abs(i * c) for i, c in zip(I, fc))
    one = oc.refit_M0(M0, T1, T2, T1c, T2c, te=(0.08,)).astype(np.float64)
    img = M0 * (1 - np.exp(-4.5 / T1)) * np.exp(-0.08 / T2)
    fit = one * (1 - np.exp(-4.5 / T1c)) * np.exp(-0.08 / T2c)
    assert np.max(np.abs(fit - img) / img) <= 2e-7
    assert np.array_equal(oc.refit_M0(M0, T1, T2, T1c, T2c, te=()), M0.astype(np.float32))


def test_quantize_rejects_what_cannot_be_clustered():
    p = mapped_phantom(8, 8, 1, 2, seed=12)
    bad = dataclasses.replace(p, T1=np.where(np.arange(p.K) == 3, np.inf, p.T1).astype(np.float32))
    with pytest.raises(ValueError):
        oc.quantize(bad)
    tiny = dataclasses.replace(p, T2=np.full(p.K, 1e-6, np.float32))
    with pytest.raises(ValueError):
        oc.quantize(tiny)
    far = dataclasses.replace(p, dB0=np.full(p.K, 20000.0, np.float32))
    with pytest.raises(ValueError):
        oc.quantize(far)


def test_mapped_phantom_clusters_reduce_groups():
    """On the parameter-mapping stand-in, n clusters leave at most n distinct
    (T1, T2, dB0) values and so at most n x (distinct x) Gx-type keys."""
    p = mapped_phantom(48, 48, 2, 12, seed=13)
    before = np.unique(np.stack([p.T1, p.T2, p.dB0]), axis=1).shape[1]
    r = oc.cluster_phantom(p, 32)
    q = r.phantom
    after = np.unique(np.stack([q.T1, q.T2, q.dB0]), axis=1).shape[1]
    assert before > 32 and after == 32 == len(r.centres)
    gx = np.unique(np.stack([q.x, q.T1, q.T2, q.dB0]), axis=1).shape[1]
    assert gx <= 32 * len(np.unique(q.x))
    # every isochromat carries its cluster's centre
    assert np.array_equal(q.T1, r.centres[r.labels, 0].astype(np.float32))


def test_equal_sse_goes_to_the_smaller_id():
    """Two translated copies of one two-blob set: the first split separates the
    copies, which then have exactly equal SSE, so the second split must take
    id 0, and the third the other copy (id 1)."""
    rng = np.random.default_rng(14)
    half = np.concatenate([rng.integers(0, 6, size=(3, 40)),
                           rng.integers(0, 6, size=(3, 40)) + np.array([[300], [0], [0]])],
                          axis=1)
    X = np.concatenate([half, half + np.array([[0], [50000], [0]])], axis=1).astype(np.int64)
    X = X[:, rng.permutation(X.shape[1])]
    labels, centres, history = oc.bisecting_kmeans(X, 4)
    assert history[0] == (0, 1)
    sizes = np.bincount(labels)
    assert history[1] == (0, 2) and history[2] == (1, 3)
    cols = list(X.T)
    s0 = py_sse([cols[k] for k in np.flatnonzero((labels == 0) | (labels == 2))])
    s1 = py_sse([cols[k] for k in np.flatnonzero((labels == 1) | (labels == 3))])
    assert s0 == s1 and np.all(sizes == 40)
