"""Group-reducing preprocessing (Sec. 3.3, Fig. 4) on the GPU against the
clustering oracle.

Cluster ids per isochromat, centre values and the new T1 / T2 / dB0 are
compared bit for bit: the features are integers, every sum is exact, and both
sides form means and distances with one rounding per FP64 operation, so any
difference is a defect.  The refitted M0 goes through exp, whose last bit may
differ between the CUDA and host math libraries: within one float32 ulp."""

import dataclasses
import hashlib
import os

import numpy as np
import pytest

import oracle
from oracle import cluster as oc
from mrsim_inputs import configs, phantom_digest
from mrsim_inputs.phantom import continuous_phantom, mapped_phantom
from mrsim_inputs.sequence import spin_echo_2d

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx(mrsim):
    c = mrsim.Context(0)
    yield c
    c.close()


def gpu_cluster(mrsim, ctx, ph, n, **kw):
    hp = ctx.phantom(ph)
    h, m, labels, centres = ctx.cluster(hp, ph.K, n, **kw)
    arrays = mrsim.mrsim_phantom_read(ctx.h, h, ph.K)
    return hp, h, m, labels, centres, arrays


def within_ulp(a, b, n=1):
    """Non-negative float32 arrays within n units in the last place."""
    ia = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
    ib = np.asarray(b, np.float32).view(np.int32).astype(np.int64)
    return int(np.max(np.abs(ia - ib))) <= n


def check(r, m, labels, centres, arrays):
    assert m == len(r.centres)
    assert np.array_equal(labels, r.labels)
    assert np.array_equal(centres, r.centres)
    for name in ("T1", "T2", "dB0"):
        assert np.array_equal(arrays[name], getattr(r.phantom, name)), name
    assert within_ulp(arrays["M0"], r.phantom.M0)


def oracle_kw(kw):
    return {k: v for k, v in kw.items() if k in ("scale", "max_iter", "te", "tr")}


CASES = {
    "mapped_b0_field": (lambda: configs.mapped_small(32, 32, 2), [1, 7, 64]),
    "mapped_b0_zero": (lambda: mapped_phantom(32, 32, 2, 16, seed=1006), [32]),
    "per_isochromat_b0": (lambda: continuous_phantom(16, 16, 2, 3, seed=47), [16]),
}


@pytest.mark.parametrize("case", list(CASES))
def test_cluster_matches_oracle(mrsim, ctx, case):
    make, ns = CASES[case]
    ph = make()
    for n in ns:
        r = oc.cluster_phantom(ph, n)
        hp, h, m, labels, centres, arrays = gpu_cluster(mrsim, ctx, ph, n)
        check(r, m, labels, centres, arrays)
        ctx.free("ph", h)
        ctx.free("ph", hp)


def test_cluster_settings_and_early_stop(mrsim, ctx):
    """Other feature scales, a capped number of 2-means passes, another echo
    model, no refit, and fewer distinct values than clusters asked."""
    ph = configs.mapped_small(32, 32, 2)
    for kw in (dict(scale=(8000.0, 16000.0, 8.0)), dict(max_iter=2),
               dict(te=(0.08,), tr=2.0), dict(te=())):
        r = oc.cluster_phantom(ph, 24, **oracle_kw(kw))
        hp, h, m, labels, centres, arrays = gpu_cluster(mrsim, ctx, ph, 24, **kw)
        check(r, m, labels, centres, arrays)
        if kw.get("te") == ():
            assert np.array_equal(arrays["M0"], ph.M0)
    rng = np.random.default_rng(10)
    base = mapped_phantom(16, 16, 1, 3, seed=9)
    pick = rng.integers(0, 12, base.K)
    f32 = lambda v: np.ascontiguousarray(v[pick], np.float32)
    ph = dataclasses.replace(base, T1=f32(rng.integers(640, 192000, 12) / 64000.0),
                             T2=f32(rng.integers(640, 32000, 12) / 64000.0),
                             dB0=f32(rng.integers(-2000, 2000, 12) / 64.0))
    r = oc.cluster_phantom(ph, 16)
    hp, h, m, labels, centres, arrays = gpu_cluster(mrsim, ctx, ph, 16)
    assert m == 12
    check(r, m, labels, centres, arrays)
    for name in ("T1", "T2", "dB0", "M0"):  # values on the grid come back unchanged
        assert np.array_equal(arrays[name], getattr(ph, name))


def test_cluster_deep_and_wide_trees(mrsim, ctx):
    """Splits are computed many at a time and the greedy order is replayed on
    them: a chain-like tree (geometric dB0 values, every split peels off the
    top values) and a wide one (1024 clusters of 2048 distinct values) give
    the sequential result, ids included."""
    base = mapped_phantom(16, 16, 2, 3, seed=12)
    i = np.arange(base.K) % 200
    ph = dataclasses.replace(base, T1=np.full(base.K, 0.8, np.float32),
                             T2=np.full(base.K, 0.07, np.float32),
                             dB0=np.ascontiguousarray(0.5 * 1.05 ** i, np.float32))
    for n in (2, 150):
        r = oc.cluster_phantom(ph, n)
        hp, h, m, labels, centres, arrays = gpu_cluster(mrsim, ctx, ph, n)
        check(r, m, labels, centres, arrays)
        ctx.free("ph", h)
        ctx.free("ph", hp)
    ph = continuous_phantom(32, 32, 2, 3, seed=48)
    r = oc.cluster_phantom(ph, 1024)
    hp, h, m, labels, centres, arrays = gpu_cluster(mrsim, ctx, ph, 1024)
    check(r, m, labels, centres, arrays)
    ctx.free("ph", h)
    ctx.free("ph", hp)


def test_clustered_phantom_groups_and_signal(mrsim, ctx):
    """The clustered phantom has the group counts of its distinct keys, and its
    grouped simulation matches the oracle's simulation of the oracle's
    clustered phantom."""
    ph = configs.mapped_small(24, 24, 3)
    seq = spin_echo_2d(n_ro=24, n_pe=8, n_tr=2)
    r = oc.cluster_phantom(ph, 20)
    hp, h, m, labels, centres, arrays = gpu_cluster(mrsim, ctx, ph, 20)
    check(r, m, labels, centres, arrays)
    hs = ctx.sequence(seq)
    hg = ctx.group(h, hs)
    q = r.phantom
    for gtype, pos in ((mrsim.G_X, q.x), (mrsim.G_Z, q.z)):
        n_groups, _ = mrsim.mrsim_group_info(hg, gtype)
        assert n_groups == np.unique(np.stack([pos, q.T1, q.T2, q.dB0]), axis=1).shape[1]
    sig, _ = ctx.run(h, hs, hg, mrsim.GROUPED, mrsim.FP32)
    ref, _ = oracle.simulate(q, seq, memo=True, adc_recurrence=True, want_M=False)
    assert oracle.rel_l2(sig, ref) <= 1e-4


def test_cluster_errors(mrsim, ctx):
    ph = configs.mapped_small(8, 8, 1)
    hp = ctx.phantom(ph)
    bad = []
    for n, kw in ((0, {}), (mrsim.MAX_CLUSTERS + 1, {}), (4, dict(max_iter=0)),
                  (4, dict(scale=(64000.0, -1.0, 64.0))), (4, dict(te=(0.01,) * 17)),
                  (4, dict(te=(-0.01,))), (4, dict(te=(0.01,), tr=0.0))):
        with pytest.raises(mrsim.MrsimError) as e:
            mrsim.mrsim_cluster(ctx.h, hp, ph.K, n, **kw)
        bad.append(e.value.code)
    assert all(c == mrsim.EINVAL for c in bad)
    for field, value in (("T1", np.inf), ("T2", 1e-6), ("dB0", 3.0e4)):
        arr = getattr(ph, field).copy()
        arr[5] = value
        hq = ctx.phantom(dataclasses.replace(ph, **{field: arr}))
        with pytest.raises(mrsim.MrsimError) as e:
            mrsim.mrsim_cluster(ctx.h, hq, ph.K, 4)
        assert e.value.code == mrsim.EINVAL, field


def test_cluster_full_size(mrsim, ctx):
    """27,525,120 isochromats into 256 clusters, against the oracle's result
    stored by tests/golden/make_cluster_reference.py."""
    path = os.path.join(GOLDEN, "cluster_mapped_27m_oracle.npz")
    d = np.load(path)
    ph = configs.mapped_27m()
    assert str(d["phantom_digest"]) == phantom_digest(ph), "phantom differs from the stored one"
    hp, h, m, labels, centres, arrays = gpu_cluster(mrsim, ctx, ph, int(d["n_clusters"]))
    assert m == len(d["centres"])
    assert hashlib.sha256(np.ascontiguousarray(labels).tobytes()).hexdigest() == \
        str(d["labels_sha256"])
    assert np.array_equal(centres, d["centres"])
    assert np.array_equal(np.bincount(labels, minlength=m), d["sizes"])
    assert np.array_equal(arrays["T1"], centres[labels, 0].astype(np.float32))
    assert within_ulp(arrays["M0"][d["m0_index"]], d["m0"])
    ctx.free("ph", h)
    ctx.free("ph", hp)
