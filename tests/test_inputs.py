"""The seeded input generators (no method arithmetic): the stored full-size
oracle signals stay tied to the inputs the generators produce today, coil maps
and k-space layouts are deterministic and well formed."""

import os

import numpy as np

from mrsim_inputs import coil_maps, configs, phantom_digest, sequence_digest
from mrsim_inputs.phantom import log_candidates, mapped_phantom
from mrsim_inputs.sequence import epi_2d, fse_2d, kspace_layout, spin_echo_2d

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_generators_reproduce_the_stored_full_size_inputs():
    ph = configs.full_phantom()
    pd = phantom_digest(ph)
    for name, seq in (("fse", configs.fse_sequence()), ("epi", configs.epi_sequence())):
        d = np.load(os.path.join(GOLDEN, f"{name}_27m_oracle.npz"))
        assert str(d["phantom_digest"]) == pd
        assert str(d["sequence_digest"]) == sequence_digest(seq)


def test_coil_maps_are_seeded_and_bounded():
    ph = configs.small_phantom(16, 16, 2)
    a, b, c = coil_maps(ph, 4, seed=9), coil_maps(ph, 4, seed=9), coil_maps(ph, 4, seed=10)
    assert a.shape == (4, 2, ph.K) and a.dtype == np.float32
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    mag = np.hypot(a[:, 0], a[:, 1])
    assert np.all(mag > 0) and np.all(mag <= 1.0)


def test_kspace_layouts_cover_the_grid_once():
    for seq in (spin_echo_2d(n_ro=16, n_pe=16), fse_2d(n_ro=32, n_pe=32, etl=8),
                epi_2d(n_ro=16, n_lines=16)):
        L = kspace_layout(seq)
        assert len(L["row"]) * L["n_ro"] == seq.n_samples
        hits = np.zeros((L["n_pe"], L["n_ro"]), int)
        i = np.arange(L["n_ro"])
        for a in range(len(L["row"])):
            hits[L["row"][a], (L["col0"][a] + L["dir"][a] * i) % L["n_ro"]] += 1
        assert np.all(hits == 1)


def test_mapped_phantom_takes_values_from_the_candidate_sets():
    """T1 and T2 of the parameter-mapping stand-in are log-spaced candidates
    (constant ratio, end points 10-3000 ms and 10-500 ms), dB0 = 0, seeded."""
    c1 = log_candidates(0.010, 3.0, 100)
    ratio = c1[1:] / c1[:-1]
    assert c1[0] == 0.010 and c1[-1] == 3.0
    assert np.max(np.abs(ratio / ratio[0] - 1.0)) < 1e-12
    assert abs(ratio[0] ** 99 - 300.0) < 1e-9
    p, q = mapped_phantom(32, 32, 2, 6, seed=21), mapped_phantom(32, 32, 2, 6, seed=21)
    assert phantom_digest(p) == phantom_digest(q)
    c2 = log_candidates(0.010, 0.5, 100)
    assert np.isin(p.T1, c1.astype(np.float32)).all()
    assert np.isin(p.T2, c2.astype(np.float32)).all()
    assert not p.dB0.any() and p.K == 32 * 32 * 2
    n_pairs = np.unique(np.stack([p.T1, p.T2]), axis=1).shape[1]
    assert 50 < n_pairs < 100 * 100


def test_generator_reproduces_the_stored_clustering_input():
    d = np.load(os.path.join(GOLDEN, "cluster_mapped_27m_oracle.npz"))
    assert str(d["phantom_digest"]) == phantom_digest(configs.mapped_27m())
