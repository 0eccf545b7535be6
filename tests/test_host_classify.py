"""The library's host-side sequence classifier (mrsim_classify: the part of
mrsim_sequence that needs no device) against the oracle's independent
classifier, bit for bit, on every workload of the repository (runs on CPU)."""

import ctypes

import numpy as np
import pytest

import oracle
from mrsim_inputs import configs
from mrsim_inputs.sequence import SeqBuilder, gre_2d, radial_2d, spin_echo_2d

from test_gpu_parity import general_type_sequence
from test_oracle_two_axis import spiral_like_sequence


@pytest.fixture(scope="module")
def mrsim():
    from paper_2508_03960_gb300 import build, mrsim as m
    build.build()
    return m


SEQUENCES = {
    "se_32": lambda: configs.se_32()[1],
    "fse_27m": configs.fse_sequence,
    "epi_27m": configs.epi_sequence,
    "gre": lambda: gre_2d(n_ro=16, n_pe=8),
    "se_small": lambda: spin_echo_2d(n_ro=16, n_pe=8, n_tr=2),
    "radial_oblique": lambda: radial_2d(n_ro=16, n_spokes=8, oblique_deg=20.0),
    "general_types": general_type_sequence,
    "spiral_like": spiral_like_sequence,
}


@pytest.mark.parametrize("two_axis", [False, True])
@pytest.mark.parametrize("name", list(SEQUENCES))
def test_classification_equals_oracle(mrsim, name, two_axis):
    seq = SEQUENCES[name]()
    got = mrsim.mrsim_classify(seq, mrsim.CLASSIFY_TWO_AXIS if two_axis else 0)
    ref = oracle.classify(seq, two_axis=two_axis)
    assert set(got) == set(ref)
    for k in ref:
        assert np.array_equal(got[k].astype(np.int64), ref[k].astype(np.int64)), k
    assert int(got["n_samples"].sum()) == seq.n_samples


def one_segment(**kw):
    b = SeqBuilder()
    b.add(10e-6, 4)
    fields = dict(dt=10e-6, repeat=2, b1=(0.0, 0.0), g=(0.0, 0.0, 0.0), adc=False)
    fields.update(kw)
    b.add(fields["dt"], fields["repeat"], b1=fields["b1"], g=fields["g"], adc=fields["adc"])
    return b.build()


def test_classification_errors(mrsim):
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_classify(one_segment(b1=(1e-6, 0.0), adc=True))
    assert e.value.code == mrsim.EUNSUPPORTED
    seq = one_segment()
    seq.dt[1] = 0.0
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_classify(seq)
    assert e.value.code == mrsim.EINVAL
    seq = one_segment(g=(np.nan, 0.0, 0.0))
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_classify(seq)
    assert e.value.code == mrsim.EINVAL


def test_small_capacity_reports_the_count_only(mrsim):
    seq = spin_echo_2d(n_ro=8, n_pe=4, n_tr=2)
    lib = mrsim.lib()
    arrs = [np.ascontiguousarray(seq.dt, np.float64), np.ascontiguousarray(seq.repeat, np.int32)]
    arrs += [np.ascontiguousarray(a, np.float32) for a in (seq.b1re, seq.b1im, seq.gx, seq.gy,
                                                           seq.gz)]
    arrs += [np.ascontiguousarray(seq.adc, np.uint8)]
    n = ctypes.c_int64(-1)
    typ = np.full(4, 99, np.uint8)
    rc = lib.mrsim_classify(seq.n_seg, *[a.ctypes.data for a in arrs], 0, 1, ctypes.byref(n),
                            typ.ctypes.data, None, None, None, None, None)
    assert rc == 0 and n.value == len(oracle.classify(seq)["type"]) > 1
    assert np.all(typ == 99)
    assert lib.mrsim_classify(seq.n_seg, *[a.ctypes.data for a in arrs], 0, 1, None,
                              *[None] * 6) == mrsim.EINVAL
    assert lib.mrsim_classify(seq.n_seg, *[a.ctypes.data for a in arrs], 2, 1, ctypes.byref(n),
                              *[None] * 6) == mrsim.EINVAL  # unknown flag
