"""Batched launcher: uneven (phantom, sequence) jobs in one CUDA-graph launch
chain with persistent fused kernels.  Every job's signal must equal its own
grouped run and the FP64 oracle within the FP32 tolerance (signal rel-L2
1e-4): jobs of known gradient types, and jobs with subsequences without a
type (the per-isochromat fallback kernels inside the graph), a given initial
state, about one group per isochromat (direct advances) and receive coils.

Batched vs single run: the same formulas, but the batched preparation composes
each pulse's sub-steps with a CTA-wide tree while a single run may split them
over fewer lanes, and FP32 block sums are added in another order; the FP32
transitions then differ by ~1e-7 and the signals by up to ~1e-6 (cancellation
in the k-space sum).  Bound: rel-L2 1e-5, ten times the largest seen."""

import dataclasses

import numpy as np
import pytest

import oracle
from mrsim_inputs import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(mrsim):
    c = mrsim.Context(0)
    yield c
    c.close()


def jobs():
    sizes = [4096, 9000, 23000, 3000, 61000, 14000]
    out = []
    for i, K in enumerate(sizes):
        ph, seq = configs.batch_job(i, K)
        out.append((ph, seq))
    return out


def test_batch_matches_single_runs_and_oracle(mrsim, ctx):
    js = jobs()
    hps, hss, hgs, sigs, singles = [], [], [], [], []
    for ph, seq in js:
        hp = ctx.phantom(ph)
        hs = ctx.sequence(seq)
        hg = ctx.group(hp, hs)
        hps.append(hp); hss.append(hs); hgs.append(hg)
        sigs.append(np.zeros(2 * seq.n_samples))
        singles.append(ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32)[0])
    for rep in range(2):  # the second call relaunches the cached graph
        for s in sigs:
            s[:] = np.nan
        mrsim.mrsim_run_batch(ctx.h, hps, hss, hgs, sigs)
        for (ph, seq), s, one in zip(js, sigs, singles):
            b = s.view(np.complex128)
            assert oracle.rel_l2(b, one) <= 1e-5
    for (ph, seq), s in zip(js, sigs):
        ref, _ = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
        assert oracle.rel_l2(s.view(np.complex128), ref) <= 1e-4


def general_job_sequence():
    """A with-RF subsequence and a with-ADC window with gradients on all three
    axes (neither has a type), between subsequences of known types."""
    from mrsim_inputs import SeqBuilder
    b = SeqBuilder()
    b.rf_sinc(90, "x", 1e-3, 10e-6, 4.0, 0.01)
    b.add(1e-3, 1, g=(2e-3, 1e-3, -3e-3))
    for _ in range(40):                                   # RF with Gx, Gy and Gz
        b.add(10e-6, 1, b1=(2e-6, 0.5e-6), g=(1e-3, 0.5e-3, 2e-3))
    b.add(2e-3, 1, g=(0, 1e-3, 0))
    b.add(10e-6, 16, g=(5e-3, 2e-3, 1e-3), adc=True)      # ADC on three axes
    b.add(1e-3, 1)
    b.add(10e-6, 16, g=(5e-3, 0, 0), adc=True)            # Gx-only
    b.rf_hard(30, "y", 100e-6, 10e-6)
    b.add(10e-6, 8, adc=True)                             # no-grads ADC
    b.add(5e-3, 1)
    return b.build()


def widened_jobs():
    """(name, phantom, sequence) of every kind the launcher takes beyond the
    known-type jobs above, and one job that combines them."""
    from mrsim_inputs import coil_maps
    from mrsim_inputs.phantom import continuous_phantom
    from mrsim_inputs.sequence import spin_echo_2d
    gen = general_job_sequence()
    se = spin_echo_2d(n_ro=32, n_pe=16, n_tr=2)
    base, fse = configs.batch_job(2, 9000)
    K = base.K
    rng = np.random.default_rng(77)
    Mi = np.stack([rng.uniform(-0.3, 0.3, K), rng.uniform(-0.3, 0.3, K),
                   rng.uniform(0.2, 1.0, K)]).astype(np.float32) * base.M0
    with_init = dataclasses.replace(base, M_init=np.ascontiguousarray(Mi))
    direct = continuous_phantom(24, 24, 4, 2, seed=33)
    plain = configs.batch_job(0, 4096)[0]
    coils = dataclasses.replace(plain, coils=coil_maps(plain, 3, seed=9))
    both = dataclasses.replace(with_init, coils=coil_maps(with_init, 2, seed=10))
    return [("general", configs.batch_job(1, 6000)[0], gen),
            ("initial_state", with_init, fse),
            ("direct", direct, se),
            ("coils", coils, se),
            ("general_init_coils", both, gen),
            ("plain_known", configs.batch_job(3, 3000)[0], configs.batch_job(3, 3000)[1])]


def test_batch_widened_jobs(mrsim, ctx):
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, 0)
    try:
        js = widened_jobs()
        hps, hss, hgs, sigs, singles, P = [], [], [], [], [], []
        for name, ph, seq in js:
            hp = ctx.phantom(ph)
            hs = ctx.sequence(seq)
            hg = ctx.group(hp, hs)
            hps.append(hp); hss.append(hs); hgs.append(hg)
            n_coils = 0 if ph.coils is None else ph.coils.shape[0]
            P.append(n_coils)
            sigs.append(np.zeros(2 * seq.n_samples * max(n_coils, 1)))
            singles.append(ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32)[0])
        info = [mrsim.mrsim_seq_info(h) for h in hss]
        assert any(4 in list(i["gtype"]) for i in info)  # a subsequence without a type
        for rep in range(2):  # the second call relaunches the cached graph
            for s in sigs:
                s[:] = np.nan
            mrsim.mrsim_run_batch(ctx.h, hps, hss, hgs, sigs)
            for (name, ph, seq), s, one, n_coils in zip(js, sigs, singles, P):
                b = s.view(np.complex128)
                if n_coils:
                    b = b.reshape(n_coils, seq.n_samples)
                assert oracle.rel_l2(b.ravel(), np.asarray(one).ravel()) <= 1e-5, name
        for (name, ph, seq), s, n_coils in zip(js, sigs, P):
            ref, _ = oracle.simulate(ph, seq, memo=True, want_M=False)
            b = s.view(np.complex128)
            if n_coils:
                b = b.reshape(n_coils, seq.n_samples)
                for j in range(n_coils):
                    assert oracle.rel_l2(b[j], ref[j]) <= 1e-4, (name, j)
            else:
                assert oracle.rel_l2(b, ref) <= 1e-4, name
    finally:
        mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, 1)


def test_batch_errors(mrsim, ctx):
    ph, seq = configs.batch_job(0, 4096)
    ph2, _ = configs.batch_job(1, 4096)
    hp, hp2 = ctx.phantom(ph), ctx.phantom(ph2)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    sig = np.zeros(2 * seq.n_samples)
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_run_batch(ctx.h, [hp2], [hs], [hg], [sig])
    assert e.value.code == mrsim.ESTATE
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_run_batch(ctx.h, [], [], [], [])
    assert e.value.code == mrsim.EINVAL
