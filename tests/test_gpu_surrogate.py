"""Learned with-RF transitions (surrogate): the GPU network against the FP64
reference network, training with the fallback gate, and what it gains.

Tolerances of the network check.  W2 is given in BF16-representable values,
so both sides use the same weights.  The forward pass feeds the tensor-core
layer h1 as hi + lo BF16 parts (~2^-17 relative); every contraction of the
backward pass (dh1, dW2 with db2, dW3, dW1 with db1, all on tcgen05 tensor
cores over a tile of 128 samples) takes single BF16 operands (unit roundoff
2^-9 ~ 2e-3 relative per operand), which, summed over up to 128 terms with
independent rounding, leaves ~5e-3 relative error in the gradients.  Bounds:
outputs and loss 1e-4 (rel-L2), gradients 3e-2 (rel-L2 over all 18,828
parameters) with cosine similarity > 0.999, every parameter block 5e-2.
"""

import time

import numpy as np
import pytest

import oracle
from oracle import mlp
from mrsim_inputs import configs
from mrsim_inputs.phantom import continuous_phantom

pytestmark = pytest.mark.gpu

DOMAIN_LO = [-0.010, -80.0, 0.8, 0.3, 0.04]
DOMAIN_HI = [0.010, 80.0, 1.2, 1.5, 0.2]


def bf16(a):
    b = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32)


@pytest.fixture(scope="module")
def ctx(mrsim):
    c = mrsim.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n", [1, 64, 128, 200, 300])
def test_network_forward_and_gradients_match_fp64_reference(mrsim, ctx, n):
    rng = np.random.default_rng(n)
    p = {k: rng.normal(0, 0.3, s) for k, s in mlp.SHAPES.items()}
    p["W2"] = bf16(p["W2"]).astype(np.float64)
    flat = mlp.pack(p).astype(np.float32)
    x = rng.uniform(-1, 1, (n, 5))
    t = rng.normal(0, 0.5, (n, 12))
    y, g, L = mrsim.mrsim_surrogate_eval(ctx.h, flat, x.astype(np.float32), t.astype(np.float32))
    x64 = x.astype(np.float32).astype(np.float64)
    t64 = t.astype(np.float32).astype(np.float64)
    y_ref, _ = mlp.forward(p, x64)
    L_ref, g_ref = mlp.loss_and_grad(p, x64, t64)
    gr = mlp.pack(g_ref)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 1e-4
    assert abs(L - L_ref) / L_ref < 1e-4
    assert np.linalg.norm(g - gr) / np.linalg.norm(gr) < 3e-2
    assert float(g @ gr) / (np.linalg.norm(g) * np.linalg.norm(gr)) > 0.999
    # every parameter block is exercised (a transposed operand would not match)
    o = 0
    for k in mlp.ORDER:
        m = int(np.prod(mlp.SHAPES[k]))
        gb, rb = g[o:o + m], gr[o:o + m]
        assert np.linalg.norm(gb - rb) / max(np.linalg.norm(rb), 1e-12) < 5e-2, k
        o += m


@pytest.mark.parametrize("n", [1, 127, 128, 300, 4096])
def test_tensor_core_inference_matches_fp64_reference(mrsim, ctx, n):
    """The tcgen05 inference kernel (layer 2 on the tensor cores with a TMEM
    accumulator; h1 as BF16 hi + lo) against the FP64 network of
    oracle/mlp.py with the same (BF16-representable) W2: ragged tiles of 128
    rows, one row, several tiles."""
    rng = np.random.default_rng(1000 + n)
    p = {k: rng.normal(0, 0.3, s) for k, s in mlp.SHAPES.items()}
    p["W2"] = bf16(p["W2"]).astype(np.float64)
    flat = mlp.pack(p).astype(np.float32)
    x = rng.uniform(-1, 1, (n, 5)).astype(np.float32)
    y = mrsim.mrsim_surrogate_infer(ctx.h, flat, x)
    y_ref, _ = mlp.forward(p, x.astype(np.float64))
    e = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    assert e < 1e-4, e
    assert np.max(np.abs(y - y_ref)) < 1e-3 * np.max(np.abs(y_ref))


@pytest.fixture(scope="module")
def trained(mrsim, ctx):
    _, seq = configs.surrogate_fse()
    hs = ctx.sequence(seq)
    t0 = time.time()
    sur = mrsim.mrsim_surrogate_train(ctx.h, hs, DOMAIN_LO, DOMAIN_HI, n_train=1 << 22,
                                      epochs=300, batch=8192, lr=1e-2, seed=1005, bound=1e-3)
    dt = time.time() - t0
    yield seq, hs, sur, dt
    mrsim.mrsim_free_surrogate(sur)


def test_training_converges_and_gate_bounds_served_error(mrsim, ctx, trained):
    seq, hs, sur, dt = trained
    st = mrsim.mrsim_surrogate_stats(sur)
    assert st["networks"] == 2  # the 90x and 180y slice-selective pulses
    assert st["train_loss"] < 1e-6
    assert st["cells_served"] > 0.05  # the gate serves a cell only at half the bound
    assert st["val_served_max_err"] <= 1e-3  # the gate's bound holds on validation draws


@pytest.mark.parametrize("shape", [(32, 32, 4), (128, 128, 16)])
def test_every_served_transition_of_a_run_is_within_the_bound(mrsim, ctx, trained, shape):
    """The gate bounds the error of each served group, not only of the
    validation draws: on the groups of real phantoms (per-isochromat dB0 and
    b1, the configuration's T1 / T2 regions) the transition the network
    serves differs from the exact FP64 one by at most the bound in every
    entry, for every served (group, pulse) pair."""
    seq, hs, sur, _ = trained
    ph = continuous_phantom(*shape, 3, seed=1005 + shape[0])
    hp = ctx.phantom(ph)
    hs2 = ctx.sequence(seq)
    hg = ctx.group(hp, hs2)
    err, served = mrsim.mrsim_surrogate_check(ctx.h, sur, hs2, hg)
    n_z = mrsim.mrsim_group_info(hg, mrsim.G_Z)[0]
    ctx.free("grp", hg)
    ctx.free("seq", hs2)
    ctx.free("ph", hp)
    print(f"served {served} of {2 * n_z} (group, pulse) pairs, largest entry error {err:.3e}")
    assert served > 0.1 * n_z
    assert err <= 1e-3, err


def test_surrogate_run_against_oracle_and_exact_grouped(mrsim, ctx, trained):
    seq, hs, sur, _ = trained
    ph, _ = configs.surrogate_fse()
    ref, Mref = oracle.simulate(ph, seq, memo=True, adc_recurrence=True)
    hp = ctx.phantom(ph)
    hs2 = ctx.sequence(seq)
    hg = ctx.group(hp, hs2)
    exact, _ = ctx.run(hp, hs2, hg, mrsim.GROUPED, mrsim.FP32)
    assert oracle.rel_l2(exact, ref) <= 1e-4
    mrsim.mrsim_surrogate_use(ctx.h, sur)
    s_sig, M = ctx.run(hp, hs2, hg, mrsim.SURROGATE, mrsim.FP32, K=ph.K, want_M=True)
    st = mrsim.mrsim_surrogate_stats(sur, ctx.h)
    mrsim.mrsim_surrogate_use(ctx.h, None)
    n_z = mrsim.mrsim_group_info(hg, mrsim.G_Z)[0]
    assert st["groups_served"] + st["groups_exact"] == 2 * n_z
    assert st["groups_served"] > 0
    # accepted transitions are within 1e-3 per entry: the signal stays close
    err = oracle.rel_l2(s_sig, ref)
    assert err <= 1e-2, err
    assert np.max(np.abs(M - Mref)) <= 2e-2


def test_surrogate_gain_over_exact_preparation(mrsim, ctx, trained):
    """Per-isochromat dB0 and b1 make almost every isochromat its own group, so
    the grouped method's preparation step (Eq. 7 per group) costs as much as
    plain stepping; the network replaces it."""
    seq, hs, sur, _ = trained
    ph = continuous_phantom(256, 256, 16, 3, seed=1005)
    hp = ctx.phantom(ph)
    hs2 = ctx.sequence(seq)
    hg = ctx.group(hp, hs2)
    import torch
    sig = np.zeros(2 * seq.n_samples)

    def timed(mode):
        mrsim.mrsim_run(ctx.h, hp, hs2, hg, mode, mrsim.FP32, sig)  # warm-up
        t0 = time.perf_counter()
        for _ in range(3):
            mrsim.mrsim_run(ctx.h, hp, hs2, hg, mode, mrsim.FP32, sig)
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) / 3
        # preparation-step kernels of one more run (CUDA events per launch)
        mrsim.mrsim_profile_reset(ctx.h)
        mrsim.mrsim_profile_enable(ctx.h, True)
        mrsim.mrsim_run(ctx.h, hp, hs2, hg, mode, mrsim.FP32, sig)
        prof = mrsim.mrsim_profile_get(ctx.h)
        mrsim.mrsim_profile_enable(ctx.h, False)
        prep = sum(v[1] for k, v in prof.items() if k in ("precompute_f32", "sur_gate", "sur_infer"))
        return t, prep, sig.view(np.complex128).copy()

    t_exact, p_exact, s_exact = timed(mrsim.GROUPED)
    mrsim.mrsim_surrogate_use(ctx.h, sur)
    t_sur, p_sur, s_sur = timed(mrsim.SURROGATE)
    st = mrsim.mrsim_surrogate_stats(sur, ctx.h)
    mrsim.mrsim_surrogate_use(ctx.h, None)
    served = st["groups_served"] / (st["groups_served"] + st["groups_exact"])
    assert served > 0.1
    print(f"exact {t_exact * 1e3:.1f} ms (preparation {p_exact:.1f} ms), surrogate "
          f"{t_sur * 1e3:.1f} ms (preparation {p_sur:.1f} ms), served {served:.3f}")
    # the preparation step shrinks with the served fraction, and so does the run
    assert p_sur < p_exact, (p_sur, p_exact, served)
    assert t_sur < t_exact, (t_sur, t_exact, served)
    assert oracle.rel_l2(s_sur, s_exact) <= 1e-2
