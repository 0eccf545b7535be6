"""Cartesian image reconstruction (mrsim_recon_cartesian) against the oracle's
(numpy FFT) reconstruction: random k-space through the SE, FSE and EPI
layouts (FP64 both sides: rel-L2 1e-12), host and device pointers, and the
image of a grouped FP32 simulation against the image of the oracle's signal
(the FP32 signal tolerance, 1e-4, carries over by linearity)."""

import numpy as np
import pytest

import oracle
from oracle.recon import recon_cartesian
from mrsim_inputs import configs
from mrsim_inputs.sequence import epi_2d, fse_2d, kspace_layout, spin_echo_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(mrsim):
    c = mrsim.Context(0)
    yield c
    c.close()


def layouts():
    out = [kspace_layout(spin_echo_2d(n_ro=16, n_pe=16)),
           kspace_layout(fse_2d(n_ro=32, n_pe=32, etl=8)),
           kspace_layout(epi_2d(n_ro=16, n_lines=12))]
    # a non-square layout with repeated and missing rows and both directions
    rng = np.random.default_rng(3)
    out.append(dict(n_ro=24, n_pe=10, row=rng.integers(0, 10, 14).astype(np.int32),
                    col0=rng.integers(0, 24, 14).astype(np.int32),
                    dir=np.where(rng.random(14) < 0.5, 1, -1).astype(np.int8)))
    return out


@pytest.mark.parametrize("which", range(4))
def test_recon_matches_oracle(mrsim, ctx, which):
    L = layouts()[which]
    rng = np.random.default_rng(10 + which)
    n = len(L["row"]) * L["n_ro"]
    sig = rng.normal(size=n) + 1j * rng.normal(size=n)
    ref = recon_cartesian(sig, L)
    img = mrsim.mrsim_recon_cartesian(ctx.h, sig, L)
    assert oracle.rel_l2(img, ref) <= 1e-12


def test_recon_device_pointers(mrsim, ctx):
    import torch
    L = layouts()[1]
    rng = np.random.default_rng(21)
    n = len(L["row"]) * L["n_ro"]
    sig = rng.normal(size=n) + 1j * rng.normal(size=n)
    d_sig = torch.from_numpy(sig.view(np.float64).copy()).cuda()
    d_img = torch.zeros(2 * L["n_pe"] * L["n_ro"], dtype=torch.float64, device="cuda")
    mrsim.mrsim_recon_cartesian(ctx.h, d_sig, L, d_img, mrsim.PTR_DEVICE)
    img = d_img.cpu().numpy().view(np.complex128).reshape(L["n_pe"], L["n_ro"])
    assert oracle.rel_l2(img, recon_cartesian(sig, L)) <= 1e-12


def test_image_of_grouped_simulation(mrsim, ctx):
    ph = configs.small_phantom(32, 32, 4)
    seq = fse_2d(n_ro=32, n_pe=32, etl=8, rf_dur=2e-3, rf_dt=10e-6, dwell=10e-6, esp=10e-3,
                 tr=1.0)
    L = kspace_layout(seq)
    ref, _ = oracle.simulate(ph, seq, memo=True, adc_recurrence=True, want_M=False)
    hp = ctx.phantom(ph)
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    sig, _ = ctx.run(hp, hs, hg, mrsim.GROUPED, mrsim.FP32)
    img = mrsim.mrsim_recon_cartesian(ctx.h, sig, L)
    assert oracle.rel_l2(img, recon_cartesian(ref, L)) <= 1e-4


def test_recon_errors(mrsim, ctx):
    L = dict(layouts()[0])
    sig = np.zeros(len(L["row"]) * L["n_ro"], np.complex128)
    bad = dict(L, n_ro=15)
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_recon_cartesian(ctx.h, np.zeros(len(L["row"]) * 15, np.complex128), bad)
    assert e.value.code == mrsim.EINVAL
    bad = dict(L, row=np.where(np.arange(len(L["row"])) == 3, L["n_pe"], L["row"]).astype(np.int32))
    with pytest.raises(mrsim.MrsimError) as e:
        mrsim.mrsim_recon_cartesian(ctx.h, sig, bad)
    assert e.value.code == mrsim.EINVAL
