"""GPU large/small-scale merge (Sec. 2.4, Eqs. 4-5) against the oracle.

gg_large_scales (Eq. 5 with the cloud-in-cell deconvolution) and
gg_zeldovich_merge (Eq. 4 on the fine displacement plus the interpolated
coarse large scales, then Eq. 3): FP64 within 1e-12 of the oracle, FP32
within 1e-5 relative L2; grid ratios 2 (size-specialised kernels) and 3/2
(run-time kernels); the whole chain coarse psi -> large scales -> merge; a
cut below the fundamental mode gives back gg_zeldovich bit for bit; and
512^3 FP32 against the FP64 path.
"""
import math

import numpy as np
import pytest

from oracle import fields as ofields
from oracle import merge as omerge
from oracle import noise as onoise
from tests.gpu_helpers import min_image, rel_l2
from tests.oracle_cases import cosmology_from

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BBKS = dict(omega_m=0.3, h=0.7, n_s=0.96, sigma_8=0.8, tf="bbks", omega_l=-1.0,
            omega_b=0.049, t_cmb=2.7255)
C = cosmology_from(BBKS)
Z = 30.0


@pytest.fixture(scope="module")
def gg():
    from paper_2511_10353_gb300 import build
    build.build(verbose=False)
    import paper_2511_10353_gb300 as m
    return m


def _dt(prec):
    return torch.float64 if prec == "f64" else torch.float32


def _close(got, want, prec, what=""):
    got = np.asarray(got, dtype=np.float64)
    if prec == "f64":
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), what
    else:
        assert rel_l2(got, want) < 1e-5, what


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,cells", [(16, 2.0), (16, 0.5), (24, 1.0), (64, 2.0), (64, 0.25)])
def test_large_scales_matches_oracle(gg, n, cells, prec):
    box = 2.0 * n
    r_s = cells * box / n
    f = onoise.white_noise(9, n)
    plan = gg.Plan(n, box, BBKS, Z, prec)
    got = plan.large_scales(torch.tensor(f, dtype=_dt(prec), device="cuda"), r_s).cpu().numpy()
    plan.close()
    _close(got, omerge.large_scales(f, box, r_s), prec)


def _check_zeldovich(out, want, box, prec):
    for j in range(3):
        _close(out["psi"][j].cpu().numpy(), want["psi"][j], prec, "psi%d" % j)
        _close(out["vel"][j].cpu().numpy(), want["vel"][j], prec, "vel%d" % j)
        pos = out["pos"][j].cpu().numpy().astype(np.float64)
        assert pos.min() >= 0.0 and pos.max() < box
        d = min_image(pos - want["pos"][j], box)
        psi_max = np.abs(want["psi"][j]).max()
        if prec == "f64":
            assert np.abs(d).max() < 1e-12 * max(1.0, psi_max) + 4e-16 * box, j
        else:  # FP32 rounding of a coordinate near L plus the psi error
            assert np.abs(d).max() < 4 * np.spacing(np.float32(box)) + 1e-5 * psi_max, j


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nh,nl", [(32, 16), (24, 16), (64, 32)])
def test_merge_matches_oracle(gg, nh, nl, prec):
    box = 64.0
    r_s = 2 * box / nl
    coarse = ofields.zeldovich(nl, box, C, Z, seed=3)
    large = [omerge.large_scales(coarse["psi"][j], box, r_s) for j in range(3)]
    noise = onoise.white_noise(4, nh)
    want = omerge.merged_zeldovich(nh, box, C, Z, large, r_s, noise=noise)
    plan = gg.Plan(nh, box, BBKS, Z, prec)
    out = plan.zeldovich_merge([torch.tensor(g, dtype=_dt(prec), device="cuda") for g in large], r_s,
                               noise=torch.tensor(noise, dtype=_dt(prec), device="cuda"))
    plan.sync()
    plan.close()
    _check_zeldovich(out, want, box, prec)


def test_whole_chain_fp64(gg):
    """coarse psi (GPU) -> large scales (GPU) -> merge (GPU) against the oracle chain."""
    nh, nl, box = 32, 16, 48.0
    r_s = 2 * box / nl
    lo = gg.Plan(nl, box, BBKS, Z, "f64")
    psi_lo = lo.zeldovich(seed=5, pos=False, vel=False)["psi"]
    large = [lo.large_scales(psi_lo[j], r_s) for j in range(3)]
    hi = gg.Plan(nh, box, BBKS, Z, "f64")
    out = hi.zeldovich_merge(large, r_s, seed=6)
    hi.sync()
    coarse = ofields.zeldovich(nl, box, C, Z, seed=5)
    olarge = [omerge.large_scales(coarse["psi"][j], box, r_s) for j in range(3)]
    want = omerge.merged_zeldovich(nh, box, C, Z, olarge, r_s, seed=6)
    _check_zeldovich(out, want, box, "f64")
    lo.close()
    hi.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cut_below_fundamental_is_plain_zeldovich(gg, prec):
    n, box = 32, 50.0
    plan = gg.Plan(n, box, BBKS, Z, prec)
    ref = plan.zeldovich(seed=2)
    plan.sync()
    got = plan.zeldovich_merge([None, None, None], r_s=10 * box, seed=2)  # keeps every mode
    plan.sync()
    for k in ("psi", "pos", "vel"):
        for j in range(3):
            assert torch.equal(got[k][j], ref[k][j]), (k, j)
    plan.close()


def test_merge_512_fp32_against_fp64(gg):
    nh, nl, box = 512, 256, 500.0
    r_s = 2 * box / nl
    rng = torch.Generator(device="cuda").manual_seed(0)
    large64 = [torch.randn((nl, nl, nl), generator=rng, device="cuda", dtype=torch.float64) * 0.3
               for _ in range(3)]
    p64 = gg.Plan(nh, box, BBKS, 100.0, "f64")
    o64 = p64.zeldovich_merge(large64, r_s, seed=1, pos=False, vel=False)
    p64.sync()
    p64.close()
    p32 = gg.Plan(nh, box, BBKS, 100.0, "f32")
    o32 = p32.zeldovich_merge([g.float() for g in large64], r_s, seed=1, pos=False, vel=False)
    p32.sync()
    p32.close()
    for j in range(3):
        a, b = o32["psi"][j].double(), o64["psi"][j]
        assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) < 1e-5
