"""GPU power spectrum and moments (Sec. 2.1 diagnostics) against the oracle.

Shell counts exact; FP64 shell powers and mean |k| within 1e-12, FP32 within
1e-5 (relative); moments likewise. At 512^3 (FP32) the measured power of the
path's own Eq. 1 density field follows the input spectrum: in every shell
from b = 4 on, P / <D^2 P(k)>_shell is 1 within five standard deviations of
its sampling error sqrt(2 / count).
"""
import math

import numpy as np
import pytest

from oracle import noise as onoise
from oracle import stats as ostats

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BBKS = dict(omega_m=0.3, h=0.7, n_s=0.96, sigma_8=0.8, tf="bbks", omega_l=-1.0,
            omega_b=0.049, t_cmb=2.7255)


@pytest.fixture(scope="module")
def gg():
    from paper_2511_10353_gb300 import build
    build.build(verbose=False)
    import paper_2511_10353_gb300 as m
    return m


def _dt(prec):
    return torch.float64 if prec == "f64" else torch.float32


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,nbins", [(16, 8), (24, 12), (64, 32), (64, 5)])
def test_power_spectrum_matches_oracle(gg, n, nbins, prec):
    box = 3.0 * n
    f = onoise.white_noise(13, n) * 0.5 + 0.25
    plan = gg.Plan(n, box, BBKS, 20.0, prec)
    k, p, c = plan.power_spectrum(torch.tensor(f, dtype=_dt(prec), device="cuda"), nbins)
    plan.close()
    kw, pw, cw = ostats.power_spectrum(f, box, nbins)
    assert np.array_equal(c, cw)
    tol = 1e-12 if prec == "f64" else 1e-5
    assert np.abs(k - kw).max() <= tol * kw.max()
    assert np.all(np.abs(p - pw) <= tol * np.abs(pw) + 1e-300)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_moments_match_oracle(gg, prec):
    n = 48
    f = onoise.white_noise(2, n) * 1.5 - 0.2
    plan = gg.Plan(n, 100.0, BBKS, 20.0, prec)
    got = plan.moments(torch.tensor(f, dtype=_dt(prec), device="cuda"))
    plan.close()
    fr = f.astype(np.float32).astype(np.float64) if prec == "f32" else f
    want = ostats.moments(fr)
    tol = 1e-12 if prec == "f64" else 1e-9
    assert abs(got[0] - want[0]) < tol * (1 + abs(want[0]))
    assert abs(got[1] - want[1]) < tol * want[1]
    assert got[2] == want[2] and got[3] == want[3]


def test_512_density_follows_input_spectrum(gg):
    n, box, z = 512, 500.0, 100.0
    plan = gg.Plan(n, box, BBKS, z, "f32")
    delta = plan.gaussian_field(seed=1)
    k, p, c = plan.power_spectrum(delta)
    mom = plan.moments(delta)
    plan.close()
    # expected shell averages of D^2 P(k) = V S(m2)^2 from the library's FP64
    # filter table S(m2) = D sqrt(P/V) (pinned against the oracle on the host)
    s = gg.filter_table(n, box, BBKS, z, 3 * (n // 2) ** 2 + 1)
    st = torch.tensor(s, dtype=torch.float64, device="cuda")
    half = n // 2
    m = torch.arange(n, device="cuda")
    m = torch.where(m < half, m, m - n)
    mz = torch.arange(half, device="cuda")
    expect = torch.zeros(half, dtype=torch.float64, device="cuda")
    count = torch.zeros(half, dtype=torch.float64, device="cuda")
    for x in range(n):  # plane by plane: modes with |m_j| = N/2 left out
        mx = int(m[x])
        if abs(mx) == half:
            continue
        my = m[:, None]
        m2 = mx * mx + my * my + mz[None, :] ** 2
        b = torch.floor(torch.sqrt(m2.double()) + 0.5).long()
        ok = (my.abs() != half).expand_as(m2) & (b < half)
        w = torch.where(mz[None, :] == 0, 1.0, 2.0).double().expand_as(m2)
        val = box ** 3 * st[m2] ** 2
        expect.index_add_(0, b[ok], (w * val)[ok])
        count.index_add_(0, b[ok], w[ok])
    expect = (expect / count.clamp(min=1)).cpu().numpy()
    assert np.array_equal(c, count.cpu().numpy().astype(np.int64))
    for sh in range(4, half):
        assert abs(p[sh] / expect[sh] - 1) < 5 * math.sqrt(2.0 / c[sh]), sh
    # the Eq. 1 field has zero mean (k = 0 dropped) and variance sum_k P / V
    assert abs(mom[0]) < 1e-6 * math.sqrt(mom[1])
