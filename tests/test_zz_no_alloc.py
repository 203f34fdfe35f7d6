"""The no-allocation density entry point, gg_gaussian_field_static.

Some callers cannot call cudaMalloc (their device memory belongs to their own
pool allocator, or they must not take cudaMalloc's implicit synchronisation).
gg_gaussian_field_static serves them for grids up to GG_STATIC_MAX_N^3 from
arrays that live in the library's device image. This test calls it through
the C ABI, twice in a row, and compares each result with the density field
of the plan-based gg_gaussian_field on the same seed (FP64 within 1e-12,
FP32 within 1e-5 relative L2, the tolerances of the other parity tests).
It lives in a file that pytest collects last and must pass on its own in a
fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BBKS = dict(omega_m=0.3, h=0.7, n_s=0.96, sigma_8=0.8, tf="bbks", omega_l=-1.0,
            omega_b=0.049, t_cmb=2.7255)
MAX_N = 64


@pytest.fixture(scope="module")
def gg():
    from paper_2511_10353_gb300 import build
    build.build(verbose=False)
    import paper_2511_10353_gb300 as m
    f = m.lib().gg_gaussian_field_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(m.Params), ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    return m


def _static(gg, n, box, z, prec, seed, noise=None):
    p, _keep = gg.make_params(n, box, BBKS, z, prec)
    dt = torch.float64 if prec == "f64" else torch.float32
    out = torch.full((n, n, n), float("nan"), dtype=dt, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = gg.lib().gg_gaussian_field_static(ctypes.byref(p), seed,
                                           None if noise is None else noise.data_ptr(),
                                           out.data_ptr(), stream)
    assert st == gg.GG_OK, gg.lib().gg_last_error(None)
    return out


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,prec", [(64, "f32"), (64, "f64"), (48, "f32"), (32, "f64")])
def test_matches_plan_on_two_calls_in_a_row(gg, n, prec):
    box, z = 1.5 * n, 30.0
    tol = 1e-12 if prec == "f64" else 1e-5
    plan = gg.Plan(n, box, BBKS, z, prec)
    for seed in (11, 12):
        want = plan.gaussian_field(seed=seed)
        plan.sync()
        got = _static(gg, n, box, z, prec, seed)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert _rel(got, want) < tol, (n, prec, seed)
    plan.close()


def test_caller_noise(gg):
    n = 32
    plan = gg.Plan(n, 40.0, BBKS, 10.0, "f64")
    noise = torch.randn((n, n, n), dtype=torch.float64, device="cuda")
    want = plan.gaussian_field(noise=noise)
    plan.sync()
    for _ in range(2):
        got = _static(gg, n, 40.0, 10.0, "f64", 0, noise=noise)
        assert _rel(got, want) < 1e-12


def test_rejects_grids_beyond_the_limit(gg):
    p, _keep = gg.make_params(2 * MAX_N, 100.0, BBKS, 10.0, "f32")
    out = torch.empty(8, device="cuda")
    st = gg.lib().gg_gaussian_field_static(ctypes.byref(p), 1, None, out.data_ptr(), None)
    assert st == gg.GG_EINVAL
    assert b"static scratch limit" in gg.lib().gg_last_error(None)
