"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: the FP64 path within 1e-12 relative L2 of the oracle (the
rounding of two 3-D transforms is ~1e-15); the FP32 path within 1e-5
relative L2 on displacements and velocities. FP32 positions carry the FP32
rounding of q + psi, i.e. up to ulp(L): they are compared as minimum-image
differences within 4 ulp(L) + 1e-5 max|psi|. Philox words are bit-exact.
"""
import math

import numpy as np
import pytest

from oracle import noise as onoise
from tests.gpu_helpers import min_image, rel_l2, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BBKS = dict(omega_m=0.3, h=0.7, n_s=0.96, sigma_8=0.8, tf="bbks", omega_l=-1.0,
            omega_b=0.049, t_cmb=2.7255)
EH_NW = dict(omega_m=0.31, h=0.68, n_s=0.965, sigma_8=0.81, tf="eh_nw", omega_l=-1.0,
             omega_b=0.049, t_cmb=2.7255)


@pytest.fixture(scope="module")
def gg():
    from paper_2511_10353_gb300 import build
    build.build(verbose=False)
    import paper_2511_10353_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return m


def _np(t):
    return t.detach().cpu().numpy()


def _compare(gpu, ora, box, prec, comps=(0, 1, 2), keys=("psi", "pos", "vel")):
    tol = 1e-12 if prec == "f64" else 1e-5
    for j in comps:
        psi_o = ora["psi"][j]
        if "psi" in keys and gpu["psi"][j] is not None:
            assert rel_l2(_np(gpu["psi"][j]), psi_o) < tol, ("psi", j)
        if "vel" in keys and gpu["vel"][j] is not None:
            assert rel_l2(_np(gpu["vel"][j]), ora["vel"][j]) < tol, ("vel", j)
        if "pos" in keys and gpu["pos"][j] is not None:
            pos = _np(gpu["pos"][j]).astype(np.float64)
            assert pos.min() >= 0.0 and pos.max() < box
            d = min_image(pos - ora["pos"][j], box)
            if prec == "f64":
                assert np.abs(d).max() < 1e-12 * max(1.0, np.abs(psi_o).max()) + 4e-16 * box
            else:
                ulp = np.spacing(np.float32(box))
                assert np.abs(d).max() < 4 * ulp + 1e-5 * np.abs(psi_o).max(), ("pos", j)


def test_noise_bits_bit_exact(gg):
    for first, count in ((0, 1 << 16), (2**32 - 7, 20), (12345678901, 1000)):
        for seed in (1, 48, 2**40 + 3):
            got = _np(gg.noise_bits(seed, first, count)).view(np.uint32)
            want = onoise.noise_bits(seed, np.arange(first, first + count, dtype=np.uint64))
            assert np.array_equal(got, want), (seed, first)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [6, 16, 18, 64])
def test_white_noise_values(gg, prec, n):
    plan = gg.Plan(n, 10.0, BBKS, 10.0, prec)
    w = _np(plan.white_noise(seed=7)).astype(np.float64)
    want = onoise.white_noise(7, n)
    if prec == "f64":
        assert np.abs(w - want).max() < 1e-14 * max(1.0, np.abs(want).max())
    else:
        assert rel_l2(w, want) < 1e-6 and np.abs(w - want).max() < 1e-3


@pytest.mark.parametrize("n", [4, 6, 8, 12, 16, 18, 24, 36, 48, 64, 96])
def test_zeldovich_fp64_matches_oracle(gg, n):
    w = dict(n=n, box=100.0 * n / 64, cosmo=BBKS, z_init=50.0)
    plan = gg.Plan(n, w["box"], BBKS, 50.0, "f64")
    out = plan.zeldovich(seed=1)
    torch.cuda.synchronize()
    plan.sync()
    _compare(out, run_oracle(w, seed=1), w["box"], "f64")


def test_config_64_fp64(gg):
    """Plain method, FP64: 64^3, L = 100 Mpc/h, BBKS, z = 50, seed 1."""
    w = dict(n=64, box=100.0, cosmo=BBKS, z_init=50.0)
    plan = gg.Plan(64, 100.0, BBKS, 50.0, "f64")
    out = plan.zeldovich(seed=1)
    plan.sync()
    _compare(out, run_oracle(w, seed=1), 100.0, "f64")


@pytest.mark.parametrize("n", [16, 48, 64, 128, 192])
def test_zeldovich_fp32_matches_oracle(gg, n):
    w = dict(n=n, box=float(n), cosmo=BBKS, z_init=50.0)
    plan = gg.Plan(n, w["box"], BBKS, 50.0, "f32")
    out = plan.zeldovich(seed=3)
    plan.sync()
    _compare(out, run_oracle(w, seed=3), w["box"], "f32")


@pytest.mark.parametrize("n,prec", [(256, "f32"), (384, "f32"), (384, "f64")])
def test_batched_workload_sizes_match_oracle(gg, n, prec):
    """The size-specialised codelets of the batched workload's larger grids
    (N = 256: radix 8.8.4; N = 384: 8.8.2.3 with 24 elements a thread and
    register stage pairs) against the oracle on Philox noise, with that
    workload's cell size (L = N Mpc/h) and z = 50, in the autotuner's
    variants and in variant 0."""
    w = dict(n=n, box=float(n), cosmo=BBKS, z_init=50.0)
    ora = run_oracle(w, seed=5)
    plan = gg.Plan(n, w["box"], BBKS, 50.0, prec)
    for tune in (False, True):
        if tune:
            plan.autotune(1)
        out = plan.zeldovich(seed=5)
        plan.sync()
        _compare(out, ora, w["box"], prec)
        del out
    plan.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_caller_noise_and_eh(gg, prec):
    n = 32
    w = dict(n=n, box=2000.0 * n / 1536, cosmo=EH_NW, z_init=100.0)
    grid = np.random.default_rng(5).standard_normal((n, n, n))
    dt = torch.float64 if prec == "f64" else torch.float32
    plan = gg.Plan(n, w["box"], EH_NW, 100.0, prec)
    out = plan.zeldovich(noise=torch.tensor(grid, dtype=dt, device="cuda"))
    plan.sync()
    ora = run_oracle(w, noise_grid=grid.astype(np.float32).astype(np.float64) if prec == "f32" else grid)
    _compare(out, ora, w["box"], prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gaussian_field(gg, prec):
    n = 48
    w = dict(n=n, box=75.0, cosmo=BBKS, z_init=20.0)
    plan = gg.Plan(n, 75.0, BBKS, 20.0, prec)
    d = _np(plan.gaussian_field(seed=11))
    plan.sync()
    ora = run_oracle(w, seed=11, components=(), want_delta=True)
    assert rel_l2(d, ora["delta"]) < (1e-12 if prec == "f64" else 1e-5)


def test_partial_outputs_and_corner_lattice(gg):
    n, box = 24, 30.0
    w = dict(n=n, box=box, cosmo=BBKS, z_init=5.0)
    plan = gg.Plan(n, box, BBKS, 5.0, "f64", corner=True)
    shape = (n, n, n)
    e = lambda: torch.empty(shape, dtype=torch.float64, device="cuda")
    out = {"psi": [None, e(), None], "pos": [e(), None, None], "vel": [None, None, e()]}
    plan.zeldovich(seed=9, out=out)
    plan.sync()
    ora = run_oracle(w, seed=9, corner=True)
    _compare(out, ora, box, "f64")


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [24, 64, 192])
def test_pos_vel_only_outputs(gg, n, prec):
    """pos + vel without psi (the z inverse instantiation of the plain path,
    component fixed at compile time): bit-identical to the same outputs of a
    call that also writes psi (the run-time-flag kernel), and within the
    parity tolerances of the oracle."""
    box = 1.25 * n
    w = dict(n=n, box=box, cosmo=BBKS, z_init=40.0)
    plan = gg.Plan(n, box, BBKS, 40.0, prec)
    plain = plan.zeldovich(seed=12, psi=False)
    full = plan.zeldovich(seed=12)
    plan.sync()
    for k in ("pos", "vel"):
        for j in range(3):
            assert torch.equal(plain[k][j], full[k][j]), (k, j)
    ora = run_oracle(w, seed=12)
    _compare(plain, ora, box, prec, keys=("pos", "vel"))
    plan.close()


def test_planted_mode_closed_form(gg):
    """W(x_n) = cos(k0.x_n): delta = s cos, psi = -s k0/|k0|^2 sin (Eqs. 1-2)."""
    from tests.oracle_cases import cosmology_from
    n, box, z = 32, 64.0, 30.0
    c = cosmology_from(BBKS)
    i = np.arange(n)
    ix, iy, iz = np.meshgrid(i, i, i, indexing="ij")
    m0 = (2, -3, 5)
    phase = 2 * math.pi * (m0[0] * ix + m0[1] * iy + m0[2] * iz) / n
    plan = gg.Plan(n, box, BBKS, z, "f64")
    out = plan.zeldovich(noise=torch.tensor(np.cos(phase), device="cuda"), pos=False, vel=False)
    plan.sync()
    k0 = 2 * math.pi / box * np.array(m0, dtype=float)
    kk = math.sqrt((k0 ** 2).sum())
    s = plan.info["growth"] * math.sqrt(c.power(kk) * n ** 3 / box ** 3)
    for j in range(3):
        want = -s * k0[j] / kk ** 2 * np.sin(phase)
        np.testing.assert_allclose(_np(out["psi"][j]), want, atol=1e-12 * s / kk)


def test_repeatable_and_seed_dependent(gg):
    plan = gg.Plan(32, 50.0, BBKS, 50.0, "f32")
    a = _np(plan.zeldovich(seed=4, pos=False, vel=False)["psi"][2])
    b = _np(plan.zeldovich(seed=4, pos=False, vel=False)["psi"][2])
    c = _np(plan.zeldovich(seed=5, pos=False, vel=False)["psi"][2])
    assert np.array_equal(a, b)
    assert rel_l2(c, a) > 0.5


def test_host_buffer_entry_point(gg):
    n = 32
    plan = gg.Plan(n, 50.0, BBKS, 50.0, "f64")
    dev = plan.zeldovich(seed=2)
    host = plan.zeldovich_host(seed=2)
    for k in ("psi", "pos", "vel"):
        for j in range(3):
            assert np.array_equal(host[k][j].numpy(), _np(dev[k][j]))
    grid = torch.randn((n, n, n), dtype=torch.float64)
    h2 = plan.zeldovich_host(noise=grid, psi=True, pos=False, vel=False)
    d2 = plan.zeldovich(noise=grid.cuda(), pos=False, vel=False)
    assert np.array_equal(h2["psi"][1].numpy(), _np(d2["psi"][1]))
    # pageable outputs take the staged path (device buffer + copy)
    page = {k: [torch.empty((n, n, n), dtype=torch.float64) for _ in range(3)]
            for k in ("psi", "pos", "vel")}
    h3 = plan.zeldovich_host(seed=2, out=page)
    for k in ("psi", "pos", "vel"):
        for j in range(3):
            assert np.array_equal(h3[k][j].numpy(), _np(dev[k][j]))


def test_invalid_device_arguments(gg):
    import ctypes
    plan = gg.Plan(16, 10.0, BBKS, 10.0, "f32")
    t = torch.empty(16 ** 3 + 1, dtype=torch.float32, device="cuda")
    bad = t[1:]  # 4-byte offset: not 16-byte aligned
    arr = (ctypes.c_void_p * 3)(bad.data_ptr(), None, None)
    st = gg.lib().gg_zeldovich(plan.handle, 1, None, arr, None, None)
    assert st == gg.GG_EINVAL
    assert b"unaligned" in gg.lib().gg_last_error(plan.handle)
