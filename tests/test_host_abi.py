"""Host-side checks of the C ABI (no GPU needed, no device calls).

* libgg.so loads and exports every function declared in include/gg.h;
* the library's FP64 host mathematics (growth, velocity factor, sigma_8
  normalisation, P(k), the Eq. 1 filter table) equals the oracle's;
* invalid parameters are rejected with GG_EINVAL.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_2511_10353_gb300 as gg
from paper_2511_10353_gb300 import workloads as W
from oracle import fields
from tests.oracle_cases import cosmology_from

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_10353_gb300 import build
    build.build(verbose=False)


def _declared():
    text = open(os.path.join(ROOT, "include", "gg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gg_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    names = _declared()
    assert "gg_zeldovich" in names and "gg_plan" in names and len(names) >= 15
    h = ctypes.CDLL(gg.library_path())
    for name in names:
        assert hasattr(h, name), name
    assert gg.lib().gg_version() >= 100


@pytest.mark.parametrize("cfg,z", [(W.BBKS, 50.0), (W.BBKS, 100.0), (W.EH_NW, 100.0)])
def test_host_scalars_match_oracle(cfg, z):
    c = cosmology_from(cfg)
    info = gg.cosmo_eval(64, 100.0, cfg, z)
    a = 1.0 / (1.0 + z)
    assert abs(info["a"] - a) < 1e-15
    assert abs(info["growth"] - c.growth(a)) < 1e-11 * c.growth(a)
    assert abs(info["growth_rate"] - c.growth_rate(a)) < 1e-11
    assert abs(info["vfac"] - c.velocity_factor(a)) < 1e-10 * c.velocity_factor(a)
    assert abs(info["amplitude"] - c.amplitude()) < 1e-10 * c.amplitude()
    assert abs(info["sigma_8"] - cfg["sigma_8"]) < 1e-10


@pytest.mark.parametrize("cfg", [W.BBKS, W.EH_NW])
def test_host_power_matches_oracle(cfg):
    c = cosmology_from(cfg)
    k = np.logspace(-4, 1.5, 200)
    np.testing.assert_allclose(gg.power(cfg, k), c.power(k), rtol=1e-10)


def test_host_power_table():
    base = cosmology_from(W.BBKS)
    tk = np.logspace(-4, 2, 3000)
    cfg = dict(W.BBKS, tf="table", tab_k=tk, tab_p=base.power(tk) * 5.0)
    k = np.array([1e-3, 0.02, 0.3, 3.0])
    np.testing.assert_allclose(gg.power(cfg, k), base.power(k), rtol=3e-4)
    keep = dict(cfg, sigma_8=0.0)  # keep the table amplitude
    np.testing.assert_allclose(gg.power(keep, k), 5.0 * base.power(k), rtol=1e-6)
    assert gg.power(keep, np.array([1e-5, 200.0])).tolist() == [0.0, 0.0]


def test_filter_table_matches_oracle_filter():
    n, box, z = 32, 80.0, 30.0
    c = cosmology_from(W.BBKS)
    s = gg.filter_table(n, box, W.BBKS, z, 3 * (n // 2) ** 2 + 1)
    filt = fields.density_filter(n, box, c, c.growth(1 / (1 + z)))
    mx, my, mz = fields.integer_modes(n)
    m2 = (mx * mx + my * my + mz * mz)
    keep = fields.keep_mask(n)
    np.testing.assert_allclose(s[m2[keep]], filt[keep], rtol=1e-11)
    assert s[0] == 0.0


def test_workspace_size_scales():
    a = gg.workspace_size(64, 100.0, W.BBKS, 50.0, "f32")
    b = gg.workspace_size(64, 100.0, W.BBKS, 50.0, "f64")
    assert a >= 2 * 64 ** 3 * 4 and b >= 2 * 64 ** 3 * 8


@pytest.mark.parametrize("bad", [
    dict(n=63), dict(n=0), dict(n=10), dict(n=8192), dict(box=0.0), dict(box=-1.0),
    dict(z_init=-0.5), dict(cosmo=dict(W.BBKS, sigma_8=0.0)), dict(cosmo=dict(W.BBKS, omega_m=0.0)),
    dict(cosmo=dict(W.BBKS, h=-0.7)), dict(cosmo=dict(W.EH_NW, omega_b=0.5)),
    dict(cosmo=dict(W.BBKS, tf="table", tab_k=[0.1, 0.05], tab_p=[1.0, 2.0])),
    dict(prec=7),
])
def test_invalid_parameters_rejected(bad):
    args = dict(n=64, box=100.0, cosmo=W.BBKS, z_init=50.0, prec="f32")
    args.update(bad)
    p, _keep = gg.make_params(args["n"], args["box"], args["cosmo"], args["z_init"], args["prec"])
    if args["prec"] == 7:
        p.prec = 7
    info = gg.Info()
    st = gg.lib().gg_cosmo_eval(ctypes.byref(p), ctypes.byref(info))
    assert st == gg.GG_EINVAL
    assert gg.lib().gg_last_error(None)


def test_null_arguments_rejected():
    L = gg.lib()
    assert L.gg_plan(None, None, None) == gg.GG_EINVAL
    assert L.gg_zeldovich(None, 1, None, None, None, None) == gg.GG_EINVAL
    assert L.gg_sync(None) == gg.GG_EINVAL
    assert L.gg_noise_bits(1, -1, 4, None, None) == gg.GG_EINVAL
    assert L.gg_large_scales(None, 1.0, None, None) == gg.GG_EINVAL
    null3 = gg._VP3(None, None, None)
    assert L.gg_zeldovich_merge(None, 1, None, 1.0, 8, null3, null3, null3, null3) == gg.GG_EINVAL
    assert L.gg_set_shift(None, None) == gg.GG_EINVAL
    assert L.gg_zeldovich_gas(None, 1, None, 0.1, null3, null3, null3, null3) == gg.GG_EINVAL
    assert L.gg_particle_ids(None, 16, 0, None) == gg.GG_EINVAL
    assert L.gg_degrade(None, 32, None, None) == gg.GG_EINVAL
    assert L.gg_power_spectrum(None, None, 4, None, None, None) == gg.GG_EINVAL
    assert L.gg_field_moments(None, None, None) == gg.GG_EINVAL
    L.gg_free(None)


def test_quadrature_is_exact_for_polynomials():
    """EdS (Om = 1): the growth integral of x^{3/2} is exact, so D(a) = a to rounding."""
    eds = dict(W.BBKS, omega_m=1.0, omega_l=0.0)
    for z in (0.0, 1.0, 99.0):
        info = gg.cosmo_eval(64, 100.0, eds, z)
        assert abs(info["growth"] - 1 / (1 + z)) < 1e-13
        assert abs(info["growth_rate"] - 1.0) < 1e-12
        assert abs(info["vfac"] - 100.0 * math.sqrt(1 + z)) < 1e-10


@pytest.mark.parametrize("kind,n,origin,extent,want", [
    ("2", 16, (0, 0, 0), None, (32, 32, 32)),
    ("3/2", 16, (0, 0, 0), None, (24, 24, 24)),
    ("4/3", 12, (3, 0, 6), (6, 12, 3), (8, 16, 4)),
    ("hr", 7, (1, 2, 3), (2, 3, 7), (4, 6, 14)),
    ("2-sine", 10, (8, 0, 2), (4, 2, 10), (8, 4, 20)),
])
def test_refine_dims(kind, n, origin, extent, want):
    assert gg.refine_dims(n, kind, origin, extent) == want


@pytest.mark.parametrize("kind,n,origin,extent", [
    ("2", 15, (0, 0, 0), None),          # n not a multiple of the parent patch
    ("4/3", 16, (0, 0, 0), None),
    ("2", 16, (1, 0, 0), None),          # origin off the patch grid
    ("2", 16, (16, 0, 0), None),         # origin outside the box
    ("2", 16, (0, 0, 0), (18, 16, 16)),  # extent larger than the box
    ("2", 16, (0, 0, 0), (3, 16, 16)),   # extent off the patch grid
    ("3/2", 16, (0, 0, 0), (16, -2, 16)),
])
def test_refine_invalid_rejected(kind, n, origin, extent):
    p = gg.refine_params(n, kind, "f32", origin, extent)
    dims = (ctypes.c_int64 * 3)()
    assert gg.lib().gg_refine_dims(ctypes.byref(p), dims) == gg.GG_EINVAL
    assert gg.lib().gg_last_error(None)
    # the same check comes before any device work in gg_refine_noise
    assert gg.lib().gg_refine_noise(ctypes.byref(p), None, 1, None, None) == gg.GG_EINVAL


def test_refine_bad_kind_precision_and_pointers():
    L = gg.lib()
    p = gg.refine_params(16, "2")
    p.kind = 9
    assert L.gg_refine_dims(ctypes.byref(p), (ctypes.c_int64 * 3)()) == gg.GG_EINVAL
    p = gg.refine_params(16, "2")
    p.prec = 3
    assert L.gg_refine_dims(ctypes.byref(p), (ctypes.c_int64 * 3)()) == gg.GG_EINVAL
    p = gg.refine_params(16, "2")
    assert L.gg_refine_dims(None, (ctypes.c_int64 * 3)()) == gg.GG_EINVAL
    assert L.gg_refine_dims(ctypes.byref(p), None) == gg.GG_EINVAL
    # NULL or misaligned buffers: rejected before any device call
    assert L.gg_refine_noise(ctypes.byref(p), None, 1, None, None) == gg.GG_EINVAL
    assert L.gg_refine_noise(ctypes.byref(p), 4, 1, 4096, None) == gg.GG_EINVAL
    assert b"aligned" in L.gg_last_error(None)
