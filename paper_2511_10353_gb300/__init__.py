"""Python binding of the GB300 Zel'dovich initial-conditions library (libgg.so).

Argument marshalling only: every step of the path (Philox noise, the r2c /
c2r transform passes, the Eq. 1 / Eq. 2 filters and the Eq. 3 epilogue of
Ginnungagap, arXiv:2511.10353) runs in the library's sm_103a kernels. PyTorch
provides device memory and the current CUDA stream. There is no CPU path:
when libgg.so is missing or no GPU is visible, the calls raise.

    import paper_2511_10353_gb300 as gg
    plan = gg.Plan(n=512, box=500.0, cosmo=gg.workloads.BBKS, z_init=100.0, prec="f32")
    out = plan.zeldovich(seed=1)          # dict of psi / pos / vel, 3 tensors each
"""
import ctypes
import math
import os

import numpy as np

from . import workloads  # noqa: F401  (plain parameter dicts)

__all__ = ["Plan", "Batch", "GGError", "noise_bits", "cosmo_eval", "power", "filter_table",
           "workspace_size", "library_path", "lib", "workloads"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgg.so")
_lib = None

GG_OK, GG_EINVAL, GG_ENOMEM, GG_ECUDA, GG_ETIMEOUT = 0, -1, -2, -3, -4
GG_TEST_NONE, GG_TEST_SKIP_COPY, GG_TEST_STALL_COUNT = 0, 1, 2
GG_F32, GG_F64 = 0, 1
TF = {"bbks": 0, "eh_nw": 1, "table": 2}
GG_Q_CORNER = 0x1
_STATUS = {GG_EINVAL: "GG_EINVAL", GG_ENOMEM: "GG_ENOMEM", GG_ECUDA: "GG_ECUDA",
           GG_ETIMEOUT: "GG_ETIMEOUT"}


class GGError(RuntimeError):
    """A library call returned a status other than GG_OK."""

    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), message))
        self.status = status


class Cosmo(ctypes.Structure):
    _fields_ = [("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double),
                ("omega_b", ctypes.c_double), ("h", ctypes.c_double), ("n_s", ctypes.c_double),
                ("sigma_8", ctypes.c_double), ("t_cmb", ctypes.c_double),
                ("tf", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("tab_k", ctypes.POINTER(ctypes.c_double)),
                ("tab_p", ctypes.POINTER(ctypes.c_double)), ("tab_n", ctypes.c_int64)]


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("box", ctypes.c_double), ("prec", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("cosmo", Cosmo), ("z_init", ctypes.c_double),
                ("growth_override", ctypes.c_double * 2)]


class Info(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("growth", ctypes.c_double),
                ("growth_rate", ctypes.c_double), ("hubble", ctypes.c_double),
                ("vfac", ctypes.c_double), ("amplitude", ctypes.c_double),
                ("sigma_8", ctypes.c_double), ("n", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64)]


class RefineParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("prec", ctypes.c_int), ("kind", ctypes.c_int),
                ("origin", ctypes.c_int64 * 3), ("extent", ctypes.c_int64 * 3)]


# Appendix A refinement kinds (gg_refine_kind)
REFINE_KINDS = {"hr": 0, "3/2": 1, "2": 2, "2-linear": 3, "2-sine": 4, "4/3": 5}

_VP3 = ctypes.c_void_p * 3

# name -> (restype, argtypes); mirrors include/gg.h
_SIGS = {
    "gg_version": (ctypes.c_int, []),
    "gg_cosmo_eval": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(Info)]),
    "gg_power": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int64]),
    "gg_filter_table": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_int64]),
    "gg_workspace_size": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]),
    "gg_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Params),
                               ctypes.c_void_p]),
    "gg_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gg_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Info)]),
    "gg_white_noise": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "gg_noise_bits": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "gg_gaussian_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "gg_zeldovich": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gg_zeldovich_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gg_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "gg_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "gg_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "gg_plan_variants": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gg_plan_set_variants": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gg_plan_set_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "gg_plan_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "gg_batch_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p]),
    "gg_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "gg_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "gg_batch_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "gg_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int64)]),
    "gg_batch_free": (None, [ctypes.c_void_p]),
    "gg_batch_launches": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "gg_batch_set_persistent": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "gg_batch_test_arm_fault": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32]),
    "gg_zeldovich_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gg_smooth": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    "gg_cic_density": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gg_cic_density_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p]),
    "gg_set_shift": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gg_zeldovich_gas": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "gg_particle_ids": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_void_p]),
    "gg_degrade": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "gg_power_spectrum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gg_field_moments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gg_large_scales": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "gg_zeldovich_merge": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                          ctypes.c_double, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gg_refine_dims": (ctypes.c_int, [ctypes.POINTER(RefineParams), ctypes.POINTER(ctypes.c_int64)]),
    "gg_refine_noise": (ctypes.c_int, [ctypes.POINTER(RefineParams), ctypes.c_void_p, ctypes.c_uint64,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "gg_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "gg_test_arm_fault": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32]),
    "gg_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "gg_free": (None, [ctypes.c_void_p]),
}


def library_path():
    return _LIB_PATH


def lib():
    """The loaded libgg.so. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libgg.so is not built (%s); run `python -m "
                               "paper_2511_10353_gb300.build`" % _LIB_PATH)
        h = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def _check(status, plan=None):
    if status != GG_OK:
        msg = lib().gg_last_error(plan)
        raise GGError(status, msg.decode() if msg else "")


def make_params(n, box, cosmo, z_init, prec="f32", corner=False, growth_override=None):
    """Fill a Params struct; returns (params, keepalive) (table arrays stay referenced)."""
    p = Params()
    p.n = int(n)
    p.box = float(box)
    p.prec = GG_F64 if prec in ("f64", "fp64", "double", GG_F64) else GG_F32
    p.flags = GG_Q_CORNER if corner else 0
    c = p.cosmo
    c.omega_m = cosmo["omega_m"]
    c.omega_l = cosmo.get("omega_l", -1.0)
    c.omega_b = cosmo.get("omega_b", 0.049)
    c.h = cosmo["h"]
    c.n_s = cosmo["n_s"]
    c.sigma_8 = cosmo["sigma_8"]
    c.t_cmb = cosmo.get("t_cmb", 2.7255)
    c.tf = TF[cosmo.get("tf", "bbks")]
    keep = []
    if cosmo.get("tf") == "table":
        tk = np.ascontiguousarray(cosmo["tab_k"], dtype=np.float64)
        tp = np.ascontiguousarray(cosmo["tab_p"], dtype=np.float64)
        keep += [tk, tp]
        c.tab_k = tk.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.tab_p = tp.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.tab_n = len(tk)
    p.z_init = float(z_init)
    g = growth_override if growth_override is not None else (math.nan, math.nan)
    p.growth_override[0], p.growth_override[1] = float(g[0]), float(g[1])
    return p, keep


def _info_dict(info):
    return {f: getattr(info, f) for f, _ in Info._fields_}


def cosmo_eval(n, box, cosmo, z_init, prec="f32", **kw):
    """Host-only FP64 scalars (growth, rate, velocity factor, amplitude, sigma_8)."""
    p, _keep = make_params(n, box, cosmo, z_init, prec, **kw)
    info = Info()
    _check(lib().gg_cosmo_eval(ctypes.byref(p), ctypes.byref(info)))
    return _info_dict(info)


def power(cosmo, k, n=64, box=100.0, z_init=0.0):
    """Host-only normalised P(k, z=0) from the library's FP64 code."""
    p, _keep = make_params(n, box, cosmo, z_init)
    k = np.ascontiguousarray(k, dtype=np.float64)
    out = np.empty_like(k)
    _check(lib().gg_power(ctypes.byref(p), k.ctypes.data, out.ctypes.data, k.size))
    return out


def filter_table(n, box, cosmo, z_init, count):
    """Host-only FP64 S(m2) = D sqrt(P/V) for m2 = 0..count-1."""
    p, _keep = make_params(n, box, cosmo, z_init)
    out = np.empty(int(count), dtype=np.float64)
    _check(lib().gg_filter_table(ctypes.byref(p), out.ctypes.data, out.size))
    return out


def workspace_size(n, box, cosmo, z_init, prec="f32"):
    p, _keep = make_params(n, box, cosmo, z_init, prec)
    out = ctypes.c_size_t()
    _check(lib().gg_workspace_size(ctypes.byref(p), ctypes.byref(out)))
    return out.value


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the library has no CPU path")
    return torch


def _stream_ptr(torch):
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_ptr(t, dtype, numel):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError("expected a contiguous CUDA %s tensor of %d elements" % (dtype, numel))
    return t.data_ptr()


def noise_bits(seed, first_group, count, device=None):
    """Raw Philox4x32-10 words (count, 4) as int32 (bitwise uint32) on the GPU."""
    torch = _torch()
    out = torch.empty((int(count), 4), dtype=torch.int32, device=device or "cuda")
    _check(lib().gg_noise_bits(ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), int(first_group),
                               int(count), out.data_ptr(), _stream_ptr(torch)))
    return out


def refine_params(n, kind="2", prec="f32", origin=(0, 0, 0), extent=None):
    p = RefineParams()
    p.n = int(n)
    p.prec = 1 if prec in ("f64", "fp64", "double") else 0
    if kind not in REFINE_KINDS:
        raise ValueError("refinement kind must be one of %s" % sorted(REFINE_KINDS))
    p.kind = REFINE_KINDS[kind]
    for j in range(3):
        p.origin[j] = int(origin[j])
        p.extent[j] = 0 if extent is None else int(extent[j])
    return p


def refine_dims(n, kind="2", origin=(0, 0, 0), extent=None):
    """Shape of the child grid of gg_refine_noise."""
    p = refine_params(n, kind, "f32", origin, extent)
    dims = (ctypes.c_int64 * 3)()
    _check(lib().gg_refine_dims(ctypes.byref(p), dims))
    return tuple(int(d) for d in dims)


def refine_noise(parent, seed_child, kind="2", origin=(0, 0, 0), extent=None, out=None):
    """Appendix A: refined white noise of the box [origin, origin + extent)
    (parent cells) of the periodic parent grid ``parent`` (n^3, float32 or
    float64 CUDA tensor). Returns the child grid (a new tensor, or ``out``)."""
    torch = _torch()
    n = int(parent.shape[0])
    prec = "f64" if parent.dtype == torch.float64 else "f32"
    dtype = torch.float64 if prec == "f64" else torch.float32
    p = refine_params(n, kind, prec, origin, extent)
    dims = (ctypes.c_int64 * 3)()
    _check(lib().gg_refine_dims(ctypes.byref(p), dims))
    shape = tuple(int(d) for d in dims)
    src = _dev_ptr(parent, dtype, n ** 3)
    if out is None:
        out = torch.empty(shape, dtype=dtype, device=parent.device)
    dst = _dev_ptr(out, dtype, shape[0] * shape[1] * shape[2])
    _check(lib().gg_refine_noise(ctypes.byref(p), src, ctypes.c_uint64(int(seed_child) & 0xFFFFFFFFFFFFFFFF),
                                 dst, _stream_ptr(torch)))
    return out


class Plan:
    """A plan for one (N, L, cosmology, z, precision): tables + workspace on the GPU."""

    def __init__(self, n, box, cosmo, z_init, prec="f32", corner=False, growth_override=None):
        torch = _torch()
        self.torch = torch
        self.n = int(n)
        self.prec = "f64" if prec in ("f64", "fp64", "double") else "f32"
        self.dtype = torch.float64 if self.prec == "f64" else torch.float32
        self.device = torch.device("cuda", torch.cuda.current_device())
        p, keep = make_params(n, box, cosmo, z_init, self.prec, corner, growth_override)
        h = ctypes.c_void_p()
        _check(lib().gg_plan(ctypes.byref(h), ctypes.byref(p), _stream_ptr(torch)))
        self._h = h
        del keep
        info = Info()
        _check(lib().gg_plan_info(self._h, ctypes.byref(info)), self._h)
        self.info = _info_dict(info)

    # -------------------------------------------------------------- helpers
    @property
    def handle(self):
        return self._h

    def _bind_stream(self):
        _check(lib().gg_set_stream(self._h, _stream_ptr(self.torch)), self._h)

    def empty(self):
        return self.torch.empty((self.n, self.n, self.n), dtype=self.dtype, device=self.device)

    def _cells(self):
        return self.n ** 3

    # ----------------------------------------------------------------- calls
    def white_noise(self, seed, out=None):
        out = self.empty() if out is None else out
        self._bind_stream()
        _check(lib().gg_white_noise(self._h, ctypes.c_uint64(int(seed)),
                                    _dev_ptr(out, self.dtype, self._cells())), self._h)
        return out

    def gaussian_field(self, seed=0, noise=None, out=None):
        out = self.empty() if out is None else out
        self._bind_stream()
        _check(lib().gg_gaussian_field(self._h, ctypes.c_uint64(int(seed)),
                                       _dev_ptr(noise, self.dtype, self._cells()),
                                       _dev_ptr(out, self.dtype, self._cells())), self._h)
        return out

    def zeldovich(self, seed=0, noise=None, psi=True, pos=True, vel=True, out=None):
        """Positions, velocities and displacements; returns {"psi": [..], "pos": .., "vel": ..}.

        ``out`` may supply preallocated tensors in the same dict form (entries None
        to skip an output).
        """
        if out is None:
            out = {k: [self.empty() for _ in range(3)] if want else [None] * 3
                   for k, want in (("psi", psi), ("pos", pos), ("vel", vel))}
        arrs = []
        for k in ("psi", "pos", "vel"):
            arrs.append(_VP3(*[_dev_ptr(t, self.dtype, self._cells()) for t in out[k]]))
        self._bind_stream()
        _check(lib().gg_zeldovich(self._h, ctypes.c_uint64(int(seed)),
                                  _dev_ptr(noise, self.dtype, self._cells()), *arrs), self._h)
        return out

    def set_shift(self, shift):
        """Periodic shift (Mpc/h) of every later position output."""
        arr = (ctypes.c_double * 3)(*[float(v) for v in shift])
        _check(lib().gg_set_shift(self._h, arr), self._h)

    def zeldovich_gas(self, gas_fraction, seed=0, noise=None, psi=False, vel=True, out=None):
        """Dark-matter and gas-partner positions (Sec. 2.2); returns
        {"psi", "pos", "pos_gas", "vel"}."""
        if out is None:
            out = {"psi": [self.empty() for _ in range(3)] if psi else [None] * 3,
                   "pos": [self.empty() for _ in range(3)],
                   "pos_gas": [self.empty() for _ in range(3)],
                   "vel": [self.empty() for _ in range(3)] if vel else [None] * 3}
        arrs = [_VP3(*[_dev_ptr(t, self.dtype, self._cells()) for t in out[k]])
                for k in ("psi", "pos", "pos_gas", "vel")]
        self._bind_stream()
        _check(lib().gg_zeldovich_gas(self._h, ctypes.c_uint64(int(seed)),
                                      _dev_ptr(noise, self.dtype, self._cells()),
                                      float(gas_fraction), *arrs), self._h)
        return out

    def particle_ids(self, n_finest=None, offset=0, out=None):
        """Coordinate-based int64 IDs of the N^3 particles (Sec. 2.2)."""
        nf = self.n if n_finest is None else int(n_finest)
        if out is None:
            out = self.torch.empty((self.n,) * 3, dtype=self.torch.int64, device=self.device)
        self._bind_stream()
        _check(lib().gg_particle_ids(self._h, nf, int(offset),
                                     _dev_ptr(out, self.torch.int64, self._cells())), self._h)
        return out

    def degrade(self, high, out=None):
        """Sec. 2.4: a field of (r N)^3 points degraded to this plan's grid."""
        nh = int(high.shape[0])
        out = self.empty() if out is None else out
        self._bind_stream()
        _check(lib().gg_degrade(self._h, nh, _dev_ptr(high, self.dtype, nh ** 3),
                                _dev_ptr(out, self.dtype, self._cells())), self._h)
        return out

    def power_spectrum(self, field, nbins=None):
        """Shell-averaged power spectrum of a field: (k, P, count) numpy arrays."""
        import numpy as np
        nb = self.n // 2 if nbins is None else int(nbins)
        k, p, c = np.zeros(nb), np.zeros(nb), np.zeros(nb, dtype=np.int64)
        self._bind_stream()
        _check(lib().gg_power_spectrum(self._h, _dev_ptr(field, self.dtype, self._cells()), nb,
                                       k.ctypes.data, p.ctypes.data, c.ctypes.data), self._h)
        return k, p, c

    def moments(self, field):
        """(mean, variance, min, max) of a field, FP64."""
        out = (ctypes.c_double * 4)()
        self._bind_stream()
        _check(lib().gg_field_moments(self._h, _dev_ptr(field, self.dtype, self._cells()), out),
               self._h)
        return tuple(out)

    def large_scales(self, field, r_s, out=None):
        """Sec. 2.4, Eq. 5 with the cloud-in-cell deconvolution of a real field."""
        out = self.empty() if out is None else out
        self._bind_stream()
        _check(lib().gg_large_scales(self._h, float(r_s), _dev_ptr(field, self.dtype, self._cells()),
                                     _dev_ptr(out, self.dtype, self._cells())), self._h)
        return out

    def zeldovich_merge(self, large, r_s, seed=0, noise=None, psi=True, pos=True, vel=True,
                        out=None):
        """Sec. 2.4: gg_zeldovich keeping modes with |k| r_s >= 1 (Eq. 4) plus the
        cloud-in-cell interpolation of the coarse grids ``large`` (three n_low^3
        tensors or None, Eq. 5 already applied, e.g. by ``large_scales``)."""
        n_low = next((int(t.shape[0]) for t in large if t is not None), 1)
        if out is None:
            out = {k: [self.empty() for _ in range(3)] if want else [None] * 3
                   for k, want in (("psi", psi), ("pos", pos), ("vel", vel))}
        lg = _VP3(*[None if t is None else _dev_ptr(t, self.dtype, n_low ** 3) for t in large])
        arrs = [_VP3(*[_dev_ptr(t, self.dtype, self._cells()) for t in out[k]])
                for k in ("psi", "pos", "vel")]
        self._bind_stream()
        _check(lib().gg_zeldovich_merge(self._h, ctypes.c_uint64(int(seed)),
                                        _dev_ptr(noise, self.dtype, self._cells()), float(r_s),
                                        n_low, lg, *arrs), self._h)
        return out

    def zeldovich_host(self, seed=0, noise=None, psi=True, pos=True, vel=True, out=None):
        """The same path with host (pinned) tensors in and out; synchronous."""
        torch = self.torch
        shape = (self.n, self.n, self.n)
        if out is None:
            out = {k: [torch.empty(shape, dtype=self.dtype, pin_memory=True) for _ in range(3)]
                   if want else [None] * 3 for k, want in (("psi", psi), ("pos", pos), ("vel", vel))}
        arrs = [_VP3(*[None if t is None else t.data_ptr() for t in out[k]])
                for k in ("psi", "pos", "vel")]
        nptr = None
        if noise is not None:
            if noise.is_cuda or noise.dtype != self.dtype or not noise.is_contiguous():
                raise ValueError("noise must be a contiguous host tensor of the plan's dtype")
            nptr = noise.data_ptr()
        self._bind_stream()
        _check(lib().gg_zeldovich_host(self._h, ctypes.c_uint64(int(seed)), nptr, *arrs), self._h)
        return out

    def sync(self):
        _check(lib().gg_sync(self._h), self._h)

    def arm_fault(self, kind="skip_copy", wait_us=2000):
        """Fault test: the next y forward pass issues no tile copies, so its
        waits give up after wait_us and the next sync raises GG_ETIMEOUT."""
        k = {"none": GG_TEST_NONE, "skip_copy": GG_TEST_SKIP_COPY}[kind]
        _check(lib().gg_test_arm_fault(self._h, k, int(wait_us)), self._h)

    # ------------------------------------------------------- adjoint form
    def _ptrs3(self, ts):
        return _VP3(*[None if t is None else _dev_ptr(t, self.dtype, self._cells()) for t in ts])

    def zeldovich_adjoint(self, g_psi, out=None):
        """sum_j J_j^T g_psi[j] (J_j: noise -> psi_j); entries may be None."""
        out = self.empty() if out is None else out
        self._bind_stream()
        _check(lib().gg_zeldovich_adjoint(self._h, self._ptrs3(g_psi),
                                          _dev_ptr(out, self.dtype, self._cells())), self._h)
        return out

    def smooth(self, field, radius, out=None):
        """Gaussian smoothing exp(-k^2 R^2/2) (symmetric; its own adjoint)."""
        out = self.empty() if out is None else out
        self._bind_stream()
        _check(lib().gg_smooth(self._h, float(radius), _dev_ptr(field, self.dtype, self._cells()),
                               _dev_ptr(out, self.dtype, self._cells())), self._h)
        return out

    def cic_density(self, psi, out=None):
        """CIC density contrast of the particles at q + psi."""
        out = self.empty() if out is None else out
        self._bind_stream()
        _check(lib().gg_cic_density(self._h, self._ptrs3(psi),
                                    _dev_ptr(out, self.dtype, self._cells())), self._h)
        return out

    def cic_density_adjoint(self, psi, g_delta):
        """Transpose of the CIC Jacobian at psi applied to g_delta: 3 grids."""
        out = [self.empty() for _ in range(3)]
        self._bind_stream()
        _check(lib().gg_cic_density_adjoint(self._h, self._ptrs3(psi),
                                            _dev_ptr(g_delta, self.dtype, self._cells()),
                                            self._ptrs3(out)), self._h)
        return out

    def autotune(self, reps=3):
        """Time each tile variant of the transform passes; keep the fastest per pass."""
        self._bind_stream()
        _check(lib().gg_autotune(self._h, int(reps)), self._h)
        return self.variants()

    def variants(self):
        """Tile variant per pass: z fwd, y fwd, x fused, y inv (x), y inv (y/z), z inv."""
        out = (ctypes.c_int32 * 6)()
        _check(lib().gg_plan_variants(self._h, out), self._h)
        return list(out)

    def set_variants(self, v):
        """Force the tile variant per pass (6 ints in 0..2)."""
        arr = (ctypes.c_int32 * 6)(*[int(x) for x in v])
        _check(lib().gg_plan_set_variants(self._h, arr), self._h)

    def set_layout(self, chunked):
        """Spectrum layout between the y passes of a three-component run:
        False plain, True chunk-major (bit-identical results)."""
        _check(lib().gg_plan_set_layout(self._h, 1 if chunked else 0), self._h)

    def layout(self):
        """True if the next three-component run keeps the spectrum chunk-major."""
        out = ctypes.c_int32(0)
        _check(lib().gg_plan_layout(self._h, ctypes.byref(out)), self._h)
        return bool(out.value)

    def set_profiling(self, on=True):
        """Bracket every launch with CUDA events on the plan's stream."""
        _check(lib().gg_set_profiling(self._h, 1 if on else 0), self._h)

    def profile(self, reset=True):
        """{kernel kind: {"ms": total, "launches": count, "bytes": per launch}}."""
        cap = 16
        cnt = ctypes.c_int(cap)
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        launches = (ctypes.c_int64 * cap)()
        nbytes = (ctypes.c_double * cap)()
        _check(lib().gg_profile_read(self._h, 1 if reset else 0, ctypes.byref(cnt), names, ms,
                                     launches, nbytes), self._h)
        return {names[i].decode(): {"ms": ms[i], "launches": launches[i], "bytes": nbytes[i]}
                for i in range(cnt.value)}

    def close(self):
        if getattr(self, "_h", None):
            lib().gg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many realizations (each a workload dict with n, box, cosmo, z_init, prec)
    run as one CUDA graph of batched persistent launches (gg_batch_*)."""

    def __init__(self, specs):
        torch = _torch()
        self.torch = torch
        self.specs = list(specs)
        self.count = len(self.specs)
        arr = (Params * self.count)()
        self._keep = []
        for i, w in enumerate(self.specs):
            p, keep = make_params(w["n"], w["box"], w["cosmo"], w["z_init"], w.get("prec", "f32"))
            arr[i] = p
            self._keep.append(keep)
        self.stream = torch.cuda.Stream()  # graph capture needs a non-default stream
        h = ctypes.c_void_p()
        _check(lib().gg_batch_plan(ctypes.byref(h), arr, self.count,
                                   ctypes.c_void_p(self.stream.cuda_stream)))
        self._h = h
        g = ctypes.c_int()
        c = ctypes.c_int64()
        _check(lib().gg_batch_info(self._h, ctypes.byref(g), ctypes.byref(c)))
        self.groups, self.cells = g.value, c.value

    def dtype(self, i):
        return self.torch.float64 if self.specs[i].get("prec") == "f64" else self.torch.float32

    def empty_outputs(self, psi=False, pos=True, vel=True):
        t = self.torch
        def mk(i):
            n = self.specs[i]["n"]
            return t.empty((n, n, n), dtype=self.dtype(i), device="cuda")
        return {k: [[mk(i) for _ in range(3)] if want else [None] * 3 for i in range(self.count)]
                for k, want in (("psi", psi), ("pos", pos), ("vel", vel))}

    def autotune(self, reps=2):
        _check(lib().gg_batch_autotune(self._h, int(reps)))

    def run(self, seeds, out):
        """out: dict psi/pos/vel -> list (per realization) of 3 tensors or None."""
        seeds_arr = (ctypes.c_uint64 * self.count)(*[int(x) for x in seeds])
        arrs = []
        for k in ("psi", "pos", "vel"):
            ptrs = []
            for i in range(self.count):
                n = self.specs[i]["n"]
                for j in range(3):
                    tns = out[k][i][j] if out.get(k) is not None else None
                    ptrs.append(_dev_ptr(tns, self.dtype(i), n ** 3) if tns is not None else None)
            arrs.append((ctypes.c_void_p * (3 * self.count))(*ptrs))
        self.stream.wait_stream(self.torch.cuda.current_stream())
        _check(lib().gg_batch_run(self._h, seeds_arr, *arrs))
        self.torch.cuda.current_stream().wait_stream(self.stream)
        return out

    def sync(self):
        _check(lib().gg_batch_sync(self._h))

    def set_persistent(self, on=True, chunk=None):
        """Later runs as one persistent launch over every pass and realization
        (FP32, N in 64..384), or one launch per pass and group (the default).
        chunk: most tiles per work item (a power of two up to 256; default 64)."""
        v = (int(chunk) if chunk else 1) if on else 0
        _check(lib().gg_batch_set_persistent(self._h, v))

    def arm_fault(self, kind="stall_count", wait_us=2000):
        """Fault test: the next persistent run stalls one pass counter, so its
        waits give up after wait_us and the next sync raises GG_ETIMEOUT."""
        k = {"none": GG_TEST_NONE, "stall_count": GG_TEST_STALL_COUNT}[kind]
        _check(lib().gg_batch_test_arm_fault(self._h, k, int(wait_us)))

    def launches(self):
        """Kernels one run launches (kernel nodes of the captured graph)."""
        k = ctypes.c_int()
        _check(lib().gg_batch_launches(self._h, ctypes.byref(k)))
        return k.value

    def close(self):
        if getattr(self, "_h", None):
            lib().gg_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
