"""Named synthetic workloads (plain parameter dicts; no arithmetic of the method).

These stand in for the paper's runs, whose tabulated power spectrum and white
noise files are not available: analytic BBKS / Eisenstein-Hu no-wiggle
spectra and Philox noise replace them. The box sizes follow the paper's
single-resolution runs (a 500 Mpc/h box with 512^3 cells, Sec. 3.3; a
64-100 Mpc/h box, Secs. 3.1 and 3.4; a 2000 Mpc/h box at the 1536^3 scale).
Both the CUDA path (through the binding) and the tests' oracle calls read
these dicts, so the two sides see identical inputs.
"""

BBKS = dict(omega_m=0.3, h=0.7, n_s=0.96, sigma_8=0.8, tf="bbks", omega_l=-1.0,
            omega_b=0.049, t_cmb=2.7255)

EH_NW = dict(omega_m=0.31, h=0.68, n_s=0.965, sigma_8=0.81, tf="eh_nw", omega_l=-1.0,
             omega_b=0.049, t_cmb=2.7255)

WORKLOADS = {
    # plain method, FP64, 64^3 in a 100 Mpc/h box, z = 50
    "zeldovich_64_fp64": dict(n=64, box=100.0, cosmo=BBKS, z_init=50.0, seed=1, prec="f64"),
    # plain method on the GPU, 512^3 in a 500 Mpc/h box, z = 100
    "zeldovich_512_fp32": dict(n=512, box=500.0, cosmo=BBKS, z_init=100.0, seed=1, prec="f32"),
    "zeldovich_512_fp64": dict(n=512, box=500.0, cosmo=BBKS, z_init=100.0, seed=1, prec="f64"),
    # precision form at scale: 1536^3, 2000 Mpc/h, EH no-wiggle, z = 100
    "zeldovich_1536_fp32": dict(n=1536, box=2000.0, cosmo=EH_NW, z_init=100.0, seed=1, prec="f32"),
    # differentiation form: 512^3, 500 Mpc/h, FP32, 4096 targets, R = 8 Mpc/h
    "adjoint_512_fp32": dict(n=512, box=500.0, cosmo=BBKS, z_init=100.0, seed=1, prec="f32",
                             targets=4096, smoothing=8.0),
    "adjoint_64_fp64": dict(n=64, box=100.0, cosmo=BBKS, z_init=50.0, seed=1, prec="f64",
                            targets=4096, smoothing=8.0),
}


def batched_realizations(count=48, sizes=(128, 192, 256, 384)):
    """The batched form: seeds 1..count, N cycling through ``sizes``, L = N Mpc/h."""
    out = []
    for i in range(count):
        n = sizes[i % len(sizes)]
        out.append(dict(n=n, box=float(n), cosmo=BBKS, z_init=50.0, seed=i + 1, prec="f32"))
    return out


# Appendix A white-noise refinement: a 768^3 parent (Philox white noise,
# seed 1) doubled to the 1536^3 grid of the largest Zel'dovich workload with
# the bases of Eqs. A.10-A.13; new coefficients from seed 2.
REFINE_WORKLOADS = {
    "refine_768_1536_fp32": dict(n=768, kind="2", prec="f32", seed_parent=1, seed_child=2),
    # the same at an eighth of the size (profiling captures)
    "refine_384_768_fp32": dict(n=384, kind="2", prec="f32", seed_parent=1, seed_child=2),
}
