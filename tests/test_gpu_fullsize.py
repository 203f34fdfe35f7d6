"""Full-size parity on the 512^3 workload in the bench's launch configuration.

512^3, L = 500 Mpc/h, BBKS, z = 100, seed 1: the FP32 and FP64 GPU paths
against the complete FP64 oracle (its noise computed on a spawn-started
process pool). FP32 within 1e-5 relative L2 on displacements and
velocities; FP64 within 1e-12.
"""
import numpy as np
import pytest

from tests.gpu_helpers import min_image, rel_l2, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BBKS = dict(omega_m=0.3, h=0.7, n_s=0.96, sigma_8=0.8, tf="bbks", omega_l=-1.0,
            omega_b=0.049, t_cmb=2.7255)
W512 = dict(n=512, box=500.0, cosmo=BBKS, z_init=100.0)


@pytest.fixture(scope="module")
def oracle512():
    return run_oracle(W512, seed=1)


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("f64", 1e-12)])
def test_512_matches_oracle(oracle512, prec, tol):
    from paper_2511_10353_gb300 import build
    build.build(verbose=False)
    import paper_2511_10353_gb300 as gg
    plan = gg.Plan(512, 500.0, BBKS, 100.0, prec)
    for j in range(3):
        e = lambda: torch.empty((512,) * 3, dtype=plan.dtype, device="cuda")
        out = {"psi": [None] * 3, "pos": [None] * 3, "vel": [None] * 3}
        out["psi"][j], out["pos"][j], out["vel"][j] = e(), e(), e()
        plan.zeldovich(seed=1, out=out)
        plan.sync()
        psi = out["psi"][j].cpu().numpy()
        assert rel_l2(psi, oracle512["psi"][j]) < tol
        assert rel_l2(out["vel"][j].cpu().numpy(), oracle512["vel"][j]) < tol
        d = min_image(out["pos"][j].cpu().numpy().astype(np.float64) - oracle512["pos"][j], 500.0)
        lim = 4 * float(np.spacing(np.float32(500.0))) if prec == "f32" else 1e-10
        assert np.abs(d).max() < lim + tol * np.abs(oracle512["psi"][j]).max()
        del out, psi


def test_512_pos_vel_only_matches_oracle(oracle512):
    """The bench's launch configuration: all three components, pos + vel
    only (the compile-time z inverse of the plain path), FP32."""
    from paper_2511_10353_gb300 import build
    build.build(verbose=False)
    import paper_2511_10353_gb300 as gg
    plan = gg.Plan(512, 500.0, BBKS, 100.0, "f32")
    plan.autotune(2)
    out = plan.zeldovich(seed=1, psi=False)
    plan.sync()
    lim = 4 * float(np.spacing(np.float32(500.0)))
    for j in range(3):
        assert rel_l2(out["vel"][j].cpu().numpy(), oracle512["vel"][j]) < 1e-5
        d = min_image(out["pos"][j].cpu().numpy().astype(np.float64) - oracle512["pos"][j], 500.0)
        assert np.abs(d).max() < lim + 1e-5 * np.abs(oracle512["psi"][j]).max()
    del out
    plan.close()
