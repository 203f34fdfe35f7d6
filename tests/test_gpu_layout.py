"""The chunk-major spectrum layout between the y passes.

The three-component chain can keep the spectrum as [k_z chunk][x][y][tile
width] between the y forward and the y inverse passes instead of [x][y][k_z]:
the same butterflies and filter in the same order on the same values, so the
positions and velocities agree bit for bit with the plain layout, for every
strided variant, and still match the oracle.
"""
import numpy as np
import pytest

from tests.gpu_helpers import min_image, rel_l2, run_oracle

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


def _run(gg, plan, n, prec, seed):
    dt = torch.float32 if prec == "f32" else torch.float64
    pos = [torch.empty((n, n, n), dtype=dt, device="cuda") for _ in range(3)]
    vel = [torch.empty((n, n, n), dtype=dt, device="cuda") for _ in range(3)]
    plan.zeldovich(seed=seed, out={"psi": [None] * 3, "pos": pos, "vel": vel})
    plan.sync()
    return pos, vel


@pytest.mark.parametrize("n,prec", [(64, "f32"), (192, "f32"), (256, "f32"), (512, "f32"),
                                    (64, "f64")])
def test_layouts_bit_identical(gg, n, prec):
    plan = gg.Plan(n, float(n), BBKS, 50.0, prec)
    for a in range(3):
        plan.set_variants([0, a, a, a, a, 0])
        plan.set_layout(False)
        assert not plan.layout()
        pos0, vel0 = _run(gg, plan, n, prec, seed=11)
        plan.set_layout(True)
        assert plan.layout()
        pos1, vel1 = _run(gg, plan, n, prec, seed=11)
        for j in range(3):
            assert torch.equal(pos0[j], pos1[j]), (a, j)
            assert torch.equal(vel0[j], vel1[j]), (a, j)
        assert float(vel0[2].abs().max()) > 0.0


def test_chunk_major_matches_oracle(gg):
    """FP32 parity of the chunk-major chain: velocities within 1e-5 relative
    L2 of the oracle, positions as minimum-image differences within 4 ulp(L)
    + 1e-5 max|psi| (the tolerances of the plain path)."""
    n, box = 128, 128.0
    plan = gg.Plan(n, box, BBKS, 50.0, "f32")
    plan.set_layout(True)
    assert plan.layout()
    pos, vel = _run(gg, plan, n, "f32", seed=5)
    ora = run_oracle(dict(n=n, box=box, cosmo=BBKS, z_init=50.0), seed=5)
    ulp = np.spacing(np.float32(box))
    for j in range(3):
        assert rel_l2(vel[j].cpu().numpy(), ora["vel"][j]) < 1e-5, j
        p = pos[j].cpu().numpy().astype(np.float64)
        assert p.min() >= 0.0 and p.max() < box
        d = min_image(p - ora["pos"][j], box)
        assert np.abs(d).max() < 4 * ulp + 1e-5 * np.abs(ora["psi"][j]).max(), j


def test_layout_needs_three_components(gg):
    """psi outputs, or fewer than three components, take the plain chain: the
    results equal the plain layout's whatever the switch says."""
    n = 64
    plan = gg.Plan(n, 64.0, BBKS, 50.0, "f32")
    psi = [torch.empty((n, n, n), dtype=torch.float32, device="cuda") for _ in range(3)]
    outs = []
    for lay in (False, True):
        plan.set_layout(lay)
        plan.zeldovich(seed=2, out={"psi": psi, "pos": [None] * 3, "vel": [None] * 3})
        plan.sync()
        outs.append([p.clone() for p in psi])
    for j in range(3):
        assert torch.equal(outs[0][j], outs[1][j])
    assert gg.lib().gg_plan_set_layout(plan._h, 2) == gg.GG_EINVAL  # only 0 and 1
