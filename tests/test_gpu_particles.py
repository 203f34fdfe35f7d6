"""GPU particle options (Sec. 2.2) and degrading (Sec. 2.4) against the oracle.

Periodic shift and gas pairs: positions within the parity tolerances of the
plain path (FP64 1e-12, FP32 a few ulp of L plus 1e-5 of psi), velocities
bit-identical to gg_zeldovich, and a zero shift restoring gg_zeldovich bit
for bit; coordinate IDs exactly; degraded fields within 1e-12 (FP64) /
1e-5 (FP32) of the oracle, for size-specialised and run-time grid sizes.
"""
import numpy as np
import pytest

from oracle import noise as onoise
from oracle import particles as opart
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


def _pos_close(got, want, psi, box, prec):
    g = got.cpu().numpy().astype(np.float64)
    assert g.min() >= 0.0 and g.max() < box
    d = min_image(g - want, box)
    if prec == "f64":
        assert np.abs(d).max() < 1e-12 * max(1.0, np.abs(psi).max()) + 4e-16 * box
    else:
        assert np.abs(d).max() < 4 * np.spacing(np.float32(box)) + 1e-5 * np.abs(psi).max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [64, 24])
def test_periodic_shift(gg, n, prec):
    box, z = 1.5 * n, 40.0
    shift = (0.3 * box, -1.25, 2.5 * box + 0.7)
    plan = gg.Plan(n, box, BBKS, z, prec)
    plain = plan.zeldovich(seed=4)
    plan.set_shift(shift)
    got = plan.zeldovich(seed=4)
    plan.set_shift((0.0, 0.0, 0.0))
    again = plan.zeldovich(seed=4)
    plan.sync()
    ora = run_oracle(dict(n=n, box=box, cosmo=BBKS, z_init=z), seed=4)
    want = opart.positions([ora["psi"][j] for j in range(3)], box, shift)
    for j in range(3):
        _pos_close(got["pos"][j], want[j], ora["psi"][j], box, prec)
        assert torch.equal(got["vel"][j], plain["vel"][j])
        assert torch.equal(again["pos"][j], plain["pos"][j])
    plan.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [64, 24])
def test_gas_pairs(gg, n, prec):
    box, z, f = 2.0 * n, 40.0, 0.049 / 0.3
    plan = gg.Plan(n, box, BBKS, z, prec)
    plain = plan.zeldovich(seed=6)
    got = plan.zeldovich_gas(f, seed=6, psi=True)
    plan.sync()
    ora = run_oracle(dict(n=n, box=box, cosmo=BBKS, z_init=z), seed=6)
    psi = [ora["psi"][j] for j in range(3)]
    dm, gas = opart.gas_pairs(psi, box, f)
    for j in range(3):
        _pos_close(got["pos"][j], dm[j], psi[j], box, prec)
        _pos_close(got["pos_gas"][j], gas[j], psi[j], box, prec)
        assert torch.equal(got["vel"][j], plain["vel"][j])
        assert torch.equal(got["psi"][j], plain["psi"][j])
    plan.close()


@pytest.mark.parametrize("n,nf,offset", [(16, 16, 0), (16, 48, 7), (24, 96, 10 ** 12)])
def test_particle_ids(gg, n, nf, offset):
    plan = gg.Plan(n, 10.0, BBKS, 40.0, "f32")
    got = plan.particle_ids(nf, offset).cpu().numpy()
    plan.close()
    assert np.array_equal(got, opart.particle_ids(n, nf, offset))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nl,r", [(64, 2), (64, 3), (24, 2)])
def test_degrade_matches_oracle(gg, nl, r, prec):
    nh = nl * r
    f = onoise.white_noise(21, nh)
    dt = torch.float64 if prec == "f64" else torch.float32
    plan = gg.Plan(nl, float(nl), BBKS, 40.0, prec)
    got = plan.degrade(torch.tensor(f, dtype=dt, device="cuda")).cpu().numpy().astype(np.float64)
    plan.close()
    want = opart.degrade(f, r)
    if prec == "f64":
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    else:
        assert rel_l2(got, want) < 1e-5
