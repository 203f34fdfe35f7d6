"""The adjoint form: gradients of a loss on the smoothed Zel'dovich density
with respect to the white noise, through torch.autograd.Function wrappers of
the library's kernels.

* 64^3 FP64: every piece (psi transpose, CIC density, CIC adjoint, smoothing)
  and the whole loss gradient against the FP64 oracle;
* 512^3, L = 500 Mpc/h, FP32, 4096 random targets, y ~ N(0,1), R = 8 Mpc/h:
  the FP32 adjoint gradient against central finite differences on 64 random
  cells, each loss evaluated with the GPU FP64 path (1e-4); the linear-density
  loss (exactly quadratic) as well.
"""
import numpy as np
import pytest

from oracle import adjoint as oadj
from tests.gpu_helpers import rel_l2
from tests.oracle_cases import cosmology_from

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BBKS = dict(omega_m=0.3, h=0.7, n_s=0.96, sigma_8=0.8, tf="bbks", omega_l=-1.0,
            omega_b=0.049, t_cmb=2.7255)
C = cosmology_from(BBKS)


@pytest.fixture(scope="module")
def gg():
    from paper_2511_10353_gb300 import build
    build.build(verbose=False)
    import paper_2511_10353_gb300 as m
    return m


def _np(t):
    return t.detach().cpu().numpy()


def test_pieces_fp64_match_oracle(gg):
    n, box, z, radius = 64, 100.0, 50.0, 8.0
    plan = gg.Plan(n, box, BBKS, z, "f64")
    rng = np.random.default_rng(0)
    g = [rng.standard_normal((n, n, n)) for _ in range(3)]
    got = plan.zeldovich_adjoint([torch.tensor(x, device="cuda") for x in g])
    plan.sync()
    assert rel_l2(_np(got), oadj.psi_adjoint(g, box, C, z)) < 1e-12
    f = rng.standard_normal((n, n, n))
    sm = plan.smooth(torch.tensor(f, device="cuda"), radius)
    plan.sync()
    assert rel_l2(_np(sm), oadj.smooth(f, box, radius)) < 1e-12
    psi = [oadj.psi_map(rng.standard_normal((n, n, n)), box, C, z, j) * 20.0 for j in range(3)]
    tpsi = [torch.tensor(x, device="cuda") for x in psi]
    d = plan.cic_density(tpsi)
    plan.sync()
    want = oadj.cic_density(psi, box)
    assert np.abs(_np(d) - want).max() < 1e-12 * max(1.0, np.abs(want).max())
    ga = plan.cic_density_adjoint(tpsi, torch.tensor(f, device="cuda"))
    plan.sync()
    for j, w in enumerate(oadj.cic_adjoint(psi, f, box)):
        assert rel_l2(_np(ga[j]), w) < 1e-12


@pytest.mark.parametrize("kind", ["cic", "linear"])
def test_loss_gradient_fp64_matches_oracle(gg, kind):
    from paper_2511_10353_gb300.autograd import smoothed_density_loss
    n, box, z, radius = 64, 100.0, 50.0, 8.0
    plan = gg.Plan(n, box, BBKS, z, "f64")
    rng = np.random.default_rng(1)
    w = rng.standard_normal((n, n, n))
    targets = rng.choice(n ** 3, size=4096, replace=False)
    y = rng.standard_normal(4096)
    tw = torch.tensor(w, device="cuda", requires_grad=True)
    loss = smoothed_density_loss(tw, plan, torch.tensor(targets, device="cuda"),
                                 torch.tensor(y, device="cuda"), radius, kind)
    loss.backward()
    lo, _, _ = oadj.density_loss(w, box, C, z, targets, y, radius, kind)
    assert abs(float(loss) - lo) < 1e-10 * lo
    assert rel_l2(_np(tw.grad), oadj.density_loss_grad(w, box, C, z, targets, y, radius, kind)) < 1e-10


@pytest.mark.parametrize("kind,tol", [("cic", 1e-4), ("linear", 1e-4)])
def test_512_fp32_gradient_vs_fp64_finite_differences(gg, kind, tol):
    from paper_2511_10353_gb300.autograd import smoothed_density_loss
    n, box, z, radius = 512, 500.0, 100.0, 8.0
    rng = np.random.default_rng(2)
    w64 = torch.randn((n, n, n), dtype=torch.float64, device="cuda",
                      generator=torch.Generator(device="cuda").manual_seed(5))
    targets = torch.tensor(rng.choice(n ** 3, size=4096, replace=False), device="cuda")
    y = torch.tensor(rng.standard_normal(4096), device="cuda")
    p32 = gg.Plan(n, box, BBKS, z, "f32")
    w32 = w64.float().requires_grad_(True)
    loss = smoothed_density_loss(w32, p32, targets, y.float(), radius, kind)
    loss.backward()
    grad = w32.grad.double()
    del loss, w32
    p32.close()
    torch.cuda.empty_cache()
    p64 = gg.Plan(n, box, BBKS, z, "f64")
    cells = rng.choice(n ** 3, size=64, replace=False)
    eps = 1e-2
    fd, an = [], []
    flat = w64.view(-1)
    with torch.no_grad():
        for c in cells:
            old = float(flat[c])
            flat[c] = old + eps
            lp = float(smoothed_density_loss(w64, p64, targets, y, radius, kind))
            flat[c] = old - eps
            lm = float(smoothed_density_loss(w64, p64, targets, y, radius, kind))
            flat[c] = old
            fd.append((lp - lm) / (2 * eps))
            an.append(float(grad.view(-1)[c]))
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(an - fd) / np.linalg.norm(fd) < tol, (np.abs(an - fd).max(), np.abs(fd).max())
