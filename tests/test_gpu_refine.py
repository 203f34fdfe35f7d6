"""GPU white-noise refinement (gg_refine_noise, Appendix A) against the oracle.

FP64: every child value within 1e-13 of the oracle. FP32: relative L2 below
1e-6 and no value off by more than 1e-3 (the FP32 Box-Muller of the new
coefficients, as for gg_white_noise). Sub-boxes, periodic wrap-around,
single patches and odd patch counts; a refined sub-box equals that part of
the refined box bit for bit; at 768^3 -> 1536^3 (FP32) sampled patches
against the oracle and the statistics of the whole child field.
"""
import numpy as np
import pytest

from oracle import noise as onoise
from oracle import refine as oref
from tests.gpu_helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = list(oref.KINDS)


@pytest.fixture(scope="module")
def gg():
    from paper_2511_10353_gb300 import build
    build.build(verbose=False)
    import paper_2511_10353_gb300 as m
    return m


def _dev(a, prec):
    return torch.tensor(a, dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda")


def _check(got, want, prec):
    if prec == "f64":
        assert np.abs(got - want).max() < 1e-13 * max(1.0, np.abs(want).max())
    else:
        assert rel_l2(got, want) < 1e-6
        assert np.abs(got - want).max() < 1e-3


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [6, 12, 30])
def test_full_box_matches_oracle(gg, kind, n, prec):
    parent = onoise.white_noise(5, n)
    got = gg.refine_noise(_dev(parent, prec), 77, kind).cpu().numpy().astype(np.float64)
    want = oref.refine(parent, kind, 77)
    assert got.shape == want.shape
    _check(got, want, prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind", KINDS)
def test_sub_boxes_match_oracle(gg, kind, prec):
    nl = oref.KINDS[kind][0]
    n = 12
    parent = onoise.white_noise(6, n)
    boxes = [((0, 0, 0), (nl, nl, nl)),                      # one patch
             ((n - nl, 0, n - nl), (2 * nl, nl, 2 * nl)),    # wraps in x and z
             ((2 * nl, nl, 0), (n, 2 * nl, 3 * nl)),         # wraps in x, odd patch count
             ((nl, 2 * nl, nl), (3 * nl, n - nl, n))]
    for origin, extent in boxes:
        got = gg.refine_noise(_dev(parent, prec), 3, kind, origin, extent).cpu().numpy().astype(np.float64)
        want = oref.refine(parent, kind, 3, origin, extent)
        assert got.shape == want.shape, (origin, extent)
        _check(got, want, prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["2", "3/2", "4/3", "hr"])
def test_sub_box_is_part_of_full_box_bitwise(gg, kind, prec):
    nl, nh, _, _ = oref.KINDS[kind]
    n = 24
    parent = _dev(onoise.white_noise(8, n), prec)
    full = gg.refine_noise(parent, 11, kind).cpu().numpy()
    origin, extent = (n - 2 * nl, 3 * nl, 0), (4 * nl, 2 * nl, n)
    sub = gg.refine_noise(parent, 11, kind, origin, extent).cpu().numpy()
    nc = n // nl * nh
    idx = [(o // nl * nh + np.arange(x // nl * nh)) % nc for o, x in zip(origin, extent)]
    assert np.array_equal(sub, full[np.ix_(*idx)])


def test_parent_coefficients_survive_fp64(gg):
    n = 16
    parent = onoise.white_noise(12, n)
    for kind in KINDS:
        nl, _, f, _ = oref.KINDS[kind]
        if n % nl:
            continue
        child = gg.refine_noise(_dev(parent, "f64"), 4, kind).cpu().numpy()
        a = oref.parent_coefficients(child, kind)
        back = np.einsum("im,jn,kl,xiyjzk->xmynzl", f, f, f, a).reshape(n, n, n)
        assert np.abs(back - parent).max() < 1e-13, kind


def test_writes_only_the_child_box(gg):
    n = 12
    parent = _dev(onoise.white_noise(2, n), "f32")
    dims = gg.refine_dims(n, "2", (2, 4, 6), (4, 2, 6))
    out = torch.full((dims[0] * dims[1] * dims[2] + 64,), 7.0, dtype=torch.float32, device="cuda")
    gg.refine_noise(parent, 1, "2", (2, 4, 6), (4, 2, 6), out=out[: dims[0] * dims[1] * dims[2]].view(dims))
    torch.cuda.synchronize()
    assert torch.all(out[-64:] == 7.0)
    assert not torch.any(out[:-64] == 7.0)


def test_fullsize_768_to_1536_fp32_sampled(gg):
    """768^3 -> 1536^3 doubling (FP32), the parent being the library's own
    white noise: 96 random patches against the oracle, and the moments of
    the whole child field (unit white noise)."""
    n, kind = 768, "2"
    plan = gg.Plan(n, 1000.0, dict(omega_m=0.3, h=0.7, n_s=0.96, sigma_8=0.8, tf="bbks",
                                   omega_l=-1.0, omega_b=0.049, t_cmb=2.7255), 50.0, "f32")
    parent = plan.white_noise(seed=1)
    child = gg.refine_noise(parent, 2, kind)
    torch.cuda.synchronize()
    assert tuple(child.shape) == (1536, 1536, 1536)
    rng = np.random.default_rng(0)
    gp = rng.integers(0, n // 2, size=(96, 3))
    gp[0] = (0, 0, 0)
    gp[1] = (n // 2 - 1,) * 3
    gpt = torch.tensor(gp, device="cuda")
    o2 = torch.arange(2, device="cuda")
    o4 = torch.arange(4, device="cuda")
    px = gpt[:, 0, None] * 2 + o2
    py = gpt[:, 1, None] * 2 + o2
    pz = gpt[:, 2, None] * 2 + o2
    v = parent[px[:, :, None, None], py[:, None, :, None], pz[:, None, None, :]].double().cpu().numpy()
    cx = gpt[:, 0, None] * 4 + o4
    cy = gpt[:, 1, None] * 4 + o4
    cz = gpt[:, 2, None] * 4 + o4
    got = child[cx[:, :, None, None], cy[:, None, :, None], cz[:, None, None, :]].double().cpu().numpy()
    want = oref.refine_patches(v, kind, 2, n, gp)
    assert rel_l2(got, want) < 1e-6
    assert np.abs(got - want).max() < 1e-3
    s1 = s2 = 0.0
    for i in range(0, 1536, 96):  # FP64 sums, slab by slab
        slab = child[i:i + 96].double()
        s1 += slab.sum().item()
        s2 += (slab * slab).sum().item()
        del slab
    cells = 1536 ** 3
    m = s1 / cells
    var = s2 / cells - m * m
    assert abs(m) < 5 / cells ** 0.5
    assert abs(var - 1) < 5 * (2 / cells) ** 0.5
    del child, parent
    plan.close()
    torch.cuda.empty_cache()
