"""The tile autotuner: every variant computes the same numbers.

Variants change how the transforms are tiled over threads (elements per
thread, columns per tile, lines per CTA, one or two outputs per launch, CTA
or warp barriers between stages), not
the butterflies themselves, so the results are bit-identical across variants;
the autotuner keeps a valid variant for every pass and the path still matches
the oracle afterwards.
"""
import itertools

import numpy as np
import pytest

from tests.gpu_helpers import rel_l2, run_oracle

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


@pytest.mark.parametrize("n,prec", [(64, "f32"), (128, "f32"), (192, "f32"), (384, "f32"), (512, "f32"),
                                    (64, "f64")])
def test_variants_bit_identical(gg, n, prec):
    plan = gg.Plan(n, float(n), BBKS, 50.0, prec)
    ref = None
    for v in range(4):
        a = min(v, 2)  # the strided passes have three variants, the z passes four
        plan.set_variants([v, a, a, a, a, v])
        out = plan.zeldovich(seed=7)
        plan.sync()
        got = [out[k][j].cpu().numpy() for k in ("psi", "pos", "vel") for j in range(3)]
        if ref is None:
            ref = got
        else:
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), v


def test_autotune_then_parity(gg):
    n = 128
    plan = gg.Plan(n, 128.0, BBKS, 50.0, "f32")
    v = plan.autotune(2)
    assert len(v) == 6 and all(0 <= x <= 2 for x in v[1:5]) and 0 <= v[0] <= 3 and 0 <= v[5] <= 3
    out = plan.zeldovich(seed=3)
    plan.sync()
    ora = run_oracle(dict(n=n, box=128.0, cosmo=BBKS, z_init=50.0), seed=3)
    for j in range(3):
        assert rel_l2(out["psi"][j].cpu().numpy(), ora["psi"][j]) < 1e-5


def test_set_variants_rejects_out_of_range(gg):
    plan = gg.Plan(32, 32.0, BBKS, 50.0, "f32")
    with pytest.raises(gg.GGError):
        plan.set_variants([0, 0, 3, 0, 0, 0])
    with pytest.raises(gg.GGError):
        plan.set_variants([4, 0, 0, 0, 0, 0])
