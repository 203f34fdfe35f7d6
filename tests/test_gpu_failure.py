"""Failure detection of the device-side waits, without a GPU fault.

Every copy wait of the transform passes is bounded (the global timer); when
it runs out the CTA records GG_ETIMEOUT in the plan's error word and
returns. gg_test_arm_fault makes the next y forward pass issue none of its
tile copies, so every CTA's first wait runs out after a few milliseconds.
The test checks that gg_sync reports GG_ETIMEOUT, that the error is cleared,
and that the next call on the same plan gives the normal result, for the
size-specialised kernel (N = 64) and the run-time kernel (N = 48).
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("n,prec", [(64, "f32"), (48, "f32"), (64, "f64")])
def test_copy_wait_timeout_is_reported_and_plan_recovers(gg, n, prec):
    plan = gg.Plan(n, float(n), BBKS, 50.0, prec)
    want = plan.zeldovich(seed=3, pos=False, vel=False)["psi"]
    plan.sync()
    want = [t.clone() for t in want]
    plan.arm_fault("skip_copy", wait_us=3000)
    plan.zeldovich(seed=3, pos=False, vel=False)
    with pytest.raises(gg.GGError) as ex:
        plan.sync()
    assert ex.value.status == gg.GG_ETIMEOUT
    plan.sync()  # the error word was cleared
    got = plan.zeldovich(seed=3, pos=False, vel=False)["psi"]
    plan.sync()
    for j in range(3):
        assert torch.equal(got[j], want[j]), j
    plan.close()


def test_disarm_and_argument_checks(gg):
    plan = gg.Plan(32, 32.0, BBKS, 50.0, "f32")
    with pytest.raises(gg.GGError) as ex:
        plan.arm_fault("skip_copy", wait_us=0)
    assert ex.value.status == gg.GG_EINVAL
    plan.arm_fault("skip_copy", wait_us=1000)
    plan.arm_fault("none")
    out = plan.zeldovich(seed=1, pos=False, vel=False)["psi"]
    plan.sync()
    assert np.isfinite(out[0].cpu().numpy()).all()
    plan.close()


def test_persistent_batch_wait_timeout_and_recovery(gg):
    """The persistent batched launch: one work item never counts itself done,
    so every wait on its pass gives up after a few milliseconds; the run
    stops, gg_batch_sync reports GG_ETIMEOUT, and the next run (the graph
    captured again without the fault) equals the normal result."""
    specs = [dict(n=64, box=64.0, cosmo=BBKS, z_init=50.0),
             dict(n=128, box=128.0, cosmo=BBKS, z_init=50.0)]
    b = gg.Batch(specs)
    b.set_persistent(True)
    ref = b.empty_outputs()
    b.run([1, 2], ref)
    b.sync()
    ref = {k: [[t.clone() if t is not None else None for t in r] for r in v] for k, v in ref.items()}
    out = b.empty_outputs()
    b.arm_fault("stall_count", wait_us=3000)
    b.run([1, 2], out)
    with pytest.raises(gg.GGError) as ex:
        b.sync()
    assert ex.value.status == gg.GG_ETIMEOUT
    b.run([1, 2], out)
    b.sync()
    for k in ("pos", "vel"):
        for i in range(2):
            for j in range(3):
                assert torch.equal(out[k][i][j], ref[k][i][j]), (k, i, j)
    b.close()
