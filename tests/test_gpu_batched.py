"""The batched form: many realizations as one CUDA graph of batched launches.

Every realization of a batch must equal the solo gg_zeldovich run with its
seed, bit for bit (the noise is keyed by (seed, cell index) and the batched
launches run the same butterflies), including after the graph is replayed
with new seeds and output buffers. The 48-realization workload (N cycling
128/192/256/384, L = N Mpc/h, seeds 1..48) is checked on one realization of
each size.
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


def _solo(gg, w, seed):
    plan = gg.Plan(w["n"], w["box"], w["cosmo"], w["z_init"], w.get("prec", "f32"))
    out = plan.zeldovich(seed=seed)
    plan.sync()
    res = {k: [t.cpu().numpy() for t in out[k]] for k in ("psi", "pos", "vel")}
    plan.close()
    return res


def test_small_mixed_batch_equals_solo_runs(gg):
    specs = []
    for i, n in enumerate((32, 48, 64, 32, 48, 64, 32)):
        specs.append(dict(n=n, box=float(n), cosmo=BBKS, z_init=50.0,
                          prec="f64" if i == 6 else "f32"))
    b = gg.Batch(specs)
    assert b.groups == 4
    out = b.empty_outputs(psi=True)
    for seeds in ([1, 2, 3, 4, 5, 6, 7], [21, 22, 23, 24, 25, 26, 27]):
        b.run(seeds, out)
        b.sync()
        for i, w in enumerate(specs):
            want = _solo(gg, w, seeds[i])
            for k in ("psi", "pos", "vel"):
                for j in range(3):
                    assert np.array_equal(out[k][i][j].cpu().numpy(), want[k][j]), (i, k, j)
    # one launch per pass and group: z forward, y forward, x, two y inverse
    # passes (two-output passes may split), three z inverse passes
    assert 8 * b.groups <= b.launches() <= 10 * b.groups
    b.close()


def test_partial_outputs(gg):
    specs = [dict(n=64, box=64.0, cosmo=BBKS, z_init=50.0)] * 3
    b = gg.Batch(specs)
    out = b.empty_outputs(psi=False, pos=True, vel=False)
    out["pos"][1] = [None, out["pos"][1][1], None]
    b.run([5, 6, 7], out)
    b.sync()
    want = _solo(gg, specs[1], 6)
    assert np.array_equal(out["pos"][1][1].cpu().numpy(), want["pos"][1])
    want0 = _solo(gg, specs[0], 5)
    for j in range(3):
        assert np.array_equal(out["pos"][0][j].cpu().numpy(), want0["pos"][j])
    b.close()


def test_batched_48_workload(gg):
    from paper_2511_10353_gb300.workloads import batched_realizations
    specs = batched_realizations()
    b = gg.Batch(specs)
    assert b.groups == 4 and b.cells == 12 * (128 ** 3 + 192 ** 3 + 256 ** 3 + 384 ** 3)
    b.autotune(1)
    out = b.empty_outputs()
    seeds = [w["seed"] for w in specs]
    b.run(seeds, out)
    b.sync()
    for i in (0, 5, 10, 47):
        want = _solo(gg, specs[i], seeds[i])
        for k in ("pos", "vel"):
            for j in range(3):
                assert np.array_equal(out[k][i][j].cpu().numpy(), want[k][j]), (i, k, j)
    # members of the two largest sizes against the oracle directly (not only
    # against solo runs of the same kernels): realization 3 (256^3, seed 3)
    # and realization 4 (384^3, seed 4), FP32 within 1e-5 relative L2
    from tests.gpu_helpers import min_image, rel_l2, run_oracle
    for i in (2, 3):
        w = specs[i]
        ora = run_oracle(w, seed=seeds[i])
        for j in range(3):
            vel = out["vel"][i][j].cpu().numpy()
            assert rel_l2(vel, ora["vel"][j]) < 1e-5, (i, j)
            pos = out["pos"][i][j].cpu().numpy().astype(np.float64)
            d = min_image(pos - ora["pos"][j], w["box"])
            ulp = np.spacing(np.float32(w["box"]))
            assert np.abs(d).max() < 4 * ulp + 1e-5 * np.abs(ora["psi"][j]).max(), (i, j)
        del ora
    b.close()


def _equal_outputs(a, b, count):
    for k in ("psi", "pos", "vel"):
        for i in range(count):
            for j in range(3):
                x, y = a[k][i][j], b[k][i][j]
                if x is None:
                    continue
                assert torch.equal(x, y), (k, i, j)


def test_persistent_launch_equals_pass_launches(gg):
    """The whole batch as one persistent launch (work items taken in order,
    per-realization pass counters) computes the same butterflies as the
    per-pass launches: bit-identical outputs, with new seeds on replay."""
    specs = []
    for i, n in enumerate((64, 128, 192, 384, 64, 128)):  # four parameter groups
        specs.append(dict(n=n, box=float(n), cosmo=BBKS, z_init=50.0))
    b = gg.Batch(specs)
    ref = b.empty_outputs(psi=True)
    got = b.empty_outputs(psi=True)
    for seeds in ([1, 2, 3, 4, 5, 6], [11, 12, 13, 14, 15, 16]):
        b.set_persistent(False)
        b.run(seeds, ref)
        b.sync()
        b.set_persistent(True)
        b.run(seeds, got)
        b.sync()
        assert b.launches() == 1
        _equal_outputs(got, ref, len(specs))
    b.close()


def test_persistent_partial_outputs(gg):
    """Partial outputs take the generic z inverse in the persistent launch."""
    specs = [dict(n=128, box=128.0, cosmo=BBKS, z_init=50.0)] * 3
    b = gg.Batch(specs)
    b.set_persistent(True)
    out = b.empty_outputs(psi=False, pos=True, vel=False)
    out["pos"][1] = [None, out["pos"][1][1], None]
    b.run([5, 6, 7], out)
    b.sync()
    want = _solo(gg, specs[1], 6)
    assert np.array_equal(out["pos"][1][1].cpu().numpy(), want["pos"][1])
    want0 = _solo(gg, specs[0], 5)
    for j in range(3):
        assert np.array_equal(out["pos"][0][j].cpu().numpy(), want0["pos"][j])
    b.close()


def test_persistent_48_workload_against_oracle(gg):
    """The 48-realization workload as one persistent launch: bit-identical to
    the per-pass launches, and its 384^3 member within FP32 parity of the
    FP64 oracle."""
    from paper_2511_10353_gb300.workloads import batched_realizations
    from tests.gpu_helpers import min_image, rel_l2, run_oracle
    specs = batched_realizations()
    b = gg.Batch(specs)
    seeds = [w["seed"] for w in specs]
    ref = b.empty_outputs()
    got = b.empty_outputs()
    b.run(seeds, ref)
    b.sync()
    b.set_persistent(True)
    b.run(seeds, got)
    b.sync()
    assert b.launches() == 1
    _equal_outputs(got, ref, len(specs))
    del ref
    w = specs[7]  # 384^3, seed 8
    ora = run_oracle(w, seed=seeds[7])
    for j in range(3):
        assert rel_l2(got["vel"][7][j].cpu().numpy(), ora["vel"][j]) < 1e-5, j
        pos = got["pos"][7][j].cpu().numpy().astype(np.float64)
        d = min_image(pos - ora["pos"][j], w["box"])
        assert np.abs(d).max() < 4 * np.spacing(np.float32(w["box"])) + 1e-5 * np.abs(ora["psi"][j]).max()
    b.close()


def test_persistent_rejects_unsupported_batches(gg):
    specs = [dict(n=48, box=48.0, cosmo=BBKS, z_init=50.0)]
    b = gg.Batch(specs)
    with pytest.raises(gg.GGError) as ex:
        b.set_persistent(True)
    assert ex.value.status == gg.GG_EINVAL
    b.close()
