"""The 1536^3 precision workload: FP32 path at full size, in the bench's launch shape.

1536^3, L = 2000 Mpc/h, Eisenstein-Hu no-wiggle (Om=.31, h=.68, ns=.965,
s8=.81), z = 100. The complete FP64 oracle does not fit this host's memory at
this size, so:
* the Philox words and W values of sampled cells are compared with the oracle
  one by one (bit-exact words);
* a planted Fourier mode W = cos(k0.x) must give psi = -s k0/|k0|^2 sin(k0.x)
  with s from the oracle's P(k0) and growth, checked on sampled cells;
* each displacement component of the FP32 path is within 1e-5 relative L2
  of the GPU FP64 path (which the other tests pin to the oracle at <= 1e-12);
* the strided passes' tile variants agree bit for bit;
* Eq. 4's top hat at this size: the planted mode comes out unchanged above
  the cut and vanishes below it;
* the pos + vel-only path agrees bit for bit with the path that also writes
  psi;
* a random field of 64 planted Fourier modes (random amplitudes and phases,
  modes with |m_j| = N/2 - 1, modes at multiples of 3, modes with all three
  m_j != 0) gives, at 10^5 sampled cells, the closed-form sum of the modes'
  displacements built from the oracle's P(k) and growth, for psi, pos and vel
  of the FP32 path (1e-5) and psi of the FP64 path (1e-11): an
  oracle-anchored check of both 1536 codelets on a field with many modes.
"""
import math

import numpy as np
import pytest

from oracle import noise as onoise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EH_NW = dict(omega_m=0.31, h=0.68, n_s=0.965, sigma_8=0.81, tf="eh_nw", omega_l=-1.0,
             omega_b=0.049, t_cmb=2.7255)
N, BOX, Z = 1536, 2000.0, 100.0


@pytest.fixture(scope="module")
def gg():
    from paper_2511_10353_gb300 import build
    build.build(verbose=False)
    import paper_2511_10353_gb300 as m
    if torch.cuda.get_device_properties(0).total_memory < 200e9:
        pytest.skip("needs a GPU with >= 200 GB")
    return m


def _sample_idx(count, seed=0):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N ** 3, size=count, replace=False)).astype(np.int64)


def test_noise_words_and_values_sampled(gg):
    idx = _sample_idx(200000)
    groups = np.unique(idx >> 2)
    words = gg.noise_bits(1, 0, int(groups.max()) + 1)  # all groups up to the largest sampled
    got = words.cpu().numpy().view(np.uint32)[groups]
    assert np.array_equal(got, onoise.noise_bits(1, groups.astype(np.uint64)))
    del words
    plan = gg.Plan(N, BOX, EH_NW, Z, "f32")
    w = plan.white_noise(seed=1).reshape(-1)
    vals = w[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    want = onoise.noise_at(1, idx)
    assert np.sqrt(np.mean((vals - want) ** 2)) < 1e-6 and np.abs(vals - want).max() < 1e-3
    del w
    plan.close()
    torch.cuda.empty_cache()


def test_planted_mode_sampled(gg):
    from tests.oracle_cases import cosmology_from
    c = cosmology_from(EH_NW)
    m0 = (3, -7, 11)
    plan = gg.Plan(N, BOX, EH_NW, Z, "f32")
    i = torch.arange(N, device="cuda", dtype=torch.float64)
    ph = (2 * math.pi / N) * (m0[0] * i[:, None, None] + m0[1] * i[None, :, None])
    noise = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    for ix in range(0, N, 64):  # cos(k0.x) written in slabs to bound the temporaries
        noise[ix:ix + 64] = torch.cos(ph[ix:ix + 64] + (2 * math.pi / N) * m0[2] * i[None, None, :]).float()
    del ph
    psi = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    idx = _sample_idx(100000, 1)
    ix, iy, iz = idx // (N * N), (idx // N) % N, idx % N
    phase = 2 * math.pi * (m0[0] * ix + m0[1] * iy + m0[2] * iz) / N
    k0 = 2 * math.pi / BOX * np.array(m0, dtype=float)
    kk = math.sqrt((k0 ** 2).sum())
    s = plan.info["growth"] * math.sqrt(c.power(kk) * N ** 3 / BOX ** 3)
    for j in range(3):
        out = {"psi": [psi if a == j else None for a in range(3)], "pos": [None] * 3, "vel": [None] * 3}
        plan.zeldovich(noise=noise, out=out)
        plan.sync()
        got = psi.reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
        want = -s * k0[j] / kk ** 2 * np.sin(phase)
        scale = s * abs(k0[j]) / kk ** 2
        assert np.abs(got - want).max() < 2e-5 * scale, j
    del noise, psi
    plan.close()
    torch.cuda.empty_cache()


def test_fp32_within_1e5_of_fp64(gg):
    errs = []
    for j in range(3):
        p32 = gg.Plan(N, BOX, EH_NW, Z, "f32")
        a = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
        p32.zeldovich(seed=1, out={"psi": [a if c == j else None for c in range(3)],
                                   "pos": [None] * 3, "vel": [None] * 3})
        p32.sync()
        p32.close()
        torch.cuda.empty_cache()
        p64 = gg.Plan(N, BOX, EH_NW, Z, "f64")
        b = torch.empty((N, N, N), dtype=torch.float64, device="cuda")
        p64.zeldovich(seed=1, out={"psi": [b if c == j else None for c in range(3)],
                                   "pos": [None] * 3, "vel": [None] * 3})
        p64.sync()
        p64.close()
        num = den = 0.0
        for ix in range(0, N, 128):
            d = a[ix:ix + 128].double() - b[ix:ix + 128]
            num += float((d * d).sum())
            den += float((b[ix:ix + 128] ** 2).sum())
        errs.append(math.sqrt(num / den))
        del a, b
        torch.cuda.empty_cache()
    assert max(errs) < 1e-5, errs


def test_strided_variants_bit_identical(gg):
    """Strided-pass tile variants 0 and 1 at this size park the handed-off
    spectrum in shared memory and take both outputs of the x and y inverse
    passes from one launch (the next tile's copy issued during the last
    output); variant 2 keeps the spectrum in registers. The butterflies are
    the same, so all three components agree bit for bit."""
    plan = gg.Plan(N, BOX, EH_NW, Z, "f32")
    ref = [torch.empty((N, N, N), dtype=torch.float32, device="cuda") for _ in range(3)]
    cur = [torch.empty((N, N, N), dtype=torch.float32, device="cuda") for _ in range(3)]
    for i, a in enumerate((2, 0, 1)):
        plan.set_variants([0, a, a, a, a, 0])
        plan.zeldovich(seed=2, out={"psi": ref if i == 0 else cur, "pos": [None] * 3, "vel": [None] * 3})
        plan.sync()
        if i:
            for j in range(3):
                assert torch.equal(cur[j], ref[j]), (a, j)
    assert float(ref[0].abs().max()) > 0.0
    del ref, cur
    plan.close()
    torch.cuda.empty_cache()


def test_chunk_major_layout_bit_identical(gg):
    """The chunk-major spectrum between the y passes (both tile widths of this
    size: variant 0's eight columns and variant 2's four) gives the plain
    layout's positions bit for bit."""
    plan = gg.Plan(N, BOX, EH_NW, Z, "f32")
    ref = [torch.empty((N, N, N), dtype=torch.float32, device="cuda") for _ in range(3)]
    cur = [torch.empty((N, N, N), dtype=torch.float32, device="cuda") for _ in range(3)]
    for a in (0, 2):
        plan.set_variants([0, a, a, a, a, 0])
        for lay, dst in ((False, ref), (True, cur)):
            plan.set_layout(lay)
            assert plan.layout() == lay
            plan.zeldovich(seed=4, out={"psi": [None] * 3, "pos": dst, "vel": [None] * 3})
            plan.sync()
        for j in range(3):
            assert torch.equal(cur[j], ref[j]), (a, j)
    del ref, cur
    plan.close()
    torch.cuda.empty_cache()


def test_merge_cut_planted_mode(gg):
    """Eq. 4 on the full-size grid (the x pass's cut instantiation, with the
    spectrum parked in shared memory and both outputs from one launch): with
    no coarse grids to add, a planted mode with |k0| r_s >= 1 gives the plain
    path's analytic displacement and one with |k0| r_s < 1 gives zero."""
    from tests.oracle_cases import cosmology_from
    c = cosmology_from(EH_NW)
    m0 = (3, -7, 11)
    plan = gg.Plan(N, BOX, EH_NW, Z, "f32")
    i = torch.arange(N, device="cuda", dtype=torch.float64)
    ph = (2 * math.pi / N) * (m0[0] * i[:, None, None] + m0[1] * i[None, :, None])
    noise = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    for ix in range(0, N, 64):
        noise[ix:ix + 64] = torch.cos(ph[ix:ix + 64] + (2 * math.pi / N) * m0[2] * i[None, None, :]).float()
    del ph
    psi = [torch.empty((N, N, N), dtype=torch.float32, device="cuda") for _ in range(3)]
    idx = _sample_idx(100000, 2)
    ix, iy, iz = idx // (N * N), (idx // N) % N, idx % N
    phase = 2 * math.pi * (m0[0] * ix + m0[1] * iy + m0[2] * iz) / N
    k0 = 2 * math.pi / BOX * np.array(m0, dtype=float)
    kk = math.sqrt((k0 ** 2).sum())
    s = plan.info["growth"] * math.sqrt(c.power(kk) * N ** 3 / BOX ** 3)
    it = torch.from_numpy(idx).cuda()
    for r_s in (2.0 / kk, 0.5 / kk):  # kept, removed
        plan.zeldovich_merge([None] * 3, r_s, noise=noise,
                             out={"psi": psi, "pos": [None] * 3, "vel": [None] * 3})
        plan.sync()
        for j in range(3):
            got = psi[j].reshape(-1)[it].cpu().numpy().astype(np.float64)
            scale = s * abs(k0[j]) / kk ** 2
            want = -s * k0[j] / kk ** 2 * np.sin(phase) if r_s * kk >= 1 else 0.0 * phase
            assert np.abs(got - want).max() < 2e-5 * scale, (r_s, j)
    del noise, psi
    plan.close()
    torch.cuda.empty_cache()


def test_pos_vel_only_bit_identical(gg):
    """The bench's z inverse instantiation (pos + vel only, component fixed
    at compile time) against the run-time-flag kernel that also writes psi:
    the same positions and velocities bit for bit, component by component."""
    plan = gg.Plan(N, BOX, EH_NW, Z, "f32")
    e = lambda: torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    pos, vel, pos2, vel2, psi = e(), e(), e(), e(), e()
    for j in range(3):
        sel = lambda t: [t if c == j else None for c in range(3)]
        plan.zeldovich(seed=3, out={"psi": [None] * 3, "pos": sel(pos), "vel": sel(vel)})
        plan.zeldovich(seed=3, out={"psi": sel(psi), "pos": sel(pos2), "vel": sel(vel2)})
        plan.sync()
        assert torch.equal(pos, pos2) and torch.equal(vel, vel2), j
    del pos, vel, pos2, vel2, psi
    plan.close()
    torch.cuda.empty_cache()


def _modes(seed=5, count=64):
    """Random distinct modes m (|m_j| <= N/2 - 1, m != 0), amplitudes, phases."""
    rng = np.random.default_rng(seed)
    h = N // 2 - 1
    out = set()
    while len(out) < count:
        t = len(out)
        m = rng.integers(-h, h + 1, size=3)
        if t < 12:  # an edge of the kept band on one axis
            m[t % 3] = h if t % 2 else -h
        elif t < 24:  # multiples of 3 on every axis (radix-3 stage inputs)
            m = 3 * rng.integers(-(h // 3), h // 3 + 1, size=3)
        elif t < 40:  # low |m|: the largest displacements
            m = rng.integers(-8, 9, size=3)
        if (m != 0).all() or (t < 12 and m.any()):
            out.add(tuple(int(v) for v in m))
    modes = np.array(sorted(out), dtype=np.int64)
    return modes, rng.uniform(0.5, 2.0, size=count), rng.uniform(0.0, 2 * math.pi, size=count)


def _mode_noise(modes, amp, ph, dtype):
    """W(x_n) = sum_t a_t cos(2 pi m_t.n / N + phi_t) on the device, in FP64
    (phases reduced exactly in integers), stored in `dtype`."""
    noise = torch.empty((N, N, N), dtype=dtype, device="cuda")
    i = torch.arange(N, device="cuda", dtype=torch.int64)
    for x0 in range(0, N, 64):
        acc = torch.zeros((64, N, N), dtype=torch.float64, device="cuda")
        for (mx, my, mz), a, p in zip(modes.tolist(), amp.tolist(), ph.tolist()):
            r = (mx * i[x0:x0 + 64, None, None] + my * i[None, :, None] + mz * i[None, None, :]) % N
            acc += a * torch.cos(r.double() * (2 * math.pi / N) + p)
            del r
        noise[x0:x0 + 64] = acc.to(dtype)
        del acc
    return noise


def _mode_psi(modes, amp, ph, idx, c, growth):
    """Closed form at cells idx: psi_j = -sum_t a_t s_t k_j/|k|^2 sin(k.x + phi_t),
    s_t = D sqrt(P(|k_t|) N^3 / V) (Eqs. 1-2 for one planted mode, summed)."""
    ix, iy, iz = idx // (N * N), (idx // N) % N, idx % N
    psi = np.zeros((3, idx.size))
    for (mx, my, mz), a, p in zip(modes.tolist(), amp.tolist(), ph.tolist()):
        k = 2 * math.pi / BOX * np.array([mx, my, mz], dtype=float)
        kk = math.sqrt((k ** 2).sum())
        s = growth * math.sqrt(float(c.power(kk)) * N ** 3 / BOX ** 3)
        r = (mx * ix + my * iy + mz * iz) % N
        sn = np.sin(2 * math.pi * r / N + p)
        for j in range(3):
            psi[j] -= a * s * k[j] / kk ** 2 * sn
    return psi


def test_multimode_field_closed_form_fp32(gg):
    from tests.oracle_cases import cosmology_from
    c = cosmology_from(EH_NW)
    a_init = 1.0 / (1.0 + Z)
    modes, amp, ph = _modes()
    noise = _mode_noise(modes, amp, ph, torch.float32)
    plan = gg.Plan(N, BOX, EH_NW, Z, "f32")
    e = lambda: torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    out = {"psi": [e() for _ in range(3)], "pos": [e() for _ in range(3)],
           "vel": [e() for _ in range(3)]}
    plan.zeldovich(noise=noise, out=out)
    plan.sync()
    del noise
    idx = _sample_idx(100000, 3)
    want = _mode_psi(modes, amp, ph, idx, c, c.growth(a_init))
    vfac = c.velocity_factor(a_init)
    it = torch.from_numpy(idx).cuda()
    ulp = np.spacing(np.float32(BOX))
    for j in range(3):
        got = {k: out[k][j].reshape(-1)[it].cpu().numpy().astype(np.float64)
               for k in ("psi", "pos", "vel")}
        rel = lambda x, y: np.linalg.norm(x - y) / np.linalg.norm(y)
        assert rel(got["psi"], want[j]) < 1e-5, j
        assert rel(got["vel"], vfac * want[j]) < 1e-5, j
        q = (np.array([idx // (N * N), (idx // N) % N, idx % N])[j] + 0.5) * (BOX / N)
        d = got["pos"] - (q + want[j])
        d -= BOX * np.round(d / BOX)
        assert np.abs(d).max() < 4 * ulp + 1e-5 * np.abs(want[j]).max(), j
    del out
    plan.close()
    torch.cuda.empty_cache()


def test_multimode_field_closed_form_fp64(gg):
    from tests.oracle_cases import cosmology_from
    c = cosmology_from(EH_NW)
    modes, amp, ph = _modes()
    noise = _mode_noise(modes, amp, ph, torch.float64)
    plan = gg.Plan(N, BOX, EH_NW, Z, "f64")
    psi = torch.empty((N, N, N), dtype=torch.float64, device="cuda")
    idx = _sample_idx(100000, 4)
    want = _mode_psi(modes, amp, ph, idx, c, c.growth(1.0 / (1.0 + Z)))
    it = torch.from_numpy(idx).cuda()
    for j in range(3):
        plan.zeldovich(noise=noise, out={"psi": [psi if a == j else None for a in range(3)],
                                         "pos": [None] * 3, "vel": [None] * 3})
        plan.sync()
        got = psi.reshape(-1)[it].cpu().numpy()
        assert np.linalg.norm(got - want[j]) / np.linalg.norm(want[j]) < 1e-11, j
    del noise, psi
    plan.close()
    torch.cuda.empty_cache()
