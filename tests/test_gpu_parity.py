"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: relative L2 error <= 1e-4 for the FP32 path (FP64 only in tile
references), element by element on identical seeded inputs; the oracle uses
its own plan.  HHFFBPA must also stay within -30 dB NRMSE of BPA.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-4


@pytest.fixture(scope="module")
def hh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_23568_gb300 as m

    m.lib()
    return m


def _scene(name):
    s = synth.CONFIGS[name]()
    e = synth.scene_echo(s, device="cuda")
    return s, e


def _rel(gpu, ref):
    return oracle.rel_l2(gpu.detach().cpu().numpy().astype(np.complex128).ravel(), np.asarray(ref).ravel())


@pytest.mark.parametrize("name", ["small", "tiny"])
def test_bpa_matches_oracle(hh, name):
    s, e = _scene(name)
    img = hh.bpa_form_image(s.traj, s.freqs, s.grid, e)
    torch.cuda.synchronize()
    ref = oracle.bpa_rc(s.traj, s.freqs, e.cpu().numpy(), s.grid.points()).reshape(s.grid.shape)
    assert _rel(img, ref) < REL_TOL


CFGS = [("small", dict(leaf_size=16)), ("small", dict(leaf_size=8, merge_factor=2, taps=4, eta=1.5)),
        ("tiny", dict(leaf_size=32)), ("tiny", dict(leaf_size=64, taps=4))]


@pytest.mark.parametrize("name,cfg", CFGS)
def test_hhffbpa_matches_oracle(hh, name, cfg):
    s, e = _scene(name)
    plan = hh.Plan(s.traj, s.freqs, s.grid, **cfg)
    img = plan.form_image(e)
    cnt = plan.counters()
    assert cnt["gate_miss"] == 0 and cnt["errors"] == 0
    op = oracle.Plan(s.traj, s.freqs, s.grid, **cfg)
    ref, st = op.hhffbpa(e.cpu().numpy())
    ref = ref.reshape(s.grid.shape)
    rel = _rel(img, ref)
    assert rel < REL_TOL, (rel, cnt, st)
    bpa = oracle.bpa_rc(s.traj, s.freqs, e.cpu().numpy(), s.grid.points()).reshape(s.grid.shape)
    if cfg.get("taps", 6) == 6 and cfg.get("eta", 2.0) >= 2.0:  # the accurate settings
        assert oracle.nrmse_db(img.cpu().numpy(), bpa) < -30


def test_inline_fallbacks_match_oracle(hh):
    """A plan whose sparse lattices (eta 1.25) leave footprints on infeasible samples: the
    exact fallbacks evaluated in place by the merge blocks, against the oracle."""
    s, e = _scene("tiny")
    cfg = dict(leaf_size=32, eta=1.25)
    plan = hh.Plan(s.traj, s.freqs, s.grid, **cfg)
    img = plan.form_image(e)
    cnt = plan.counters()
    assert cnt["fallbacks"] > 0 and cnt["infeasible"] > 0, cnt
    ref, st = oracle.Plan(s.traj, s.freqs, s.grid, **cfg).hhffbpa(e.cpu().numpy())
    assert _rel(img, ref.reshape(s.grid.shape)) < REL_TOL
    assert torch.equal(img, plan.form_image(e))  # fallback sums are added in a fixed order


def test_single_level_is_bpa(hh):
    s, e = _scene("small")
    plan = hh.Plan(s.traj, s.freqs, s.grid, leaf_size=10 ** 6)
    assert plan.info()["n_levels"] == 1
    img = plan.form_image(e)
    ref = oracle.bpa_rc(s.traj, s.freqs, e.cpu().numpy(), s.grid.points()).reshape(s.grid.shape)
    assert _rel(img, ref) < REL_TOL


def test_host_buffers_match_device_buffers(hh):
    s, e = _scene("small")
    plan = hh.Plan(s.traj, s.freqs, s.grid, leaf_size=16)
    dev = plan.form_image(e).cpu()
    host_in = e.cpu().pin_memory()
    host_out = torch.empty(s.grid.shape, dtype=torch.complex64).pin_memory()
    plan.form_image(host_in, out=host_out)
    torch.cuda.synchronize()
    assert torch.equal(dev, host_out)
    b_dev = hh.bpa_form_image(s.traj, s.freqs, s.grid, e).cpu()
    b_host = hh.bpa_form_image(s.traj, s.freqs, s.grid, e.cpu())
    torch.cuda.synchronize()
    assert torch.equal(b_dev, b_host)


def test_repeat_calls_are_deterministic(hh):
    s, e = _scene("small")
    plan = hh.Plan(s.traj, s.freqs, s.grid, leaf_size=16)
    a = plan.form_image(e).clone()
    b = plan.form_image(e)
    assert torch.equal(a, b)


def test_edge_single_voxel_and_thin_grid(hh):
    s, e = _scene("small")
    for g in [synth.Grid(0.001, -0.002, 0.19, 1e-3, 1e-3, 1e-2, 1, 1, 1),
              synth.Grid(-0.03, 0.0, 0.18, 2e-3, 1e-3, 1e-2, 33, 1, 2)]:
        plan = hh.Plan(s.traj, s.freqs, g, leaf_size=16)
        img = plan.form_image(e)
        ref, _ = oracle.Plan(s.traj, s.freqs, g, leaf_size=16).hhffbpa(e.cpu().numpy(), g.points())
        assert _rel(img, ref.reshape(g.shape)) < REL_TOL
        bref = oracle.bpa_rc(s.traj, s.freqs, e.cpu().numpy(), g.points()).reshape(g.shape)
        assert _rel(hh.bpa_form_image(s.traj, s.freqs, g, e), bref) < REL_TOL


def _cluster(grid, centre, half=(3, 3, 2)):
    a, b, c = centre
    idx = []
    for dz in range(-half[2], half[2]):
        for dy in range(-half[1], half[1]):
            for dx in range(-half[0], half[0]):
                x, y, z = a + dx, b + dy, c + dz
                if 0 <= x < grid.nx and 0 <= y < grid.ny and 0 <= z < grid.nz:
                    idx.append((z * grid.ny + y) * grid.nx + x)
    return np.unique(np.array(idx))


def _clusters(grid, centres, half=(3, 3, 2)):
    return np.unique(np.concatenate([_cluster(grid, c, half) for c in centres]))


def _assert_each_cluster(img, grid, centres, ref_of, what):
    """Each voxel cluster on its own (a bright centre cannot hide an error at a corner):
    relative L2 and max |gpu - ref| / max |ref| both within REL_TOL."""
    for centre in centres:
        idx = _cluster(grid, centre)
        ref = ref_of(idx)
        got = img.reshape(-1)[torch.as_tensor(idx, device=img.device)].cpu().numpy().astype(np.complex128)
        rel = oracle.rel_l2(got, ref)
        mx = np.abs(got - ref).max() / np.abs(ref).max()
        assert rel < REL_TOL and mx < REL_TOL, (what, centre, rel, mx)


def test_mid_sampled_parity(hh):
    """Full-size mid workload (leaf 64: deferred fallbacks at every merge level); the oracle
    evaluates clustered voxel samples (demand-driven) and a few BPA voxels."""
    s, e = _scene("mid")
    g = s.grid
    plan = hh.Plan(s.traj, s.freqs, g, leaf_size=64)
    img = plan.form_image(e)
    cnt = plan.counters()
    # large groups of exact fallbacks are queued and evaluated after their merge, then added
    # per output in child order: deterministic
    assert cnt["fallbacks_deferred"] > 0 and cnt["queue_full"] == 0, cnt
    assert torch.equal(img, plan.form_image(e).clone())
    ec = e.cpu().numpy()
    centres = [(128, 128, 32), (20, 230, 5), (250, 10, 60)]
    op = oracle.Plan(s.traj, s.freqs, g, leaf_size=64)
    _assert_each_cluster(img, g, centres, lambda i: op.hhffbpa(ec, g.points(i))[0], ("mid", cnt))
    idx = _clusters(g, centres)
    bi = idx[::11]
    bref = oracle.bpa_rc(s.traj, s.freqs, ec, g.points(bi))
    bimg = hh.bpa_form_image(s.traj, s.freqs, g, e)
    bgot = bimg.reshape(-1)[torch.as_tensor(bi, device=img.device)].cpu().numpy()
    assert oracle.rel_l2(bgot.astype(np.complex128), bref) < REL_TOL
    # accuracy of the fast method over the whole volume
    assert oracle.nrmse_db(img.cpu().numpy(), bimg.cpu().numpy()) < -30


@pytest.mark.parametrize("leaf", [1024, 256])
def test_large_sampled_parity_benchmark_plan(hh, leaf):
    """Full-size large workload in the benchmark's launch configuration and plan (leaf 1024,
    eta 1.5, 6 taps: four levels) and with leaf 256 (five levels): voxel clusters at the
    centre, an edge and a corner of the grid against the oracle (demand-driven), a subset
    against the oracle's BPA-RC, and the whole volume against the GPU's direct BPA (-30 dB)."""
    s, e = _scene("large")
    g = s.grid
    cfg = dict(leaf_size=leaf, eta=1.5)
    plan = hh.Plan(s.traj, s.freqs, g, **cfg)
    img = plan.form_image(e)
    cnt = plan.counters()
    assert cnt["errors"] == 0 and cnt["gate_miss"] == 0 and cnt["queue_full"] == 0, cnt
    ec = e.cpu().numpy()
    centres = [(256, 256, 64), (20, 300, 120), (500, 8, 3)]
    op = oracle.Plan(s.traj, s.freqs, g, **cfg)
    _assert_each_cluster(img, g, centres, lambda i: op.hhffbpa(ec, g.points(i))[0], ("large", cnt))
    idx = _clusters(g, centres)
    bimg = hh.bpa_form_image(s.traj, s.freqs, g, e)
    bi = idx[::13]
    bref = oracle.bpa_rc(s.traj, s.freqs, ec, g.points(bi))
    bgot = bimg.reshape(-1)[torch.as_tensor(bi, device=img.device)].cpu().numpy()
    assert oracle.rel_l2(bgot.astype(np.complex128), bref) < REL_TOL
    assert oracle.nrmse_db(img.cpu().numpy(), bimg.cpu().numpy()) < -30


@pytest.mark.parametrize("name,cfg", [("tiny", dict(leaf_size=64, taps=4)), ("large", dict(leaf_size=64))])
def test_preimage_solver_matches_oracle(hh, name, cfg):
    """The device FP32 preimage solver against the FP64 oracle's on lattice targets of leaves
    (including points near the fold at the design plane) and of the root's children."""
    s = synth.CONFIGS[name]()
    plan = hh.Plan(s.traj, s.freqs, s.grid, **cfg)
    ex = plan.export()
    oex = oracle.Plan(s.traj, s.freqs, s.grid, **cfg).export()
    ls = ex["level_start"]
    rng = np.random.default_rng(3)
    for k in [0, int(ls[1]) - 1, int(ls[1]) // 2, int(ls[-3])]:
        N, lo, eta = ex["N"][k], ex["lo"][k], ex["eta"][k]
        idx = np.stack(np.meshgrid(*[np.arange(n) for n in N], indexing="ij"), -1).reshape(-1, 3)
        if len(idx) > 20000:
            idx = idx[rng.choice(len(idx), 20000, replace=False)]
        tgt = lo + idx / eta
        g_xyz, g_ok = plan.preimages(k, tgt)
        o_xyz, o_ok = oracle.preimage(oex["rect"][k], oex["node_zbar"][k], oex["kmin"], oex["kmax"],
                                      oex["zh_floor"], oex["zh_mid"], tgt)
        zh = o_xyz[:, 2] - oex["node_zbar"][k]
        marginal = np.abs(zh - oex["zh_floor"]) < 0.02 * oex["zh_floor"]
        disagree = (g_ok != o_ok) & ~marginal
        assert disagree.sum() == 0, (k, int(disagree.sum()), int(o_ok.sum()), int(g_ok.sum()))
        both = g_ok & o_ok
        if both.any():
            err = np.abs(g_xyz[both] - o_xyz[both]).max(axis=1)
            # FP32 solution within the map's evaluation noise; worst near the fold
            assert np.quantile(err, 0.999) < 2e-6 and err.max() < 2e-5, (k, np.quantile(err, 0.999), err.max())


@pytest.mark.parametrize("z0", [0.04, 0.025])
def test_image_near_feasibility_floor(hh, z0):
    """Grids a few centimetres above the track: the lattices reach the feasibility floor
    zh_floor (a tenth of the grid's height above the track), so infeasible samples and exact
    fallbacks occur, including at targets whose preimage lies within a few per cent of the
    floor, where the FP32 solver and the oracle's FP64 solver may decide feasibility
    differently.  The image must match the oracle's wherever the two decided alike, every
    differing voxel must still be a valid HHFFBPA value (no farther from BPA-RC than the
    oracle's own worst voxel), and the decisions may differ at few voxels only."""
    s = synth.small()
    g = synth.centred_grid(24, 20, 6, 2.5e-3, 2.5e-3, 1e-2, z0)
    e = synth.scene_echo(s, device="cuda")
    plan = hh.Plan(s.traj, s.freqs, g, leaf_size=16)
    img = plan.form_image(e)
    cnt = plan.counters()
    assert cnt["errors"] == 0 and cnt["gate_miss"] == 0, cnt
    assert cnt["infeasible"] > 0 and cnt["fallbacks"] > 0, cnt  # the floor is active
    ec = e.cpu().numpy()
    ref, st = oracle.Plan(s.traj, s.freqs, g, leaf_size=16).hhffbpa(ec)
    bref = oracle.bpa_rc(s.traj, s.freqs, ec, g.points())
    got = img.cpu().numpy().astype(np.complex128).ravel()
    peak = np.abs(ref).max()
    differ = np.abs(got - ref) > REL_TOL * peak
    assert differ.mean() <= 0.01, int(differ.sum())
    assert oracle.rel_l2(got[~differ], ref[~differ]) < REL_TOL
    if differ.any():
        worst_oracle = np.abs(ref - bref).max()
        assert np.abs(got[differ] - bref[differ]).max() <= worst_oracle, (int(differ.sum()), worst_oracle)


# Range-compression variants: the decomposed FFT (k_rc_fft2) serves N_f <= 512 with
# N_fft / M <= 32; a larger oversampling takes the shared-memory FFT (k_rc_fft, N_fft <= 8192)
# and beyond that the direct DFT (k_rc).  A scene whose range extent exceeds the unambiguous
# range pi / dk stores the whole period (gate wrap, indices modulo N_fft).
RC_CASES = [("rc_fft_shared", dict(n_f=32), 64, 2048), ("rc_direct_dft", dict(n_f=32), 512, 16384),
            ("gate_wrap", dict(n_f=8), 1, 8)]


@pytest.mark.parametrize("what,scene_kw,range_os,n_fft", RC_CASES)
def test_range_compression_paths_match_oracle(hh, what, scene_kw, range_os, n_fft):
    s = synth.small(**scene_kw)
    e = synth.scene_echo(s, device="cuda")
    ec = e.cpu().numpy()
    pts = s.grid.points()
    img = hh.bpa_form_image(s.traj, s.freqs, s.grid, e, range_os=range_os)
    torch.cuda.synchronize()
    ref = oracle.bpa_rc(s.traj, s.freqs, ec, pts, os_r=range_os).reshape(s.grid.shape)
    assert _rel(img, ref) < REL_TOL, what
    cfg = dict(leaf_size=16, range_os=range_os)
    plan = hh.Plan(s.traj, s.freqs, s.grid, **cfg)
    info = plan.info()
    assert info["n_fft"] == n_fft
    if what == "gate_wrap":
        assert info["gate_bins"] == n_fft and info["gate_start"] == 0, info
    himg = plan.form_image(e)
    cnt = plan.counters()
    assert cnt["gate_miss"] == 0 and cnt["errors"] == 0, cnt
    oref, _ = oracle.Plan(s.traj, s.freqs, s.grid, leaf_size=16, os_r=range_os).hhffbpa(ec)
    assert _rel(himg, oref.reshape(s.grid.shape)) < REL_TOL, what
