"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, a library routine, an
independent brute-force computation, a limit or an invariant stated by the
paper, chosen so that a dropped term, a wrong sign/index or a transposed
operand fails at least one of them.  CPU only.
"""
import math

import numpy as np
import pytest

import oracle
import synth

C = synth.C_LIGHT


def _small_geometry(seed=3, n_pos=40, n_f=9):
    rng = np.random.default_rng(seed)
    traj = np.column_stack([rng.uniform(-0.05, 0.05, n_pos), rng.uniform(-0.05, 0.05, n_pos),
                            rng.uniform(-3e-3, 3e-3, n_pos)])
    freqs = synth.freq_list(76e9, 81e9, n_f)
    return rng, traj, freqs


# --------------------------------------------------------------------------- BPA, Eq. bpafreqdomain
def test_bpa_exact_point_target_closed_form():
    """A unit scatterer at p0 gives f(p0) = a * N_A * N_f with phase arg(a) (Eq. 1 into Eq. bpafreqdomain)."""
    rng, traj, freqs = _small_geometry()
    p0 = np.array([[0.01, -0.02, 0.25]])
    a = 0.7 * np.exp(1j * 0.4)
    s = synth.echoes(traj, freqs, p0, np.array([a])).numpy()
    f = oracle.bpa_exact(traj, freqs, s, p0)[0]
    assert abs(f - a * len(traj) * len(freqs)) < 1e-9 * len(traj) * len(freqs)


def test_bpa_exact_brute_force_and_linearity():
    rng, traj, freqs = _small_geometry(n_pos=12, n_f=5)
    s1 = rng.standard_normal((12, 5)) + 1j * rng.standard_normal((12, 5))
    s2 = rng.standard_normal((12, 5)) + 1j * rng.standard_normal((12, 5))
    pts = np.column_stack([rng.uniform(-0.03, 0.03, 6), rng.uniform(-0.03, 0.03, 6), rng.uniform(0.2, 0.3, 6)])
    k = 2 * np.pi * freqs / C
    # independent brute force in numpy with pairwise summation order
    R = np.linalg.norm(pts[:, None, :] - traj[None, :, :], axis=2)
    brute = (s1[None, :, :] * np.exp(2j * k[None, None, :] * R[:, :, None])).sum(axis=(1, 2))
    got = oracle.bpa_exact(traj, freqs, s1, pts)
    np.testing.assert_allclose(got, brute, rtol=1e-12, atol=1e-12)
    lin = oracle.bpa_exact(traj, freqs, 2.0 * s1 - 1j * s2, pts)
    np.testing.assert_allclose(lin, 2.0 * got - 1j * oracle.bpa_exact(traj, freqs, s2, pts), rtol=1e-12, atol=1e-11)


def test_bpa_exact_is_adjoint_of_forward_model():
    """<A x, s> = <x, A^H s>: BPA is the matched filter of the Born model (Eq. 1)."""
    rng, traj, freqs = _small_geometry(n_pos=25, n_f=7)
    pts = np.column_stack([rng.uniform(-0.03, 0.03, 9), rng.uniform(-0.03, 0.03, 9), rng.uniform(0.2, 0.3, 9)])
    x = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    s = rng.standard_normal((25, 7)) + 1j * rng.standard_normal((25, 7))
    Ax = synth.echoes(traj, freqs, pts, x).numpy()
    AHs = oracle.bpa_exact(traj, freqs, s, pts)
    lhs = np.vdot(Ax, s)
    rhs = np.vdot(x, AHs)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


# --------------------------------------------------------------------------- range compression
def test_rc_window_matches_zero_padded_ifft():
    """P[m] = e^{-j pi (N_f-1) m / N_fft} * N_fft * ifft(zero-padded s)[m] (Eq. rangecompression)."""
    rng = np.random.default_rng(5)
    n_pos, n_f, os_r = 3, 12, 4
    s = rng.standard_normal((n_pos, n_f)) + 1j * rng.standard_normal((n_pos, n_f))
    n_fft = oracle.nfft(n_f, os_r)
    assert n_fft == 64
    pad = np.zeros((n_pos, n_fft), complex)
    pad[:, :n_f] = s
    m = np.arange(n_fft)
    ref = n_fft * np.fft.ifft(pad, axis=1) * np.exp(-1j * np.pi * (n_f - 1) * m / n_fft)[None, :]
    got = oracle.rc_window(s, n_fft, 0, n_fft)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)
    # periodic window starting below zero
    got2 = oracle.rc_window(s, n_fft, -5, 20)
    np.testing.assert_allclose(got2, ref[:, (np.arange(-5, 15)) % n_fft], rtol=1e-11, atol=1e-11)


def test_rc_params_definition():
    freqs = synth.freq_list(76e9, 81e9, 512)
    n_fft, dR, kc, dk = oracle.rc_params(freqs, 16)
    assert n_fft == 8192
    assert dk == pytest.approx(2 * np.pi * (81e9 - 76e9) / 511 / C, rel=1e-12)
    assert dR == pytest.approx(np.pi / (8192 * dk), rel=1e-12)
    assert dR == pytest.approx(1.87e-3, rel=3e-3)
    assert kc == pytest.approx(2 * np.pi * 78.5e9 / C, rel=1e-12)


def test_bpa_rc_converges_to_bpa_exact():
    """The range-compressed BPA approaches Eq. bpafreqdomain as the oversampling grows;
    linear interpolation of the centred tone bounds the error by (pi nu)^2/2, nu <= 1/(2 OS)."""
    s = synth.small()
    e = synth.scene_echo(s).numpy()
    pts = s.grid.points()[::7]
    ref = oracle.bpa_exact(s.traj, s.freqs, e, pts)
    errs = [oracle.rel_l2(oracle.bpa_rc(s.traj, s.freqs, e, pts, os_r=os), ref) for os in (4, 16, 64)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < (np.pi / 32) ** 2 / 2
    assert 20 * np.log10(errs[1]) < -40


# --------------------------------------------------------------------------- spectral design, Sec. III
RECT = (-0.06, -0.035, 0.02, 0.037)
ZBAR = 0.001
KMIN, KMAX = 2 * np.pi * 76e9 / C, 2 * np.pi * 81e9 / C
PROBES = np.array([[0.0, 0.0, 0.3], [0.05, -0.05, 0.25], [-0.047, 0.03, 0.22], [-0.2, 0.2, 0.4],
                   [-0.05, 0.025, 0.3]])


def _fd_grad(fun, p, h=1e-6):
    g = np.zeros(3)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        g[d] = (fun(p + e) - fun(p - e)) / (2 * h)
    return g


@pytest.mark.parametrize("p", list(PROBES))
def test_uvn_jacobian_is_llt_matrix(p):
    """Eq. eq_duvw_relp: the Jacobian of (u, v, n) is T_s = [v1; v2; v3]/2pi; the printed potentials
    of Eq. eq_uvw_xyz carry signs (-, -, +)."""
    K, Ts = oracle.keypoints(RECT, ZBAR, KMIN, KMAX, p)
    for d, sign in ((0, -1), (1, -1), (2, 1)):
        g = _fd_grad(lambda q: oracle.uvn(RECT, ZBAR, KMIN, KMAX, q)[0][d], p)
        np.testing.assert_allclose(g, sign * Ts[d], rtol=2e-6, atol=1e-3)
    # T_s rows rebuilt from the key points by hand
    np.testing.assert_allclose(Ts[0], (K[1] - K[0]) / (2 * np.pi), rtol=1e-12)
    np.testing.assert_allclose(Ts[2], (K[6] - K[4]) / (2 * np.pi), rtol=1e-12)


@pytest.mark.parametrize("p", list(PROBES))
def test_sdc_phase_gradient_is_spectrum_centre(p):
    """Eq. eq_dp_kc: grad Phi = k_c = (k5 + k7)/2 with Phi of Eq. eq_sdc_phi."""
    K, _ = oracle.keypoints(RECT, ZBAR, KMIN, KMAX, p)
    g = _fd_grad(lambda q: oracle.uvn(RECT, ZBAR, KMIN, KMAX, q)[0][3], p)
    np.testing.assert_allclose(g, (K[4] + K[6]) / 2, rtol=1e-6, atol=1e-3)


def test_keypoints_closed_forms():
    """k1..k5 from Eq. eq_kfun_posp written out by hand; k6 = 2 kmax k5/|k5|; on the boresight
    axis of the subarray k7 = k6 (the condition that fixes beta)."""
    a, b, e, g = RECT
    p = np.array([0.01, 0.03, 0.27])
    K, _ = oracle.keypoints(RECT, ZBAR, KMIN, KMAX, p)

    def k0(X, Y, k):
        d = p - np.array([X, Y, ZBAR])
        return 2 * k * d / np.linalg.norm(d)

    x0 = min(max(p[0], a), b)
    y0 = min(max(p[1], e), g)
    np.testing.assert_allclose(K[0], k0(a, y0, KMAX), rtol=1e-13)
    np.testing.assert_allclose(K[1], k0(b, y0, KMAX), rtol=1e-13)
    np.testing.assert_allclose(K[2], k0(x0, e, KMAX), rtol=1e-13)
    np.testing.assert_allclose(K[3], k0(x0, g, KMAX), rtol=1e-13)
    k5 = (k0(a, e, KMIN) + k0(a, g, KMIN) + k0(b, e, KMIN) + k0(b, g, KMIN)) / 4
    np.testing.assert_allclose(K[4], k5, rtol=1e-13)
    np.testing.assert_allclose(K[5], 2 * KMAX * k5 / np.linalg.norm(k5), rtol=1e-13)
    pb = np.array([(a + b) / 2, (e + g) / 2, 0.3])
    Kb, _ = oracle.keypoints(RECT, ZBAR, KMIN, KMAX, pb)
    np.testing.assert_allclose(Kb[6], Kb[5], rtol=1e-12, atol=1e-9)


def _curl(field, p, h=1e-6):
    J = np.zeros((3, 3))
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        J[:, d] = (field(p + e) - field(p - e)) / (2 * h)
    return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]]), np.abs(J).max()


def test_k7_is_curl_free():
    """Eq. eq_k7_curlfree: curl k7 = 0, whereas k6 is not irrotational (the reason for the
    integrating factor of Eq. eq_spv_scl).  Finite differences on a large subarray."""
    rect = (-0.25, 0.0, -0.1, 0.15)
    p = np.array([0.05, -0.1, 0.25])
    c7, s7 = _curl(lambda q: oracle.keypoints(rect, ZBAR, KMIN, KMAX, q)[0][6], p)
    c6, s6 = _curl(lambda q: oracle.keypoints(rect, ZBAR, KMIN, KMAX, q)[0][5], p)
    assert np.abs(c7).max() < 1e-6 * s7
    assert np.abs(c6).max() > 1e-2 * s6


def test_local_spectrum_inside_unit_box_for_small_subarray():
    """Sec. III: after SDC and LLT the local spectrum of a small subarray fits the unit box
    |kappa| <= pi (up to the approximation of the key points)."""
    p = np.array([0.01, -0.02, 0.3])
    K, Ts = oracle.keypoints(RECT, ZBAR, KMIN, KMAX, p)
    J = np.array([-Ts[0], -Ts[1], Ts[2]])
    kc = (K[4] + K[6]) / 2
    worst = 0.0
    for X in np.linspace(RECT[0], RECT[1], 9):
        for Y in np.linspace(RECT[2], RECT[3], 9):
            for k in np.linspace(KMIN, KMAX, 5):
                d = p - np.array([X, Y, ZBAR])
                Kv = 2 * k * d / np.linalg.norm(d)
                kap = np.linalg.solve(J.T, Kv - kc)
                worst = max(worst, np.abs(kap).max() / np.pi)
    assert 0.9 < worst < 1.02


def _uvn_jacobian_fd(rect, zbar, kmin, kmax, p, h=1e-6):
    """Jacobian of (u, v, n) in (x, y, z) and grad Phi at p, by central differences of the
    oracle's map values alone (none of its key-point algebra)."""
    J = np.zeros((3, 3))
    gphi = np.zeros(3)
    for d in range(3):
        dp = np.zeros(3)
        dp[d] = h
        w1 = oracle.uvn(rect, zbar, kmin, kmax, p + dp)[0]
        w0 = oracle.uvn(rect, zbar, kmin, kmax, p - dp)[0]
        J[:, d] = (w1[:3] - w0[:3]) / (2 * h)
        gphi[d] = (w1[3] - w0[3]) / (2 * h)
    return J, gphi


def _kappa_extent(rect, zbar, kmin, kmax, pts, sources, ks):
    """Largest |kappa_d| / pi over the points of D `pts`, the aperture points `sources` and the
    wavenumbers `ks`: kappa = J^-T (K - grad Phi), K = 2 k (p - p') / |p - p'| (Eq. eq_kxyz_posp;
    the spectrum-centre grad Phi of Eq. eq_dp_kc and the local-frequency transform of
    Eq. eq_llt_spcm_trans, written here from the chain rule)."""
    best = np.zeros(3)
    for p in pts:
        J, gphi = _uvn_jacobian_fd(rect, zbar, kmin, kmax, p)
        d = p[None, :] - sources
        u = d / np.linalg.norm(d, axis=1)[:, None]
        K = 2.0 * np.asarray(ks)[None, :, None] * u[:, None, :]
        kap = np.linalg.solve(J.T, (K - gphi).reshape(-1, 3).T).T
        best = np.maximum(best, np.abs(kap).max(axis=0) / np.pi)
    return best


@pytest.mark.parametrize("name,cfg", [("small", dict(leaf_size=16)), ("tiny", dict(leaf_size=32)),
                                      ("large", dict(leaf_size=256, eta=1.6))])
def test_spectral_extent_bounds_the_subimage_spectrum(name, cfg):
    """The per-axis lattice density eta_d = eta * rho_d (rho_d from the oracle's spectral
    extent) against an independent evaluation of the transformed spectrum (Sec. III,
    Eq. eq_llt_spcm_trans: the compressed subimage's local spectrum lies in a box whose
    half-width is the sampling requirement).  For a leaf, a mid-level node and a root child:
      (1) a superset of the oracle's probe set -- a 5x5x5 grid of D (corners, face centres and
          centre included), the subarray border at 9 points per edge (the 1/4 steps included)
          at the lowest and highest member heights, k_min and k_max -- bounds rho from above
          (rho is a maximum over a subset, rounded up to 1/64) and attains it within 1/32;
      (2) the true spectrum of the subimage -- every member's 3-D position at the extreme
          wavenumbers (kappa is affine in k, so its extremes over [k_min, k_max] lie at the
          ends) over the same grid of D -- stays within rho (1 + 1/32).
    J comes from central differences of (u, v, n) and grad Phi from those of Phi, K from the
    geometry in numpy, so a transposed solve (J kappa = ...; 2-5x off), a probe at one height
    only (up to 8 % low on small subarrays) or a wrong spectrum centre fails here."""
    s = synth.CONFIGS[name]()
    ex = oracle.Plan(s.traj, s.freqs, s.grid, **cfg).export()
    g = s.grid
    eta0 = cfg.get("eta", 2.0)
    ls = ex["level_start"]
    kmin, kmax = ex["kmin"], ex["kmax"]
    ks = np.array([kmin, kmax])
    axes = [np.linspace(o, o + d * (n - 1), 5) for o, d, n in ((g.x0, g.dx, g.nx), (g.y0, g.dy, g.ny),
                                                              (g.z0, g.dz, g.nz))]
    pts = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(11)
    for k in (0, int(ls[1]) // 2, int(ls[-2]) - 1):  # a leaf, a mid-level node, a root child
        rect = ex["rect"][k]
        a, b, e, gg = rect
        zbar = ex["node_zbar"][k]
        mem = s.traj[ex["perm"][ex["begin"][k]:ex["end"][k]]]
        if len(mem) > 512:
            keep = np.concatenate([rng.choice(len(mem), 500, replace=False),
                                   np.argmin(mem, axis=0), np.argmax(mem, axis=0)])
            mem = mem[np.unique(keep)]
        t = np.linspace(0.0, 1.0, 9)
        edge = np.concatenate([np.column_stack([a + t * (b - a), np.full(9, e)]),
                               np.column_stack([a + t * (b - a), np.full(9, gg)]),
                               np.column_stack([np.full(9, a), e + t * (gg - e)]),
                               np.column_stack([np.full(9, b), e + t * (gg - e)])])
        zlo, zhi = s.traj[ex["perm"][ex["begin"][k]:ex["end"][k]], 2].min(), \
            s.traj[ex["perm"][ex["begin"][k]:ex["end"][k]], 2].max()
        border = np.concatenate([np.column_stack([edge, np.full(len(edge), zlo)]),
                                 np.column_stack([edge, np.full(len(edge), zhi)])])
        rho = ex["eta"][k] / eta0
        sup = _kappa_extent(rect, zbar, kmin, kmax, pts, border, ks)
        true = _kappa_extent(rect, zbar, kmin, kmax, pts, mem, ks)
        assert np.all(rho <= sup + 1.0 / 64 + 1e-6), (name, k, rho, sup)
        assert np.all(sup <= rho * (1 + 1.0 / 32)), (name, k, rho, sup)
        assert np.all(true <= rho * (1 + 1.0 / 32)), (name, k, rho, true)


def test_solver_jacobian_is_llt_matrix_in_squared_height():
    """The preimage solver's Jacobian in (x, y, s = zh^2) equals the key-point matrix
    diag(-1, -1, 1) T_s (Eq. eq_duvw_relp) with its z column divided by 2 zh."""
    for p in PROBES:
        Jt = oracle.jacobian_ts(RECT, ZBAR, KMIN, KMAX, p)
        zh = p[2] - ZBAR
        Js = oracle.jacobian_s(RECT, KMIN, KMAX, p[0], p[1], zh * zh)
        np.testing.assert_allclose(Js[:, :2], Jt[:, :2], rtol=1e-10, atol=1e-8)
        np.testing.assert_allclose(Js[:, 2], Jt[:, 2] / (2 * zh), rtol=1e-10, atol=1e-8)


# --------------------------------------------------------------------------- preimage
def test_preimage_round_trip():
    rng = np.random.default_rng(11)
    pts = np.column_stack([rng.uniform(-0.1, 0.1, 300), rng.uniform(-0.1, 0.1, 300), rng.uniform(0.15, 0.5, 300)])
    tg = oracle.uvn(RECT, ZBAR, KMIN, KMAX, pts)[:, :3]
    xyz, ok = oracle.preimage(RECT, ZBAR, KMIN, KMAX, 0.01, 0.3, tg)
    assert ok.all()
    np.testing.assert_allclose(xyz, pts, atol=1e-9)
    # a target beyond the reach of the difference-of-distances map has no preimage
    usat = KMAX / np.pi * (RECT[1] - RECT[0])
    _, ok2 = oracle.preimage(RECT, ZBAR, KMIN, KMAX, 0.01, 0.3, np.array([[1.05 * usat, 0.0, tg[0, 2]]]))
    assert not ok2[0]


# --------------------------------------------------------------------------- interpolation kernel
@pytest.mark.parametrize("taps,eta", [(4, 2.0), (6, 2.0), (6, 1.75), (6, 1.6)])
def test_ls_weights_identity_and_band(taps, eta):
    tau = np.linspace(0, 1, 41)
    w = oracle.ls_weights(taps, eta, tau)
    o = np.arange(-(taps // 2 - 1), taps // 2 + 1)
    e0 = (o == 0).astype(float)
    np.testing.assert_allclose(w[0], e0, atol=1e-12)          # tau = 0 reproduces the sample
    np.testing.assert_allclose(w[-1], (o == 1).astype(float), atol=1e-12)  # tau = 1 the next one
    # independent least-squares fit on a dense in-band frequency grid (numpy lstsq)
    B = 0.5 / eta
    f = np.linspace(-B, B, 2001)
    for t, wi in zip(tau[5::10], w[5::10]):
        A = np.exp(2j * np.pi * np.outer(f, o))
        rhs = np.exp(2j * np.pi * f * t)
        h_ref = np.linalg.lstsq(np.vstack([A.real, A.imag]), np.concatenate([rhs.real, rhs.imag]), rcond=None)[0]
        np.testing.assert_allclose(wi, h_ref, atol=2e-4)
        # in-band tones are reproduced to the least-squares level
        err = np.abs(A @ wi - rhs)
        assert err.max() < {(4, 2.0): 0.06, (6, 2.0): 0.01, (6, 1.75): 0.025, (6, 1.6): 0.04}[(taps, eta)]


# --------------------------------------------------------------------------- plan
def test_plan_tree_invariants():
    s = synth.tiny()
    pl = oracle.Plan(s.traj, s.freqs, s.grid, leaf_size=32, merge_factor=4, eta=2.0, taps=6)
    ex = pl.export()
    assert ex["depth_leaves"] == 6 and ex["n_levels"] == 4
    assert sorted(ex["perm"].tolist()) == list(range(len(s.traj)))
    ls = ex["level_start"]
    leaves = slice(ls[0], ls[1])
    assert (ex["end"][leaves] - ex["begin"][leaves] == 32).all()
    # every materialised node's children tile its member range
    for k in range(ls[1], ls[-1]):
        c0, nc = ex["child0"][k], ex["nchild"][k]
        assert ex["begin"][c0] == ex["begin"][k] and ex["end"][c0 + nc - 1] == ex["end"][k]
        assert (ex["end"][c0:c0 + nc - 1] == ex["begin"][c0 + 1:c0 + nc]).all()
    # first split is along x at the median: left members all have x <= right members
    root = ls[-2]
    mid = len(s.traj) // 2
    assert s.traj[ex["perm"][:mid], 0].max() <= s.traj[ex["perm"][mid:], 0].min()
    # the second split is along y inside each half
    q = len(s.traj) // 4
    assert s.traj[ex["perm"][:q], 1].max() <= s.traj[ex["perm"][q:mid], 1].min()
    # bbox of leaf members
    for k in range(ls[0], ls[0] + 5):
        m = ex["perm"][ex["begin"][k]:ex["end"][k]]
        a, b, e, g = ex["rect"][k]
        assert a <= s.traj[m, 0].min() and b >= s.traj[m, 0].max()
        assert ex["node_zbar"][k] == pytest.approx(s.traj[m, 2].mean(), abs=1e-15)


def test_plan_lattice_covers_grid_image():
    """Every voxel of D maps inside each node's lattice with its padding, and the
    box extremes found by the plan are attained (brute force over all voxels)."""
    s = synth.small()
    pl = oracle.Plan(s.traj, s.freqs, s.grid, leaf_size=16, merge_factor=4, eta=2.0, taps=6)
    ex = pl.export()
    pts = s.grid.points()
    ls = ex["level_start"]
    for k in list(range(ls[0], ls[0] + 3)) + list(range(ls[-3], ls[-2])):
        w = oracle.uvn(ex["rect"][k], ex["node_zbar"][k], ex["kmin"], ex["kmax"], pts)[:, :3]
        fi = (w - ex["lo"][k]) * ex["eta"][k]
        pad_n = 3 * ex["t"][k] + 1
        assert (fi[:, 2] >= pad_n - 1e-9).all() and (fi[:, 2] <= ex["N"][k][2] - 1 - pad_n + 1 + 1e-9).all()
        assert (fi[:, :2] >= 1).all() and (fi[:, :2] <= ex["N"][k][:2] - 2).all()


# --------------------------------------------------------------------------- HHFFBPA
def test_hhffbpa_single_level_is_bpa_rc():
    """With no factorisation (M = 1: one subarray) HHFFBPA is BPA on range-compressed data."""
    s = synth.small()
    e = synth.scene_echo(s).numpy()
    pl = oracle.Plan(s.traj, s.freqs, s.grid, leaf_size=10 ** 6)
    assert pl.info()["n_levels"] == 1
    pts = s.grid.points()[::5]
    hh, _ = pl.hhffbpa(e, pts)
    ref = oracle.bpa_rc(s.traj, s.freqs, e, pts)
    np.testing.assert_allclose(hh, ref, rtol=1e-12, atol=1e-9)


def test_hhffbpa_demand_driven_subset_equals_full():
    s = synth.small()
    e = synth.scene_echo(s).numpy()
    pl = oracle.Plan(s.traj, s.freqs, s.grid, leaf_size=16, merge_factor=4, eta=2.0, taps=6)
    full, _ = pl.hhffbpa(e)
    idx = np.array([0, 17, 400, 1234, s.grid.n_vox - 1])
    part, _ = pl.hhffbpa(e, s.grid.points(idx))
    np.testing.assert_array_equal(part, full[idx])


def test_hhffbpa_accuracy_and_point_target_tiny():
    """HHFFBPA approximates BPA (Sec. IV): NRMSE <= -30 dB on the tiny workload; the brightest
    voxel coincides with BPA's and its phase matches BPA's."""
    s = synth.tiny()
    e = synth.scene_echo(s).numpy()
    pts = s.grid.points()
    bpa = oracle.bpa_rc(s.traj, s.freqs, e, pts)
    pl = oracle.Plan(s.traj, s.freqs, s.grid, leaf_size=32, merge_factor=4, eta=2.0, taps=6)
    hh, st = pl.hhffbpa(e)
    assert oracle.nrmse_db(hh, bpa) < -40
    i = np.argmax(np.abs(bpa))
    assert np.argmax(np.abs(hh)) == i
    assert abs(np.angle(hh[i] / bpa[i])) < 0.05


def test_hhffbpa_single_scatterer_phase_closed_form():
    """A unit scatterer exactly on a voxel: HHFFBPA's value there has the closed-form phase 0
    of Eq. bpafreqdomain within 0.05 rad and magnitude within 2 % of N_A * N_f."""
    s = synth.small()
    vox = s.grid.points(np.array([s.grid.nx * s.grid.ny * 3 + s.grid.nx * 9 + 11]))
    e = synth.echoes(s.traj, s.freqs, vox, np.array([1.0 + 0j])).numpy().astype(np.complex64)
    pl = oracle.Plan(s.traj, s.freqs, s.grid, leaf_size=16, merge_factor=4, eta=2.0, taps=6)
    hh, _ = pl.hhffbpa(e, vox)
    n = len(s.traj) * len(s.freqs)
    assert abs(np.angle(hh[0])) < 0.05
    assert abs(abs(hh[0]) / n - 1) < 0.02


def test_plant_mistake_in_interpolation_is_caught():
    """A planted mistake (wrong kernel: 2 taps) must break the accuracy pin, showing the pin bites."""
    s = synth.small()
    e = synth.scene_echo(s).numpy()
    pts = s.grid.points()
    bpa = oracle.bpa_rc(s.traj, s.freqs, e, pts)
    good, _ = oracle.Plan(s.traj, s.freqs, s.grid, leaf_size=16, eta=2.0, taps=6).hhffbpa(e)
    bad, _ = oracle.Plan(s.traj, s.freqs, s.grid, leaf_size=16, eta=1.0, taps=2).hhffbpa(e)
    assert oracle.nrmse_db(good, bpa) < -35
    assert oracle.nrmse_db(bad, bpa) > -20


# --------------------------------------------------------------------------- trajectory gradient
def test_bpa_rc_traj_grad_matches_finite_differences():
    """The oracle's position gradient of L = Re sum conj(g) f against central differences of
    the oracle's own BPA-RC image (C code, an independent evaluation of the same sum)."""
    s = synth.small()
    e = synth.scene_echo(s).numpy()
    rng = np.random.default_rng(7)
    pts = s.grid.points(rng.choice(s.grid.n_vox, 40, replace=False))
    g = rng.normal(size=40) + 1j * rng.normal(size=40)
    G = oracle.bpa_rc_traj_grad(s.traj, s.freqs, e, pts, g)

    def loss(traj):
        return (np.conj(g) * oracle.bpa_rc(traj, s.freqs, e, pts)).real.sum()

    h = 1e-9  # far below the range bin (1.87 mm): no lerp kink is crossed
    for i, ax in [(0, 0), (5, 1), (17, 2), (100, 0), (200, 2), (255, 1)]:
        tp, tm = s.traj.copy(), s.traj.copy()
        tp[i, ax] += h
        tm[i, ax] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(fd - G[i, ax]) <= 1e-5 * abs(G[i, ax]), (i, ax, fd, G[i, ax])


def test_bpa_rc_traj_grad_vanishes_for_zero_image_gradient_and_is_linear():
    s = synth.small()
    e = synth.scene_echo(s).numpy()
    rng = np.random.default_rng(8)
    pts = s.grid.points(rng.choice(s.grid.n_vox, 16, replace=False))
    g1 = rng.normal(size=16) + 1j * rng.normal(size=16)
    g2 = rng.normal(size=16) + 1j * rng.normal(size=16)
    assert np.all(oracle.bpa_rc_traj_grad(s.traj, s.freqs, e, pts, np.zeros(16)) == 0)
    a = oracle.bpa_rc_traj_grad(s.traj, s.freqs, e, pts, g1 + 2 * g2)
    b = oracle.bpa_rc_traj_grad(s.traj, s.freqs, e, pts, g1) + 2 * oracle.bpa_rc_traj_grad(s.traj, s.freqs, e, pts, g2)
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-9 * np.abs(a).max())


def test_bpa_rc_adjoint_dot_product_identity():
    """<x, A s> = <A^H x, s> for the oracle's BPA-RC (C) and its adjoint written out (numpy)."""
    s = synth.small()
    rng = np.random.default_rng(3)
    e = rng.normal(size=(len(s.traj), len(s.freqs))) + 1j * rng.normal(size=(len(s.traj), len(s.freqs)))
    pts = s.grid.points(rng.choice(s.grid.n_vox, 50, replace=False))
    x = rng.normal(size=50) + 1j * rng.normal(size=50)
    lhs = np.vdot(x, oracle.bpa_rc(s.traj, s.freqs, e, pts))
    rhs = np.vdot(oracle.bpa_rc_adjoint(s.traj, s.freqs, x, pts), e)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _corner_points(g, k=4):
    ix = np.r_[0:k, g.nx - k:g.nx]
    iy = np.r_[0:k, g.ny - k:g.ny]
    return np.array([(z * g.ny + y) * g.nx + x for z in range(g.nz) for y in iy for x in ix])


@pytest.mark.parametrize("name,cfg,corners", [("small", dict(leaf_size=16), False),
                                              ("small", dict(leaf_size=16, merge_factor=2), False),
                                              ("tiny", dict(leaf_size=32, eta=1.25), True),
                                              ("tiny", dict(leaf_size=32, eta=1.1), True)])
def test_hhffbpa_adjoint_dot_product_identity(name, cfg, corners):
    """<x, H s> = <H^H x, s> for the oracle's HHFFBPA and its adjoint (C, step by step); the
    corner voxels of sparse-lattice plans take exact fallbacks and meet infeasible samples."""
    s = synth.CONFIGS[name]()
    rng = np.random.default_rng(4)
    e = rng.normal(size=(len(s.traj), len(s.freqs))) + 1j * rng.normal(size=(len(s.traj), len(s.freqs)))
    idx = _corner_points(s.grid) if corners else rng.choice(s.grid.n_vox, 40, replace=False)
    pts = s.grid.points(idx)
    x = rng.normal(size=len(idx)) + 1j * rng.normal(size=len(idx))
    pl = oracle.Plan(s.traj, s.freqs, s.grid, **cfg)
    f, st = pl.hhffbpa(e, pts)
    if corners:
        assert st["fallbacks"] > 0 and st["infeasible"] > 0, st
    lhs = np.vdot(x, f)
    rhs = np.vdot(pl.hhffbpa_adjoint(x, pts), e)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_hhffbpa_adjoint_single_level_is_bpa_rc_adjoint():
    """With one level the HHFFBPA adjoint (C) reduces to the BPA-RC adjoint written out (numpy)."""
    s = synth.small()
    rng = np.random.default_rng(5)
    idx = rng.choice(s.grid.n_vox, 30, replace=False)
    pts = s.grid.points(idx)
    x = rng.normal(size=30) + 1j * rng.normal(size=30)
    pl = oracle.Plan(s.traj, s.freqs, s.grid, leaf_size=len(s.traj))
    assert pl.info()["n_levels"] == 1
    a = pl.hhffbpa_adjoint(x, pts)
    b = oracle.bpa_rc_adjoint(s.traj, s.freqs, x, pts)
    assert oracle.rel_l2(a.ravel(), b.ravel()) < 1e-12


@pytest.mark.parametrize("name,cfg,corners", [("small", dict(leaf_size=16), False),
                                              ("tiny", dict(leaf_size=32, eta=1.25), True)])
def test_hhffbpa_traj_grad_matches_finite_differences_with_plan_fixed(name, cfg, corners):
    """The oracle's HHFFBPA position gradient (plan held fixed) against central differences
    of the oracle's HHFFBPA with one position moved in place (the plan keeps its tree,
    lattices and preimages); the corner voxels of the sparse plan take exact fallbacks."""
    s = synth.CONFIGS[name]()
    e = synth.scene_echo(s).numpy()
    rng = np.random.default_rng(9)
    idx = _corner_points(s.grid) if corners else rng.choice(s.grid.n_vox, 40, replace=False)
    pts = s.grid.points(idx)
    x = rng.normal(size=len(idx)) + 1j * rng.normal(size=len(idx))
    pl = oracle.Plan(s.traj, s.freqs, s.grid, **cfg)
    G = pl.hhffbpa_traj_grad(e, x, pts)
    if corners:
        assert pl.hhffbpa(e, pts)[1]["fallbacks"] > 0

    def loss():
        return (np.conj(x) * pl.hhffbpa(e, pts)[0]).real.sum()

    h = 1e-9
    for i, ax in [(0, 0), (7, 1), (33, 2), (len(s.traj) - 1, 1)]:
        old = pl.traj[i, ax]
        pl.traj[i, ax] = old + h
        lp = loss()
        pl.traj[i, ax] = old - h
        lm = loss()
        pl.traj[i, ax] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - G[i, ax]) <= 2e-6 * abs(G[i, ax]), (i, ax, fd, G[i, ax])
