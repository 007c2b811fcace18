"""FP64 CPU oracle for HHFFBPA and BPA -- TEST INFRASTRUCTURE ONLY.

The oracle is the plain, slow, obviously-correct reference the CUDA library is
checked against.  Only tests/, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline/reference legs may import it; the library never does, and the two
share no code.  The C source (hh_oracle.c) cites the paper passage each step
follows and lists the readings taken where the paper is silent.

Parity status per function:
  rc_window, bpa_exact, bpa_rc  -- pinned (closed forms, limits, adjoint identity)
  keypoints, uvn                -- pinned (finite-difference identities of Sec. III)
  preimage                      -- pinned (round trip)
  ls_weights                    -- pinned (identity at integer offsets, exact on
                                   in-band tones within the least-squares bound)
  plan                          -- pinned (tree invariants, brute-force bbox)
  spectral extent (lattice      -- pinned: bounded and attained, within 1/32, by an
  density per axis)                independent evaluation of the transformed spectrum
                                   (finite-difference Jacobian, numpy geometry) over a
                                   superset of its probe set, and bounding the true
                                   spectrum of every member
  hhffbpa                       -- pinned by the M=1 reduction, the interpolation
                                   identity, demand-driven = full evaluation, the
                                   point-target peak and phase, and the exact (BPA-RC)
                                   result within the accuracy bound; the paper prints
                                   no value that fixes the absolute image
  hhffbpa_adjoint, _traj_grad   -- pinned (dot-product identity; finite differences)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hh_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libhh_oracle.so")
_lib = None

C_LIGHT = 299_792_458.0


def build(force=False):
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
                               "-Wno-unused-function", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.c_int64


def _declare(L):
    L.hho_nfft.argtypes = [ctypes.c_int, ctypes.c_int]
    L.hho_nfft.restype = ctypes.c_int
    L.hho_rc_window.argtypes = [_dp, _i64, ctypes.c_int, ctypes.c_int, _i64, ctypes.c_int, _dp]
    L.hho_bpa_exact.argtypes = [_dp, _i64, _dp, ctypes.c_int, _dp, _dp, _i64, _dp]
    L.hho_bpa_rc.argtypes = [_dp, _i64, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _i64, _dp]
    L.hho_rc_params.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp]
    L.hho_keypoints.argtypes = [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
    L.hho_uvn.argtypes = [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _i64, _dp]
    L.hho_preimage.argtypes = [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, _dp, _i64, _dp, _i32p]
    L.hho_jacobian_ts.argtypes = [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
    L.hho_jacobian_s.argtypes = [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, _dp]
    L.hho_ls_weights.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _i64, _dp]
    L.hho_ls_weights.restype = ctypes.c_int
    L.hho_plan_create.argtypes = [_dp, _i64, _dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_int, ctypes.c_int]
    L.hho_plan_create.restype = ctypes.c_void_p
    L.hho_plan_destroy.argtypes = [ctypes.c_void_p]
    L.hho_plan_info.argtypes = [ctypes.c_void_p, _ip]
    L.hho_plan_export.argtypes = [ctypes.c_void_p, _ip, _ip, _dp, _dp]
    L.hho_hhffbpa.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, _dp, _dp, _i64, _dp, _ip]
    L.hho_hhffbpa.restype = ctypes.c_int
    L.hho_hhffbpa_adjoint.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, _dp, _dp, _i64, _dp]
    L.hho_hhffbpa_adjoint.restype = ctypes.c_int
    L.hho_hhffbpa_traj_grad.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, _dp, _dp, _dp, _i64, _dp]
    L.hho_hhffbpa_traj_grad.restype = ctypes.c_int
    L.hho_num_threads.restype = ctypes.c_int


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def _ri(z):
    """complex array -> interleaved float64 (re, im)."""
    z = np.ascontiguousarray(np.asarray(z), dtype=np.complex128)
    return z.view(np.float64)


def _cplx(ri, shape):
    return ri.view(np.complex128).reshape(shape)


def num_threads():
    return lib().hho_num_threads()


def nfft(n_f, os_r=16):
    return lib().hho_nfft(n_f, os_r)


def rc_params(freqs, os_r=16):
    """(n_fft, dR, k_c, dk) as the oracle defines them."""
    f = _f64(freqs)
    out = np.zeros(4)
    lib().hho_rc_params(_ptr(f), len(f), os_r, _ptr(out))
    return int(out[0]), out[1], out[2], out[3]


def rc_window(echo, n_fft, m_lo, n_bins):
    """Range profiles P[i, m] for m = m_lo .. m_lo+n_bins-1 (periodic), complex128."""
    e = _ri(echo)
    n_pos, n_f = np.asarray(echo).shape
    out = np.zeros(2 * n_pos * n_bins)
    lib().hho_rc_window(_ptr(e), n_pos, n_f, n_fft, m_lo, n_bins, _ptr(out))
    return _cplx(out, (n_pos, n_bins))


def bpa_exact(traj, freqs, echo, pts):
    t, f, p = _f64(traj), _f64(freqs), _f64(pts)
    e = _ri(echo)
    out = np.zeros(2 * len(p))
    lib().hho_bpa_exact(_ptr(t), len(t), _ptr(f), len(f), _ptr(e), _ptr(p), len(p), _ptr(out))
    return _cplx(out, (len(p),))


def bpa_rc(traj, freqs, echo, pts, os_r=16):
    t, f, p = _f64(traj), _f64(freqs), _f64(pts)
    e = _ri(echo)
    out = np.zeros(2 * len(p))
    lib().hho_bpa_rc(_ptr(t), len(t), _ptr(f), len(f), os_r, _ptr(e), _ptr(p), len(p), _ptr(out))
    return _cplx(out, (len(p),))


def bpa_rc_traj_grad(traj, freqs, echo, pts, g, os_r=16):
    """Gradient with respect to the positions of L = Re sum_p conj(g_p) f(p), f the BPA-RC
    image (Eqs. eq2_rangecompression, eq2_bpatimedomain: f(p) = sum_i exp(+j 2 k_c R_i)
    lerp(P_i, R_i / dR)) at the points pts, in FP64.  The range profiles do not depend on
    the positions and the lerp is differentiated within its bin:
    dL/dp'_i = sum_p Re[conj(g_p) exp(+j 2 k_c R) (j 2 k_c lerp + (P[m0+1] - P[m0]) / dR)] (p'_i - p) / R.
    Returns float64[n_pos][3].  Plain numpy over all (position, point) pairs: small cases."""
    t, p = _f64(traj), _f64(pts)
    g = np.asarray(g, np.complex128).ravel()
    n_fft, dR, kc, _ = rc_params(freqs, os_r)
    d = t[:, None, :] - p[None, :, :]
    R = np.sqrt((d * d).sum(-1))
    mu = R / dR
    m0 = np.floor(mu)
    frac = mu - m0
    m_lo = int(m0.min())
    P = rc_window(echo, n_fft, m_lo, int(m0.max()) - m_lo + 2)
    idx = (m0 - m_lo).astype(np.int64)
    P0 = np.take_along_axis(P, idx, 1)
    P1 = np.take_along_axis(P, idx + 1, 1)
    lerp = P0 + frac * (P1 - P0)
    E = np.exp(2j * kc * R) * (2j * kc * lerp + (P1 - P0) / dR)
    a = (np.conj(g)[None, :] * E).real
    return ((a / R)[:, :, None] * d).sum(axis=1)


def bpa_rc_adjoint(traj, freqs, x, pts, os_r=16):
    """Adjoint of the BPA-RC image at the points pts (Eqs. eq2_rangecompression,
    eq2_bpatimedomain): s[i, n] = sum_p x_p exp(-j 2 k_c R) [(1 - t) e^{-j th_n m0} + t e^{-j th_n (m0+1)}],
    th_n = 2 pi (n - (N_f - 1)/2) / N_fft, m0 = floor(R / dR) (bins mod N_fft, as the profiles),
    t = R / dR - m0: the conjugate transpose of f = A s written out, in FP64.  Returns
    complex128 [n_pos][n_f]."""
    t, p = _f64(traj), _f64(pts)
    x = np.asarray(x, np.complex128).ravel()
    n_f = len(np.asarray(freqs))
    n_fft, dR, kc, _ = rc_params(freqs, os_r)
    d = t[:, None, :] - p[None, :, :]
    R = np.sqrt((d * d).sum(-1))
    mu = R / dR
    m0 = np.floor(mu)
    frac = mu - m0
    th = 2 * np.pi * (np.arange(n_f) - (n_f - 1) / 2) / n_fft
    c = x[None, :] * np.exp(-2j * kc * R)  # [n_pos, n_pts]
    # bins taken mod N_fft, as the range profiles are (they are periodic in m up to that sign)
    e0 = np.exp(-1j * th[None, None, :] * np.mod(m0, n_fft)[:, :, None])
    e1 = np.exp(-1j * th[None, None, :] * np.mod(m0 + 1, n_fft)[:, :, None])
    return ((c * (1 - frac))[:, :, None] * e0 + (c * frac)[:, :, None] * e1).sum(axis=1)


def keypoints(rect, zbar, kmin, kmax, p):
    """(k[7][3], Ts[3][3]) at point p for subarray rect = (a, b, e, g)."""
    r, pp = _f64(rect), _f64(p)
    out = np.zeros(30)
    lib().hho_keypoints(_ptr(r), zbar, kmin, kmax, _ptr(pp), _ptr(out))
    return out[:21].reshape(7, 3), out[21:].reshape(3, 3)


def uvn(rect, zbar, kmin, kmax, pts):
    """(u, v, n, Phi) per point, float64[n][4]."""
    r, p = _f64(rect), _f64(np.atleast_2d(pts))
    out = np.zeros(4 * len(p))
    lib().hho_uvn(_ptr(r), zbar, kmin, kmax, _ptr(p), len(p), _ptr(out))
    return out.reshape(-1, 4)


def preimage(rect, zbar, kmin, kmax, zh_floor, zh_mid, targets):
    r, t = _f64(rect), _f64(np.atleast_2d(targets))
    xyz = np.zeros(3 * len(t))
    ok = np.zeros(len(t), np.int32)
    lib().hho_preimage(_ptr(r), zbar, kmin, kmax, zh_floor, zh_mid, _ptr(t), len(t), _ptr(xyz), _ptr(ok, _i32p))
    return xyz.reshape(-1, 3), ok.astype(bool)


def jacobian_ts(rect, zbar, kmin, kmax, p):
    """Jacobian of (u, v, n) in (x, y, z) from the key points: diag(-1, -1, 1) T_s."""
    r, pp = _f64(rect), _f64(p)
    out = np.zeros(9)
    lib().hho_jacobian_ts(_ptr(r), zbar, kmin, kmax, _ptr(pp), _ptr(out))
    return out.reshape(3, 3)


def jacobian_s(rect, kmin, kmax, x, y, s):
    """Jacobian of (u, v, n) in (x, y, s = zh^2) used by the preimage solver."""
    r = _f64(rect)
    out = np.zeros(9)
    lib().hho_jacobian_s(_ptr(r), kmin, kmax, x, y, s, _ptr(out))
    return out.reshape(3, 3)


def ls_weights(taps, eta, tau):
    t = _f64(np.atleast_1d(tau))
    w = np.zeros(len(t) * taps)
    if lib().hho_ls_weights(taps, eta, _ptr(t), len(t), _ptr(w)) != 0:
        raise ValueError("bad kernel parameters")
    return w.reshape(len(t), taps)


class Plan:
    """The oracle's own subarray tree and sampling grids (never the library's)."""

    def __init__(self, traj, freqs, grid, leaf_size=32, merge_factor=4, eta=2.0, taps=6, os_r=16):
        self.traj = _f64(traj)
        self.freqs = _f64(freqs)
        self.grid = grid
        self.cfg = dict(leaf_size=leaf_size, merge_factor=merge_factor, eta=eta, taps=taps, os_r=os_r)
        g = _f64(grid.as_tuple())
        self._h = lib().hho_plan_create(_ptr(self.traj), len(self.traj), _ptr(self.freqs), len(self.freqs),
                                        _ptr(g), leaf_size, merge_factor, eta, taps, os_r)
        if not self._h:
            raise ValueError("oracle plan: bad arguments")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().hho_plan_destroy(self._h)
            self._h = None

    def info(self):
        out = np.zeros(3 + 130, np.int64)
        lib().hho_plan_info(self._h, _ptr(out, _ip))
        nl = int(out[0])
        return dict(n_levels=nl, n_nodes=int(out[1]), depth_leaves=int(out[2]),
                    level_start=out[3:3 + nl + 1].copy())

    def export(self):
        inf = self.info()
        nn = inf["n_nodes"]
        perm = np.zeros(len(self.traj), np.int64)
        ni = np.zeros(10 * nn, np.int64)
        nd = np.zeros(11 * nn)
        sc = np.zeros(6)
        lib().hho_plan_export(self._h, _ptr(perm, _ip), _ptr(ni, _ip), _ptr(nd), _ptr(sc))
        ni = ni.reshape(nn, 10)
        nd = nd.reshape(nn, 11)
        return dict(perm=perm, level=ni[:, 0], depth=ni[:, 1], t=ni[:, 2], begin=ni[:, 3], end=ni[:, 4],
                    child0=ni[:, 5], nchild=ni[:, 6], N=ni[:, 7:10], rect=nd[:, :4], lo=nd[:, 4:7],
                    eta=nd[:, 7:10], node_zbar=nd[:, 10],
                    zbar=sc[0], kmin=sc[1], kmax=sc[2], zh_floor=sc[3], zh_mid=sc[4], min_ext=sc[5],
                    **inf)

    def hhffbpa_adjoint(self, x, pts=None):
        """Adjoint of hhffbpa (image values x at the points -> echoes, complex128 [n_pos][n_f]):
        the forward map's conjugate transpose, taken step by step (final, merges, leaves, range
        compression); the forward's interpolation/fallback choices depend on geometry alone."""
        if pts is None:
            pts = self.grid.points()
        p = _f64(pts)
        xr = _ri(np.asarray(x, np.complex128).ravel())
        n_pos, n_f = len(self.traj), len(self.freqs)
        out = np.zeros(2 * n_pos * n_f)
        rc = lib().hho_hhffbpa_adjoint(self._h, _ptr(self.freqs), n_f, _ptr(xr), _ptr(p), len(p), _ptr(out))
        if rc != 0:
            raise RuntimeError(f"oracle hhffbpa adjoint failed: {rc}")
        return _cplx(out, (n_pos, n_f))

    def hhffbpa_traj_grad(self, echo, x, pts=None):
        """Gradient with respect to the positions (float64 [n_pos][3]) of L = Re sum conj(x) f,
        f = hhffbpa(echo, pts), with the plan held fixed: the leaves' and the exact fallbacks'
        BPA-RC terms differentiated, their values y carried by the adjoint traversal."""
        if pts is None:
            pts = self.grid.points()
        p = _f64(pts)
        e = _ri(echo)
        xr = _ri(np.asarray(x, np.complex128).ravel())
        out = np.zeros(3 * len(self.traj))
        rc = lib().hho_hhffbpa_traj_grad(self._h, _ptr(self.freqs), len(self.freqs), _ptr(e), _ptr(xr), _ptr(p),
                                         len(p), _ptr(out))
        if rc != 0:
            raise RuntimeError(f"oracle hhffbpa traj grad failed: {rc}")
        return out.reshape(len(self.traj), 3)

    def hhffbpa(self, echo, pts=None):
        """HHFFBPA values at the given points (default: all voxels).  Returns (values, stats)."""
        if pts is None:
            pts = self.grid.points()
        p = _f64(pts)
        e = _ri(echo)
        out = np.zeros(2 * len(p))
        st = np.zeros(80, np.int64)
        rc = lib().hho_hhffbpa(self._h, _ptr(self.freqs), len(self.freqs), _ptr(e), _ptr(p), len(p), _ptr(out),
                               _ptr(st, _ip))
        if rc != 0:
            raise RuntimeError(f"oracle hhffbpa failed: {rc}")
        nl = self.info()["n_levels"]
        return _cplx(out, (len(p),)), dict(fallbacks=int(st[0]), infeasible=int(st[1]), needed=int(st[2]),
                                           leaf_updates=int(st[3]), t_profiles=st[4] * 1e-9, t_topdown=st[5] * 1e-9,
                                           t_final=st[7] * 1e-9, t_levels=(st[8:8 + nl] * 1e-9).tolist(),
                                           needed_levels=st[40:40 + nl].tolist())


def nrmse_db(x, ref):
    """20 log10(||x - ref|| / ||ref||) over all entries, complex."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    return 20 * np.log10(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))


def rel_l2(x, ref):
    x = np.asarray(x)
    ref = np.asarray(ref)
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))
