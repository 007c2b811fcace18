"""GB300 HHFFBPA: fast factorized backprojection for near-range handheld SAR.

Thin Python binding over the C ABI declared in include/hhffbp.h (ctypes).  It
only marshals arguments: every step of imaging runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  If the
library is missing, every imaging call raises -- there is no CPU fallback.

    import paper_2506_23568_gb300 as hh
    plan = hh.Plan(traj, freqs, grid)                      # grid: hh.Grid or synth.Grid
    img = plan.form_image(echo)                            # echo: complex64 [n_pos][n_f] (cuda)
    ref = hh.bpa_form_image(traj, freqs, grid, echo)       # direct BPA on the same grid
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["Grid", "Config", "Plan", "bpa_form_image", "bpa_form_image_noalloc", "bpa_traj_gradient", "bpa_adjoint",
           "bpa_image_with_offsets", "hhffbpa_image_with_offsets", "lib", "LibraryError", "status_string", "SYMBOLS"]

HH_OK = 0
HH_ERR_ARG = 1
HH_ERR_FREQ_NONUNIFORM = 2
HH_ERR_OOM = 3
HH_ERR_CUDA = 4
HH_ERR_PLAN_NONCONVERGED = 5
HH_ERR_DEVICE_FLAG = 6
HH_ERR_UNIMPLEMENTED = 7
HH_ERR_HOST_ONLY = 8
HH_ERR_SCRATCH_LIMIT = 9
HH_FLAG_HOST_ONLY = 1
HH_FLAG_FP32_REFS = 2
MUFU_OPS = {"rsqrt": 0, "sin": 1, "cos": 2, "update_mix": 3}

# every symbol declared in include/hhffbp.h
SYMBOLS = ["hhffbp_default_config", "hhffbp_interp_weights", "hhffbp_plan", "hhffbp_plan_destroy", "hhffbp_plan_info", "hhffbp_plan_export",
           "hhffbp_form_image", "hhffbp_plan_counters", "hhffbp_plan_level_counts", "hhffbp_plan_profile",
           "hhffbp_plan_stage_times", "hhffbp_plan_preimages", "hhffbp_plan_tile_fill",
           "bpa_form_image", "bpa_form_image_noalloc", "bpa_traj_gradient", "bpa_adjoint", "hhffbp_adjoint",
           "hhffbp_traj_gradient", "hhffbp_plan_update_positions", "hh_mip",
           "hhffbp_batch_create", "hhffbp_batch_form_images", "hhffbp_batch_destroy",
           "hh_status_string",
           "hh_last_cuda_error",
           "hh_release_cached_memory", "hh_kernel_launches", "hh_mufu_throughput"]
STAGE_NAMES = {0: "range_compression", 1: "need_final", 2: "need_level", 3: "leaf_subimages", 4: "merge",
               5: "final", 6: "h2d", 7: "d2h"}


class LibraryError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = status_string(status) if _lib is not None else str(status)
        if status == HH_ERR_CUDA and _lib is not None:
            msg += f" (cudaError {_lib.hh_last_cuda_error()})"
        super().__init__(f"{what}: {msg}" if what else msg)


class hh_grid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class hh_config(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("merge_factor", ctypes.c_int32), ("eta", ctypes.c_float),
                ("taps", ctypes.c_int32), ("range_os", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class hh_plan_info(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("depth_leaves", ctypes.c_int32), ("n_nodes", ctypes.c_int64),
                ("level_nodes", ctypes.c_int64 * 32), ("level_samples", ctypes.c_int64 * 32),
                ("workspace_bytes", ctypes.c_int64), ("n_fft", ctypes.c_int64), ("gate_start", ctypes.c_int64),
                ("gate_bins", ctypes.c_int64), ("dR", ctypes.c_double), ("kc", ctypes.c_double)]


_lib = None


def lib(build_if_needed=True):
    """Load (building first when sources changed) the in-tree CUDA library."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_needed and _build.needs_build():
            _build.build()
        if not os.path.exists(path):
            raise LibraryError(HH_ERR_CUDA, f"CUDA library not built ({path})")
        L = ctypes.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    vp, dp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    L.hhffbp_default_config.argtypes = [ctypes.POINTER(hh_config)]
    L.hhffbp_interp_weights.argtypes = [ctypes.c_int32, ctypes.c_double, dp, ctypes.c_int64, dp]
    L.hhffbp_plan.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int32, ctypes.POINTER(hh_grid),
                              ctypes.POINTER(hh_config), vp, ctypes.POINTER(vp)]
    L.hhffbp_plan_destroy.argtypes = [vp]
    L.hhffbp_plan_info.argtypes = [vp, ctypes.POINTER(hh_plan_info)]
    L.hhffbp_plan_export.argtypes = [vp, i64p, i64p, dp, dp]
    L.hhffbp_form_image.argtypes = [vp, vp, vp, vp]
    L.hhffbp_plan_counters.argtypes = [vp, i64p]
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.hhffbp_plan_level_counts.argtypes = [vp, i64p, ctypes.c_int32]
    L.hhffbp_plan_preimages.argtypes = [vp, ctypes.c_int64, dp, ctypes.c_int64, dp, vp]
    L.hhffbp_plan_tile_fill.argtypes = [vp, ctypes.c_int32, i64p, vp]
    L.hhffbp_plan_profile.argtypes = [vp, ctypes.c_int]
    L.hhffbp_plan_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i32p, i32p, ctypes.c_int32, i32p]
    L.bpa_form_image.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int32, ctypes.POINTER(hh_grid),
                                 ctypes.POINTER(hh_config), vp, vp, vp]
    L.bpa_traj_gradient.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int32, ctypes.POINTER(hh_grid),
                                    ctypes.POINTER(hh_config), vp, vp, vp, vp]
    L.bpa_adjoint.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int32, ctypes.POINTER(hh_grid),
                              ctypes.POINTER(hh_config), vp, vp, vp]
    L.hhffbp_adjoint.argtypes = [vp, vp, vp, vp]
    L.hhffbp_traj_gradient.argtypes = [vp, vp, vp, vp, vp]
    L.hhffbp_plan_update_positions.argtypes = [vp, dp, vp]
    L.hh_mip.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, vp]
    L.hhffbp_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(vp)]
    L.hhffbp_batch_form_images.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.hhffbp_batch_destroy.argtypes = [vp]
    L.hh_status_string.argtypes = [ctypes.c_int]
    L.hh_status_string.restype = ctypes.c_char_p
    L.hh_last_cuda_error.argtypes = []
    L.hh_kernel_launches.argtypes = []
    L.hh_kernel_launches.restype = ctypes.c_longlong
    L.hh_mufu_throughput.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, i64p, ctypes.POINTER(ctypes.c_float)]
    L.hh_release_cached_memory.argtypes = []
    for name in SYMBOLS:
        f = getattr(L, name)
        if name != "hh_status_string":
            f.restype = ctypes.c_int


def interp_weights(taps, eta, tau):
    """The merge kernels' interpolation weights at fractional positions tau (float64 [n][taps])."""
    t = _f64(tau).ravel()
    out = np.zeros((len(t), int(taps)))
    _check(lib().hhffbp_interp_weights(int(taps), float(eta), t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       len(t), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "interp_weights")
    return out


def status_string(status):
    return lib().hh_status_string(int(status)).decode()


def _check(status, what):
    if status != HH_OK:
        raise LibraryError(status, what)


class Grid(hh_grid):
    """Output grid: voxel (a, b, c) at (x0 + a dx, y0 + b dy, z0 + c dz); image [nz][ny][nx]."""

    @classmethod
    def from_any(cls, g):
        if isinstance(g, hh_grid):
            return g
        t = g.as_tuple() if hasattr(g, "as_tuple") else tuple(g)
        return cls(*[float(v) for v in t[:6]], *[int(v) for v in t[6:]])

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def Config(**kw):
    """hh_config with the library defaults, overridden by keyword."""
    c = hh_config()
    _check(lib().hhffbp_default_config(ctypes.byref(c)), "default_config")
    for k, v in kw.items():
        if not hasattr(c, k):
            raise TypeError(f"unknown config field {k}")
        setattr(c, k, v)
    return c


def _f64(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _buffer_ptr(t):
    """Device or host data pointer of a contiguous complex64 tensor/array."""
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def _checked_ptr(t, numel, what, dtype="complex64", device_only=False):
    """Data pointer of a buffer the library reads or writes `numel` elements of, after checking
    its element type, size and contiguity (and, when device_only, that it lives on the current
    CUDA device): a wrong-sized buffer would otherwise be overrun by the kernels."""
    if hasattr(t, "data_ptr"):
        import torch

        if str(t.dtype) != f"torch.{dtype}":
            raise ValueError(f"{what}: dtype {t.dtype}, expected {dtype}")
        if t.numel() != numel:
            raise ValueError(f"{what}: {t.numel()} elements, expected {numel}")
        if not t.is_contiguous():
            raise ValueError(f"{what}: tensor must be contiguous")
        if device_only and (not t.is_cuda or t.device.index != torch.cuda.current_device()):
            raise ValueError(f"{what}: must be a tensor on the current CUDA device")
        return ctypes.c_void_p(t.data_ptr())
    a = t
    if str(a.dtype) != dtype:
        raise ValueError(f"{what}: dtype {a.dtype}, expected {dtype}")
    if a.size != numel:
        raise ValueError(f"{what}: {a.size} elements, expected {numel}")
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{what}: array must be C-contiguous")
    if device_only:
        raise ValueError(f"{what}: must be a tensor on the current CUDA device")
    return ctypes.c_void_p(a.ctypes.data)


def _n_vox(g):
    return int(g.nx) * int(g.ny) * int(g.nz)


class Plan:
    """A trajectory-specific HHFFBPA plan (tree + compressed sampling grids + workspace)."""

    def __init__(self, traj, freqs, grid, stream=None, host_only=False, **cfg):
        self.traj = _f64(traj)
        self.freqs = _f64(freqs)
        self.grid = Grid.from_any(grid)
        self.config = Config(**cfg)
        if host_only:
            self.config.flags |= HH_FLAG_HOST_ONLY
        L = lib()
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(0) if host_only else _stream_ptr(stream)
        st = L.hhffbp_plan(self.traj.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(self.traj),
                           self.freqs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(self.freqs),
                           ctypes.byref(self.grid), ctypes.byref(self.config), s, ctypes.byref(h))
        _check(st, "hhffbp_plan")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().hhffbp_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        i = hh_plan_info()
        _check(lib().hhffbp_plan_info(self._h, ctypes.byref(i)), "plan_info")
        nl = i.n_levels
        return dict(n_levels=nl, depth_leaves=i.depth_leaves, n_nodes=i.n_nodes,
                    level_nodes=list(i.level_nodes[:nl]), level_samples=list(i.level_samples[:nl]),
                    workspace_bytes=i.workspace_bytes, n_fft=i.n_fft, gate_start=i.gate_start,
                    gate_bins=i.gate_bins, dR=i.dR, kc=i.kc)

    def export(self):
        inf = self.info()
        nn = inf["n_nodes"]
        perm = np.zeros(len(self.traj), np.int64)
        ni = np.zeros((nn, 10), np.int64)
        nd = np.zeros((nn, 11))
        sc = np.zeros(5)
        _check(lib().hhffbp_plan_export(self._h, perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        ni.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        nd.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "plan_export")
        ls = np.concatenate([[0], np.cumsum(inf["level_nodes"])])
        return dict(perm=perm, level=ni[:, 0], depth=ni[:, 1], t=ni[:, 2], begin=ni[:, 3], end=ni[:, 4],
                    child0=ni[:, 5], nchild=ni[:, 6], N=ni[:, 7:10], rect=nd[:, :4], lo=nd[:, 4:7],
                    eta=nd[:, 7:10], node_zbar=nd[:, 10], level_start=ls, zbar=sc[0], kmin=sc[1], kmax=sc[2],
                    zh_floor=sc[3], zh_mid=sc[4], **inf)

    def form_image(self, echo, out=None, stream=None):
        """HHFFBPA image (complex64 [nz][ny][nx]) of echo (complex64 [n_pos][n_f]).

        echo/out may be CUDA tensors (used in place) or host tensors/arrays (copied
        inside the call).  Runs asynchronously on ``stream`` (default: torch's current)."""
        import torch

        if out is None:
            dev = echo.device if hasattr(echo, "device") else torch.device("cpu")
            out = torch.empty(self.grid.shape, dtype=torch.complex64, device=dev)
        n_echo = len(self.traj) * len(self.freqs)
        _check(lib().hhffbp_form_image(self._h, _checked_ptr(echo, n_echo, "echo"),
                                       _checked_ptr(out, _n_vox(self.grid), "out"), _stream_ptr(stream)),
               "hhffbp_form_image")
        return out

    def counters(self):
        """Synchronise and read the device counters of the last form_image."""
        out = np.zeros(8, np.int64)
        st = lib().hhffbp_plan_counters(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        c = dict(fallbacks=int(out[0]), infeasible=int(out[1]), newton_fail=int(out[2]), gate_miss=int(out[3]),
                 errors=int(out[4]), fallback_updates=int(out[5]), fallbacks_deferred=int(out[6]),
                 queue_full=int(out[7]))
        _check(st, f"plan_counters {c}")
        return c

    def preimages(self, node, targets, stream=None):
        """Device preimage solver on (u, v, n) targets of a node: (xyz float64[n][3], feasible bool[n])."""
        t = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((len(t), 4))
        _check(lib().hhffbp_plan_preimages(self._h, int(node), t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           len(t), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           _stream_ptr(stream)), "plan_preimages")
        return out[:, :3], out[:, 3] > 0.5

    def level_counts(self):
        """Samples evaluated per level in the last form_image (synchronises)."""
        out = np.zeros(32, np.int64)
        _check(lib().hhffbp_plan_level_counts(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 32),
               "plan_level_counts")
        return out[:self.info()["n_levels"]].tolist()

    def tile_fill(self, level, stream=None):
        """Histogram (int64 [257]) of the launch tiles of a non-root level by how many of their
        256 lattice samples the last form_image needed (synchronises)."""
        out = np.zeros(257, np.int64)
        _check(lib().hhffbp_plan_tile_fill(self._h, int(level), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           _stream_ptr(stream)), "plan_tile_fill")
        return out

    def profile(self, enable=True):
        """Record CUDA events between the stages of each form_image."""
        _check(lib().hhffbp_plan_profile(self._h, int(bool(enable))), "plan_profile")

    def stage_times(self):
        """[(stage name, level, ms)] of the last profiled form_image (synchronises)."""
        n = 64
        ms = (ctypes.c_float * n)()
        kind = (ctypes.c_int32 * n)()
        lev = (ctypes.c_int32 * n)()
        got = ctypes.c_int32()
        _check(lib().hhffbp_plan_stage_times(self._h, ms, kind, lev, n, ctypes.byref(got)), "plan_stage_times")
        return [(STAGE_NAMES.get(kind[i], str(kind[i])), int(lev[i]), float(ms[i])) for i in range(got.value)]

    def adjoint(self, image, out=None, stream=None):
        """Adjoint of form_image (reprojection): complex64 [n_pos][n_f] echoes of an image
        (complex64 [nz][ny][nx], CUDA or host).  Runs asynchronously on ``stream``."""
        import torch

        if out is None:
            dev = image.device if hasattr(image, "device") else torch.device("cpu")
            out = torch.empty((len(self.traj), len(self.freqs)), dtype=torch.complex64, device=dev)
        _check(lib().hhffbp_adjoint(self._h, _checked_ptr(image, _n_vox(self.grid), "image"),
                                    _checked_ptr(out, len(self.traj) * len(self.freqs), "out"), _stream_ptr(stream)),
               "hhffbp_adjoint")
        return out

    def update_positions(self, traj, stream=None):
        """Replace the positions (float64 [n_pos][3]) and keep the plan: tree, sampling grids and
        range gate of the trajectory it was built from (synchronises)."""
        t = _f64(traj)
        if t.shape != self.traj.shape:
            raise ValueError(f"traj: shape {t.shape}, expected {self.traj.shape}")
        s = ctypes.c_void_p(0) if self.config.flags & HH_FLAG_HOST_ONLY else _stream_ptr(stream)
        _check(lib().hhffbp_plan_update_positions(self._h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), s),
               "hhffbp_plan_update_positions")
        self.traj = t

    def traj_gradient(self, echo, grad_image, out=None, stream=None):
        """Gradient with respect to the positions (float64 [n_pos][3], trajectory order) of a real
        loss of form_image(echo), with the plan held fixed; grad_image is the loss's gradient with
        respect to the image (complex64 CUDA tensor, torch's convention dL = Re sum conj(g) df)."""
        import torch

        gi = grad_image.contiguous()
        if gi.dtype != torch.complex64:
            gi = gi.to(torch.complex64)
        if out is None:
            out = torch.empty((len(self.traj), 3), dtype=torch.float64, device=gi.device)
        _check(lib().hhffbp_traj_gradient(self._h, _checked_ptr(echo, len(self.traj) * len(self.freqs), "echo"),
                                          _checked_ptr(gi, _n_vox(self.grid), "grad_image", device_only=True),
                                          _checked_ptr(out, 3 * len(self.traj), "out", dtype="float64",
                                                       device_only=True), _stream_ptr(stream)),
               "hhffbp_traj_gradient")
        return out


class Batch:
    """Many scans, one plan each, imaged by one CUDA graph launch (hhffbp_batch_*): the first
    form_images call (and any call with other buffers) records the scans into a graph whose
    branches run them concurrently; later calls replay it.  The plans must outlive the batch."""

    def __init__(self, plans, n_streams=8):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib().hhffbp_batch_create(arr, len(self.plans), int(n_streams), ctypes.byref(h)), "hhffbp_batch_create")
        self._h = h

    def form_images(self, echos, images=None, stream=None):
        """echos: complex64 CUDA tensors [n_pos_i][n_f_i]; returns (or fills) the images."""
        import torch

        if images is None:
            images = [torch.empty(p.grid.shape, dtype=torch.complex64, device=e.device)
                      for p, e in zip(self.plans, echos)]
        if len(echos) != len(self.plans) or len(images) != len(self.plans):
            raise ValueError("one echo and one image per plan")
        ep = (ctypes.c_void_p * len(echos))(*[_checked_ptr(e, len(p.traj) * len(p.freqs), "echo",
                                                           device_only=True).value
                                              for p, e in zip(self.plans, echos)])
        ip = (ctypes.c_void_p * len(images))(*[_checked_ptr(im, _n_vox(p.grid), "image", device_only=True).value
                                               for p, im in zip(self.plans, images)])
        _check(lib().hhffbp_batch_form_images(self._h, ep, ip, _stream_ptr(stream)), "hhffbp_batch_form_images")
        return images

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().hhffbp_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mip(image, axis=0, out=None, stream=None):
    """Maximum-intensity projection max |f| of a complex64 CUDA image [nz][ny][nx] along z
    (axis 0 -> [ny][nx]), y (axis 1 -> [nz][nx]) or x (axis 2 -> [nz][ny]); float32."""
    import torch

    nz, ny, nx = image.shape
    shape = [(ny, nx), (nz, nx), (nz, ny)][axis]
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=image.device)
    _check(lib().hh_mip(_checked_ptr(image, nx * ny * nz, "image", device_only=True), nx, ny, nz, int(axis),
                        _checked_ptr(out, shape[0] * shape[1], "out", dtype="float32", device_only=True),
                        _stream_ptr(stream)), "hh_mip")
    return out


def release_cached_memory():
    """Free device blocks cached by the library for reuse by later plans."""
    _check(lib().hh_release_cached_memory(), "release_cached_memory")


def kernel_launches():
    """Kernel launches the library has issued in this process (a counter; differences count
    the launches of a region)."""
    return int(lib().hh_kernel_launches())


def mufu_throughput(op="update_mix", iters=4096, stream=None):
    """Measured special-function-unit rate on the current device: (MUFU results per
    second, results, milliseconds) of one timed probe launch.  op: 'rsqrt', 'sin', 'cos' or
    'update_mix' (one rsqrt feeding one sine and one cosine, as in a backprojection update)."""
    ops, ms = ctypes.c_int64(0), ctypes.c_float(0)
    _check(lib().hh_mufu_throughput(MUFU_OPS[op], int(iters), _stream_ptr(stream), ctypes.byref(ops),
                                    ctypes.byref(ms)), "mufu_throughput")
    return ops.value / (ms.value * 1e-3), ops.value, ms.value


def bpa_form_image(traj, freqs, grid, echo, out=None, stream=None, range_os=16, flags=0):
    """Direct BPA on range-compressed data (complex64 [nz][ny][nx]).  flags: HH_FLAG_FP32_REFS
    takes the per-tile reference ranges and phases in FP32 (precision study)."""
    import torch

    t, f = _f64(traj), _f64(freqs)
    g = Grid.from_any(grid)
    cfg = Config(range_os=range_os, flags=flags)
    if out is None:
        dev = echo.device if hasattr(echo, "device") else torch.device("cpu")
        out = torch.empty(g.shape, dtype=torch.complex64, device=dev)
    _check(lib().bpa_form_image(t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t),
                                f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(f), ctypes.byref(g),
                                ctypes.byref(cfg), _checked_ptr(echo, len(t) * len(f), "echo"),
                                _checked_ptr(out, _n_vox(g), "out"), _stream_ptr(stream)),
           "bpa_form_image")
    return out


def bpa_traj_gradient(traj, freqs, grid, echo, grad_image, out=None, stream=None, range_os=16):
    """Gradient of a real loss of the direct BPA image with respect to the positions:
    grad_image is the loss's gradient with respect to the image (complex64 CUDA tensor
    [nz][ny][nx], torch's convention dL = Re sum conj(g) df); returns float64 [n_pos][3] on
    the image's device."""
    import torch

    t, f = _f64(traj), _f64(freqs)
    g = Grid.from_any(grid)
    cfg = Config(range_os=range_os)
    gi = grad_image.contiguous()
    if gi.dtype != torch.complex64:
        gi = gi.to(torch.complex64)
    if out is None:
        out = torch.empty((len(t), 3), dtype=torch.float64, device=gi.device)
    _check(lib().bpa_traj_gradient(t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t),
                                   f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(f), ctypes.byref(g),
                                   ctypes.byref(cfg), _checked_ptr(echo, len(t) * len(f), "echo"),
                                   _checked_ptr(gi, _n_vox(g), "grad_image", device_only=True),
                                   _checked_ptr(out, 3 * len(t), "out", dtype="float64", device_only=True),
                                   _stream_ptr(stream)),
           "bpa_traj_gradient")
    return out


def bpa_adjoint(traj, freqs, grid, image, out=None, stream=None, range_os=16):
    """Adjoint of bpa_form_image (reprojection): complex64 [n_pos][n_f] echoes from a complex64
    CUDA image [nz][ny][nx]."""
    import torch

    t, f = _f64(traj), _f64(freqs)
    g = Grid.from_any(grid)
    cfg = Config(range_os=range_os)
    x = image.contiguous()
    if x.dtype != torch.complex64:
        x = x.to(torch.complex64)
    if out is None:
        out = torch.empty((len(t), len(f)), dtype=torch.complex64, device=x.device)
    _check(lib().bpa_adjoint(t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t),
                             f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(f), ctypes.byref(g),
                             ctypes.byref(cfg), _checked_ptr(x, _n_vox(g), "image", device_only=True),
                             _checked_ptr(out, len(t) * len(f), "out", device_only=True), _stream_ptr(stream)),
           "bpa_adjoint")
    return out


def _bpa_offsets_function():
    import torch

    class _BPAOffsets(torch.autograd.Function):
        """Direct BPA image of the positions traj + offsets; the backward pass is the
        hand-written gradient kernel (bpa_traj_gradient)."""

        @staticmethod
        def forward(ctx, offsets, traj, freqs, grid, echo, range_os):
            pos = np.asarray(traj, np.float64) + offsets.detach().cpu().numpy().astype(np.float64)
            ctx.pos, ctx.freqs, ctx.grid, ctx.echo, ctx.range_os = pos, freqs, grid, echo, range_os
            ctx.offsets_device = offsets.device
            return bpa_form_image(pos, freqs, grid, echo, range_os=range_os)

        @staticmethod
        def backward(ctx, grad_image):
            g = bpa_traj_gradient(ctx.pos, ctx.freqs, ctx.grid, ctx.echo, grad_image, range_os=ctx.range_os)
            return g.to(ctx.offsets_device), None, None, None, None, None

    return _BPAOffsets


_BPA_OFFSETS = None


def _hh_offsets_function():
    import torch

    class _HHOffsets(torch.autograd.Function):
        """HHFFBPA image, with a plan held fixed, of the positions nominal + offsets; the backward
        pass is the hand-written adjoint traversal (Plan.traj_gradient)."""

        @staticmethod
        def forward(ctx, offsets, plan, nominal, echo):
            pos = nominal + offsets.detach().cpu().numpy().astype(np.float64)
            plan.update_positions(pos)
            ctx.plan, ctx.pos, ctx.echo, ctx.offsets_device = plan, pos, echo, offsets.device
            return plan.form_image(echo)

        @staticmethod
        def backward(ctx, grad_image):
            if not np.array_equal(ctx.plan.traj, ctx.pos):  # the plan was moved since: put the positions back
                ctx.plan.update_positions(ctx.pos)
            g = ctx.plan.traj_gradient(ctx.echo, grad_image)
            return g.to(ctx.offsets_device), None, None, None

    return _HHOffsets


_HH_OFFSETS = None


def hhffbpa_image_with_offsets(offsets, plan, echo, nominal=None):
    """Differentiable HHFFBPA image (complex64 CUDA tensor) of the positions nominal + offsets
    (offsets a float64 tensor [n_pos][3]; autofocus of uncertain handheld tracks).  The plan --
    tree, sampling grids and range gate of the track it was built from -- is held fixed: the
    forward pass moves its positions (Plan.update_positions) and the backward pass is the
    adjoint traversal (Plan.traj_gradient).  nominal defaults to the plan's current positions."""
    global _HH_OFFSETS
    if _HH_OFFSETS is None:
        _HH_OFFSETS = _hh_offsets_function()
    nom = np.array(plan.traj if nominal is None else nominal, np.float64)
    return _HH_OFFSETS.apply(offsets, plan, nom, echo)


def bpa_image_with_offsets(offsets, traj, freqs, grid, echo, range_os=16):
    """Differentiable direct BPA image (complex64 CUDA tensor) of the positions traj +
    offsets, offsets a float64 tensor [n_pos][3] (autofocus of uncertain tracks)."""
    global _BPA_OFFSETS
    if _BPA_OFFSETS is None:
        _BPA_OFFSETS = _bpa_offsets_function()
    return _BPA_OFFSETS.apply(offsets, traj, freqs, grid, echo, range_os)


def bpa_form_image_noalloc(traj, freqs, grid, echo, out, stream=None, range_os=16):
    """Direct BPA through the entry point with a fixed device workspace (no
    allocation inside the call).  echo and out must be device tensors of the
    current device; out is complex64 [nz][ny][nx] and is required."""
    t, f = _f64(traj), _f64(freqs)
    g = Grid.from_any(grid)
    cfg = Config(range_os=range_os)
    _check(lib().bpa_form_image_noalloc(t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t),
                                        f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(f), ctypes.byref(g),
                                        ctypes.byref(cfg),
                                        _checked_ptr(echo, len(t) * len(f), "echo", device_only=True),
                                        _checked_ptr(out, _n_vox(g), "out", device_only=True), _stream_ptr(stream)),
           "bpa_form_image_noalloc")
    return out
