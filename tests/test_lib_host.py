"""CPU tests of the C-ABI library: it loads, exports every declared symbol, and
its host planning (tree, sampling grids) equals the oracle's independent plan.
No compute call touches a GPU here (plans are built with HH_FLAG_HOST_ONLY)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2506_23568_gb300 as hh
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "hhffbp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:long\s+long|\w+)\s*\*?\s*(\w+)\s*\(", txt, flags=re.M)))


def test_library_exports_every_declared_symbol():
    L = hh.lib()
    declared = _declared_functions()
    assert set(declared) == set(hh.SYMBOLS)
    for name in declared:
        assert isinstance(getattr(L, name), ctypes._CFuncPtr)


def test_status_strings_and_defaults():
    assert hh.status_string(hh.HH_OK) == "ok"
    assert "not implemented" in hh.status_string(hh.HH_ERR_UNIMPLEMENTED)
    c = hh.Config()
    assert (c.leaf_size, c.merge_factor, c.taps, c.range_os) == (32, 4, 6, 16)
    assert c.eta == pytest.approx(2.0)


def _compare_plans(ge, oe):
    for k in ["level", "depth", "t", "begin", "end", "nchild", "N"]:
        np.testing.assert_array_equal(ge[k], oe[k], err_msg=k)
    has = ge["nchild"] > 0
    np.testing.assert_array_equal(ge["child0"][has], oe["child0"][has])
    ls = ge["level_start"]
    for k in range(ls[0], ls[-2]):  # every node's member set (order within a node is free)
        assert set(ge["perm"][ge["begin"][k]:ge["end"][k]]) == set(oe["perm"][oe["begin"][k]:oe["end"][k]])
    nonroot = slice(0, ls[-2])
    np.testing.assert_allclose(ge["rect"], oe["rect"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(ge["node_zbar"], oe["node_zbar"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(ge["lo"][nonroot], oe["lo"][nonroot], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(ge["eta"][nonroot], oe["eta"][nonroot])
    for k in ["zbar", "kmin", "kmax", "zh_floor", "zh_mid"]:  # the plan scalars
        assert ge[k] == pytest.approx(oe[k], rel=1e-14, abs=1e-15), k


@pytest.mark.parametrize("name,cfg", [("tiny", dict(leaf_size=32)), ("small", dict(leaf_size=16)),
                                      ("small", dict(leaf_size=8, merge_factor=2, taps=4, eta=1.5)),
                                      ("mid", dict(leaf_size=64)), ("large", dict(leaf_size=64))])
def test_host_plan_equals_oracle_plan(name, cfg):
    s = synth.CONFIGS[name]()
    ge = hh.Plan(s.traj, s.freqs, s.grid, host_only=True, **cfg).export()
    oe = oracle.Plan(s.traj, s.freqs, s.grid, **cfg).export()
    assert ge["n_levels"] == oe["n_levels"] and ge["depth_leaves"] == oe["depth_leaves"]
    _compare_plans(ge, oe)


def test_host_plan_ragged_position_count():
    s = synth.small()
    traj = s.traj[:229]  # not a power of two; leaves of 14 and 15 members
    ge = hh.Plan(traj, s.freqs, s.grid, host_only=True, leaf_size=14).export()
    oe = oracle.Plan(traj, s.freqs, s.grid, leaf_size=14).export()
    sizes = ge["end"][:ge["level_start"][1]] - ge["begin"][:ge["level_start"][1]]
    assert set(sizes.tolist()) <= {14, 15}
    _compare_plans(ge, oe)


def test_host_plan_single_level():
    s = synth.small()
    p = hh.Plan(s.traj, s.freqs, s.grid, host_only=True, leaf_size=10 ** 6)
    assert p.info()["n_levels"] == 1


def test_gate_covers_grid_ranges():
    s = synth.tiny()
    inf = hh.Plan(s.traj, s.freqs, s.grid, host_only=True).info()
    pts = s.grid.points()[::97]
    R = np.linalg.norm(pts[:, None, :] - s.traj[None, ::13, :], axis=2)
    assert R.min() / inf["dR"] >= inf["gate_start"] and R.max() / inf["dR"] + 1 < inf["gate_start"] + inf["gate_bins"]


@pytest.mark.parametrize("mutate,status", [
    (lambda a: a.update(traj=a["traj"][:0]), hh.HH_ERR_ARG),
    (lambda a: a.update(freqs=np.array([77e9])), hh.HH_ERR_ARG),
    (lambda a: a.update(freqs=a["freqs"] * np.r_[1.0, np.ones(len(a["freqs"]) - 2) * 1.001, 1.0]),
     hh.HH_ERR_FREQ_NONUNIFORM),
    (lambda a: a.update(freqs=a["freqs"][::-1].copy()), hh.HH_ERR_FREQ_NONUNIFORM),
    (lambda a: a.update(cfg=dict(taps=5)), hh.HH_ERR_ARG),
    (lambda a: a.update(cfg=dict(merge_factor=3)), hh.HH_ERR_ARG),
    (lambda a: a.update(cfg=dict(eta=0.5)), hh.HH_ERR_ARG),
    (lambda a: a.update(cfg=dict(leaf_size=0)), hh.HH_ERR_ARG),
    (lambda a: a.update(grid=synth.Grid(-0.01, -0.01, -0.5, 1e-3, 1e-3, 1e-2, 4, 4, 4)), hh.HH_ERR_ARG),
    (lambda a: a.update(grid=synth.Grid(-0.01, -0.01, 0.2, 1e-3, 1e-3, 1e-2, 0, 4, 4)), hh.HH_ERR_ARG),
    (lambda a: a.update(grid=synth.Grid(-0.01, -0.01, 0.2, -1e-3, 1e-3, 1e-2, 4, 4, 4)), hh.HH_ERR_ARG),
])
def test_plan_argument_errors(mutate, status):
    s = synth.small()
    a = dict(traj=s.traj, freqs=s.freqs, grid=s.grid, cfg={})
    mutate(a)
    with pytest.raises(hh.LibraryError) as ei:
        hh.Plan(a["traj"], a["freqs"], a["grid"], host_only=True, **a["cfg"])
    assert ei.value.status == status


def test_host_only_plan_refuses_imaging():
    s = synth.small()
    p = hh.Plan(s.traj, s.freqs, s.grid, host_only=True)
    L = hh.lib()
    buf = np.zeros(16, np.complex64)
    st = L.hhffbp_form_image(p._h, ctypes.c_void_p(buf.ctypes.data), ctypes.c_void_p(buf.ctypes.data), None)
    assert st == hh.HH_ERR_HOST_ONLY
    assert L.hhffbp_form_image(None, None, None, None) == hh.HH_ERR_ARG
    assert L.hhffbp_adjoint(p._h, None, None, None) == hh.HH_ERR_ARG
    cbuf = ctypes.c_void_p(buf.ctypes.data)
    assert L.hhffbp_adjoint(p._h, cbuf, cbuf, None) == hh.HH_ERR_HOST_ONLY
    assert L.hhffbp_traj_gradient(p._h, cbuf, cbuf, cbuf, None) == hh.HH_ERR_HOST_ONLY
    # a host-only plan takes new positions without any CUDA call
    p.update_positions(s.traj + 1e-4)
    assert np.allclose(p.traj, s.traj + 1e-4)
    with pytest.raises(ValueError):
        p.update_positions(s.traj[:-1])


@pytest.mark.parametrize("taps,eta", [(4, 2.0), (6, 1.6), (6, 1.75), (6, 2.0)])
def test_kernel_interp_weights_match_oracle_least_squares(taps, eta):
    """The merge kernels' interpolation weights (FP32 polynomials, evaluated as the kernels do)
    against the oracle's least-squares weights: within the FP32 rounding level everywhere on
    [0, 1), exact partition of unity to that level, and the identity at tau = 0."""
    tau = np.linspace(0.0, 1.0, 2001, endpoint=False)
    got = hh.interp_weights(taps, eta, tau)
    ref = oracle.ls_weights(taps, eta, tau)
    assert np.abs(got - ref).max() < 5e-7
    o = np.arange(-(taps // 2 - 1), taps // 2 + 1)
    np.testing.assert_allclose(got[0], (o == 0).astype(float), atol=5e-7)


def test_kernel_interp_weights_reject_bad_arguments():
    with pytest.raises(hh.LibraryError):
        hh.interp_weights(5, 2.0, [0.5])
    with pytest.raises(hh.LibraryError):
        hh.interp_weights(6, 0.5, [0.5])


def test_gradient_and_adjoint_refuse_null_buffers_without_cuda():
    """Argument errors of the direct-BPA gradient and adjoint entry points are returned before
    any CUDA call (no device needed): null echo/image/gradient buffers and bad inputs."""
    L = hh.lib()
    s = synth.small()
    t = np.ascontiguousarray(s.traj, np.float64)
    f = np.ascontiguousarray(s.freqs, np.float64)
    g = hh.Grid.from_any(s.grid)
    cfg = hh.Config(range_os=16)
    dp = ctypes.POINTER(ctypes.c_double)
    tp, fp = t.ctypes.data_as(dp), f.ctypes.data_as(dp)
    dummy = ctypes.c_void_p(1)
    assert L.bpa_traj_gradient(tp, len(t), fp, len(f), ctypes.byref(g), ctypes.byref(cfg), None, dummy, dummy,
                               None) == hh.HH_ERR_ARG
    assert L.bpa_traj_gradient(tp, len(t), fp, len(f), ctypes.byref(g), ctypes.byref(cfg), dummy, None, dummy,
                               None) == hh.HH_ERR_ARG
    assert L.bpa_traj_gradient(tp, len(t), fp, len(f), ctypes.byref(g), ctypes.byref(cfg), dummy, dummy, None,
                               None) == hh.HH_ERR_ARG
    assert L.bpa_adjoint(tp, len(t), fp, len(f), ctypes.byref(g), ctypes.byref(cfg), None, dummy,
                         None) == hh.HH_ERR_ARG
    assert L.bpa_adjoint(tp, len(t), fp, len(f), ctypes.byref(g), ctypes.byref(cfg), dummy, None,
                         None) == hh.HH_ERR_ARG
    assert L.bpa_adjoint(tp, 0, fp, len(f), ctypes.byref(g), ctypes.byref(cfg), dummy, dummy,
                         None) == hh.HH_ERR_ARG


def test_wrappers_refuse_wrong_buffers_before_any_cuda_call():
    """The binding checks element type, element count and placement of every buffer the
    kernels read or write before calling the library: a wrong-sized output would otherwise be
    overrun on the device."""
    torch = pytest.importorskip("torch")
    s = synth.small()
    echo = torch.zeros((len(s.traj), len(s.freqs)), dtype=torch.complex64)
    with pytest.raises(ValueError, match="elements"):
        hh.bpa_form_image(s.traj, s.freqs, s.grid, echo, out=torch.zeros(10, dtype=torch.complex64))
    with pytest.raises(ValueError, match="dtype"):
        hh.bpa_form_image(s.traj, s.freqs, s.grid, echo.to(torch.complex128),
                          out=torch.zeros(s.grid.shape, dtype=torch.complex64))
    with pytest.raises(ValueError, match="elements"):
        hh.bpa_form_image(s.traj, s.freqs, s.grid, echo[:-1], out=torch.zeros(s.grid.shape, dtype=torch.complex64))
    # the fixed-workspace variant takes device buffers of the current device only
    with pytest.raises(ValueError, match="CUDA device"):
        hh.bpa_form_image_noalloc(s.traj, s.freqs, s.grid, echo, torch.zeros(s.grid.shape, dtype=torch.complex64))
    plan = hh.Plan(s.traj, s.freqs, s.grid, host_only=True, leaf_size=16)
    with pytest.raises(ValueError, match="elements"):
        plan.form_image(echo, out=torch.zeros(7, dtype=torch.complex64))


def test_mufu_probe_refuses_bad_arguments():
    """Argument checks come before any CUDA call, so they hold without a device."""
    L = hh.lib()
    ops, ms = ctypes.c_int64(0), ctypes.c_float(0)
    assert L.hh_mufu_throughput(7, 16, None, ctypes.byref(ops), ctypes.byref(ms)) == hh.HH_ERR_ARG
    assert L.hh_mufu_throughput(0, 0, None, ctypes.byref(ops), ctypes.byref(ms)) == hh.HH_ERR_ARG
    assert L.hh_mufu_throughput(0, 16, None, None, ctypes.byref(ms)) == hh.HH_ERR_ARG


def _raster(nx_pos, ny_pos, pitch=0.004, z=0.0):
    """A regular raster of positions: every x value repeats across the rows (and every y value
    along a row), so that the k-d split's (coordinate, index) order is decided by the index
    inside runs of equal coordinates."""
    xs, ys = np.meshgrid(np.arange(nx_pos) * pitch, np.arange(ny_pos) * pitch, indexing="ij")
    return np.column_stack([xs.ravel() - xs.mean(), ys.ravel() - ys.mean(), np.full(xs.size, z)])


@pytest.mark.parametrize("shape,leaf", [((64, 64), 16), ((48, 40), 15), ((128, 96), 64)])
def test_host_plan_equals_oracle_plan_with_tied_coordinates(shape, leaf):
    """Runs of equal x (and y) coordinates straddle the split points: the bucket selection of
    the library's split must give exactly the oracle's halves."""
    s = synth.small()
    traj = _raster(*shape)
    ge = hh.Plan(traj, s.freqs, s.grid, host_only=True, leaf_size=leaf).export()
    oe = oracle.Plan(traj, s.freqs, s.grid, leaf_size=leaf).export()
    assert ge["n_levels"] == oe["n_levels"] and ge["depth_leaves"] == oe["depth_leaves"]
    _compare_plans(ge, oe)


def test_host_plan_equals_oracle_plan_on_a_line():
    """All positions share one x coordinate (a line along y): the splits along x fall back to
    ordering by index alone."""
    s = synth.small()
    n = 3000
    traj = np.column_stack([np.zeros(n), np.linspace(-0.06, 0.06, n), np.zeros(n)])
    ge = hh.Plan(traj, s.freqs, s.grid, host_only=True, leaf_size=20).export()
    oe = oracle.Plan(traj, s.freqs, s.grid, leaf_size=20).export()
    _compare_plans(ge, oe)


def test_host_plans_built_concurrently_equal_one_built_alone():
    """Plans built at once from several host threads (the C call releases the interpreter
    lock) share the library's worker pool, which serves one loop at a time; the others run
    their loops on threads of their own. Every plan must equal the one built alone."""
    import threading

    s = synth.CONFIGS["mid"]()
    ref = hh.Plan(s.traj, s.freqs, s.grid, host_only=True, leaf_size=256).export()
    out = [None] * 4

    def build(i):
        out[i] = hh.Plan(s.traj, s.freqs, s.grid, host_only=True, leaf_size=256).export()

    threads = [threading.Thread(target=build, args=(i,)) for i in range(len(out))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for e in out:
        for k in ["begin", "end", "N", "child0", "nchild"]:
            np.testing.assert_array_equal(e[k], ref[k], err_msg=k)
        np.testing.assert_array_equal(e["rect"], ref["rect"])
        np.testing.assert_array_equal(e["lo"], ref["lo"])
        ls = ref["level_start"]
        for k in range(ls[0], ls[-2]):
            assert set(e["perm"][e["begin"][k]:e["end"][k]]) == set(ref["perm"][ref["begin"][k]:ref["end"][k]])
