"""bpa_form_image_noalloc (fixed device workspace, no allocation inside the call)
against the allocating bpa_form_image, through the C ABI.

Two calls in a row must each reproduce bpa_form_image within the FP32 path's
tolerance (relative L2 <= 1e-4): the second call reuses the workspace the first
one left behind.  Problems beyond the workspace and host buffers are refused.
"""
import ctypes

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


def _rel(a, b):
    return oracle.rel_l2(a.cpu().numpy().astype(np.complex128).ravel(), b.cpu().numpy().astype(np.complex128).ravel())


@pytest.mark.parametrize("name", ["small", "tiny"])
def test_noalloc_matches_allocating_bpa_twice(hh, name):
    s = synth.CONFIGS[name]()
    e = synth.scene_echo(s, device="cuda")
    ref = hh.bpa_form_image(s.traj, s.freqs, s.grid, e)
    out1 = torch.full(s.grid.shape, float("nan"), dtype=torch.complex64, device="cuda")
    out2 = torch.full(s.grid.shape, float("nan"), dtype=torch.complex64, device="cuda")
    hh.bpa_form_image_noalloc(s.traj, s.freqs, s.grid, e, out1)
    hh.bpa_form_image_noalloc(s.traj, s.freqs, s.grid, e, out2)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(out1)).all() and torch.isfinite(torch.view_as_real(out2)).all()
    assert _rel(out1, ref) < REL_TOL
    assert _rel(out2, ref) < REL_TOL
    # a further call changes neither the device's free memory nor torch's pools
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    hh.bpa_form_image_noalloc(s.traj, s.freqs, s.grid, e, out1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_reserved() == reserved0
    assert _rel(out1, ref) < REL_TOL


def test_noalloc_refuses_oversize_and_host_buffers(hh):
    big = synth.CONFIGS["large"]()  # 65,536 positions: profiles far beyond the fixed workspace
    e = torch.zeros((len(big.traj), len(big.freqs)), dtype=torch.complex64, device="cuda")
    out = torch.zeros(big.grid.shape, dtype=torch.complex64, device="cuda")
    with pytest.raises(hh.LibraryError) as ei:
        hh.bpa_form_image_noalloc(big.traj, big.freqs, big.grid, e, out)
    assert ei.value.status == hh.HH_ERR_SCRATCH_LIMIT
    s = synth.CONFIGS["small"]()
    e_host = synth.scene_echo(s, device="cpu")
    out_dev = torch.empty(s.grid.shape, dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError, match="CUDA device"):  # refused by the binding before the call
        hh.bpa_form_image_noalloc(s.traj, s.freqs, s.grid, e_host, out_dev)
    # the library itself refuses host buffers too
    L = hh.lib()
    t, f = np.ascontiguousarray(s.traj, np.float64), np.ascontiguousarray(s.freqs, np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    g, cfg = hh.Grid.from_any(s.grid), hh.Config()
    st = L.bpa_form_image_noalloc(t.ctypes.data_as(dp), len(t), f.ctypes.data_as(dp), len(f), ctypes.byref(g),
                                  ctypes.byref(cfg), ctypes.c_void_p(e_host.data_ptr()),
                                  ctypes.c_void_p(out_dev.data_ptr()), None)
    assert st == hh.HH_ERR_ARG
