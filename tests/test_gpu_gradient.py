"""GPU position gradient of direct BPA (bpa_traj_gradient) and its adjoint (bpa_adjoint)
against the FP64 oracle, and the differentiable image (bpa_image_with_offsets) against
finite differences of a loss.

The kernel differentiates the BPA sum term by term; the oracle does the same in FP64
(pinned by finite differences of its own BPA-RC on the CPU).  Tolerance: relative L2
<= 1e-4 over all positions for the FP32 kernel.
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


@pytest.mark.parametrize("name", ["small", "diff"])
def test_traj_gradient_matches_oracle(hh, name):
    s = synth.CONFIGS[name]()
    if name == "diff":
        e = synth.diff_echo(s, synth.diff_offsets(len(s.traj)), device="cuda")
    else:
        e = synth.scene_echo(s, device="cuda")
    g = s.grid
    rng = np.random.default_rng(11)
    idx = rng.choice(g.n_vox, 96, replace=False)
    gv = (rng.normal(size=96) + 1j * rng.normal(size=96)).astype(np.complex64)
    gimg = torch.zeros(g.n_vox, dtype=torch.complex64, device="cuda")
    gimg[torch.as_tensor(idx, device="cuda")] = torch.as_tensor(gv, device="cuda")
    got = hh.bpa_traj_gradient(s.traj, s.freqs, g, e, gimg.reshape(g.shape)).cpu().numpy()
    ref = oracle.bpa_rc_traj_grad(s.traj, s.freqs, e.cpu().numpy(), g.points(idx), gv.astype(np.complex128))
    assert got.shape == (len(s.traj), 3)
    assert oracle.rel_l2(got.ravel(), ref.ravel()) < REL_TOL


def _entropy(img):
    img = img.to(torch.complex128)  # the loss in FP64: differences of nearby losses stay resolved
    p = img.real ** 2 + img.imag ** 2
    q = p / p.sum()
    return -(q * torch.log(q + 1e-30)).sum()


def test_autofocus_loss_gradient_matches_finite_differences(hh):
    """Image entropy of the differentiable image of positions traj + offsets: the backward
    pass (hand-written kernel) against a central difference along a random smooth direction."""
    s = synth.small()
    offs_true = synth.diff_offsets(len(s.traj), seed=5, sigma_t=16.0, rms=5e-4)
    e = synth.diff_echo(s, offs_true, device="cuda")
    offsets = torch.zeros((len(s.traj), 3), dtype=torch.float64, requires_grad=True)
    loss = _entropy(hh.bpa_image_with_offsets(offsets, s.traj, s.freqs, s.grid, e))
    loss.backward()
    grad = offsets.grad.numpy()
    assert np.isfinite(grad).all() and np.abs(grad).max() > 0
    v = synth.diff_offsets(len(s.traj), seed=6, sigma_t=16.0, rms=1.0)
    h = 2e-6
    with torch.no_grad():
        lp = _entropy(hh.bpa_form_image(s.traj + h * v, s.freqs, s.grid, e)).item()
        lm = _entropy(hh.bpa_form_image(s.traj - h * v, s.freqs, s.grid, e)).item()
    fd = (lp - lm) / (2 * h)
    an = float((grad * v).sum())
    assert abs(fd - an) <= 2e-2 * abs(an), (fd, an)


@pytest.mark.parametrize("name", ["small", "diff"])
def test_bpa_adjoint_matches_oracle(hh, name):
    s = synth.CONFIGS[name]()
    g = s.grid
    rng = np.random.default_rng(12)
    idx = rng.choice(g.n_vox, 96, replace=False)
    xv = (rng.normal(size=96) + 1j * rng.normal(size=96)).astype(np.complex64)
    x = torch.zeros(g.n_vox, dtype=torch.complex64, device="cuda")
    x[torch.as_tensor(idx, device="cuda")] = torch.as_tensor(xv, device="cuda")
    got = hh.bpa_adjoint(s.traj, s.freqs, g, x.reshape(g.shape)).cpu().numpy()
    ref = oracle.bpa_rc_adjoint(s.traj, s.freqs, xv.astype(np.complex128), g.points(idx))
    assert got.shape == (len(s.traj), len(s.freqs))
    assert oracle.rel_l2(got.astype(np.complex128).ravel(), ref.ravel()) < REL_TOL


def test_bpa_adjoint_dot_product_with_forward(hh):
    """<x, A s> = <A^H x, s> with the GPU's forward and adjoint on a full grid (FP32)."""
    s = synth.small()
    rng = np.random.default_rng(13)
    e = torch.as_tensor((rng.normal(size=(len(s.traj), len(s.freqs)))
                         + 1j * rng.normal(size=(len(s.traj), len(s.freqs)))).astype(np.complex64), device="cuda")
    x = torch.as_tensor((rng.normal(size=s.grid.shape) + 1j * rng.normal(size=s.grid.shape)).astype(np.complex64),
                        device="cuda")
    fwd = hh.bpa_form_image(s.traj, s.freqs, s.grid, e)
    adj = hh.bpa_adjoint(s.traj, s.freqs, s.grid, x)
    lhs = torch.vdot(x.reshape(-1).to(torch.complex128), fwd.reshape(-1).to(torch.complex128)).item()
    rhs = torch.vdot(adj.reshape(-1).to(torch.complex128), e.reshape(-1).to(torch.complex128)).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
