"""GPU adjoint (hhffbp_adjoint) and position gradient (hhffbp_traj_gradient) of the fast
method, through the C ABI, against the FP64 oracle's step-by-step transposes
(Plan.hhffbpa_adjoint, Plan.hhffbpa_traj_grad; pinned on the CPU by the dot-product identity
and by finite differences), the dot-product identity with the GPU's own forward, and finite
differences of an image-entropy loss with the plan held fixed.

Tolerances: relative L2 <= 1e-4 against the oracle (the FP32 path), 1e-5 for the
dot-product identity, 2e-2 for the finite difference of the FP64-reduced loss.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-4
# 4-way merges; 2-way merges with 4 taps; sparse lattices whose footprints meet infeasible
# samples and leave lattices (exact fallbacks at every level); a deeper tree on the
# differentiation scene
CASES = [("small", dict(leaf_size=16)), ("small", dict(leaf_size=8, merge_factor=2, taps=4, eta=1.5)),
         ("tiny", dict(leaf_size=32, eta=1.25)), ("diff", dict(leaf_size=64))]


@pytest.fixture(scope="module")
def hh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_23568_gb300 as m

    m.lib()
    return m


def _echo(name, s, device="cuda"):
    if name == "diff":
        return synth.diff_echo(s, synth.diff_offsets(len(s.traj)), device=device)
    return synth.scene_echo(s, device=device)


def _image_values(name, g, seed):
    """Image-domain values: every voxel of the small scenes; 96 random voxels of the larger ones
    (zero elsewhere), so that the oracle evaluates only those."""
    rng = np.random.default_rng(seed)
    idx = np.arange(g.n_vox) if g.n_vox <= 70000 else np.sort(rng.choice(g.n_vox, 96, replace=False))
    v = (rng.normal(size=len(idx)) + 1j * rng.normal(size=len(idx))).astype(np.complex64)
    full = torch.zeros(g.n_vox, dtype=torch.complex64, device="cuda")
    full[torch.as_tensor(idx, device="cuda")] = torch.as_tensor(v, device="cuda")
    return idx, v.astype(np.complex128), full.reshape(g.shape)


@pytest.mark.parametrize("name,cfg", CASES)
def test_fast_adjoint_matches_oracle(hh, name, cfg):
    s = synth.CONFIGS[name]()
    g = s.grid
    idx, xv, x = _image_values(name, g, 21)
    plan = hh.Plan(s.traj, s.freqs, g, **cfg)
    got = plan.adjoint(x)
    cnt = plan.counters()
    assert cnt["gate_miss"] == 0 and cnt["errors"] == 0, cnt
    ref = oracle.Plan(s.traj, s.freqs, g, **cfg).hhffbpa_adjoint(xv, g.points(idx))
    assert got.shape == (len(s.traj), len(s.freqs))
    rel = oracle.rel_l2(got.cpu().numpy().astype(np.complex128).ravel(), ref.ravel())
    assert rel < REL_TOL, (name, cfg, rel)


@pytest.mark.parametrize("name,cfg", CASES[:3])
def test_fast_adjoint_dot_product_with_forward(hh, name, cfg):
    """<x, A s> = <A^H x, s> with the GPU's own forward and adjoint on the full grid."""
    s = synth.CONFIGS[name]()
    rng = np.random.default_rng(22)
    e = torch.as_tensor((rng.normal(size=(len(s.traj), len(s.freqs)))
                         + 1j * rng.normal(size=(len(s.traj), len(s.freqs)))).astype(np.complex64), device="cuda")
    x = torch.as_tensor((rng.normal(size=s.grid.shape) + 1j * rng.normal(size=s.grid.shape)).astype(np.complex64),
                        device="cuda")
    plan = hh.Plan(s.traj, s.freqs, s.grid, **cfg)
    fwd = plan.form_image(e)
    adj = plan.adjoint(x)
    lhs = torch.vdot(x.reshape(-1).to(torch.complex128), fwd.reshape(-1).to(torch.complex128)).item()
    rhs = torch.vdot(adj.reshape(-1).to(torch.complex128), e.reshape(-1).to(torch.complex128)).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


def test_fast_adjoint_host_buffers(hh):
    s = synth.small()
    _, _, x = _image_values("small", s.grid, 23)
    plan = hh.Plan(s.traj, s.freqs, s.grid, leaf_size=16)
    dev = plan.adjoint(x).cpu()
    host = plan.adjoint(x.cpu().pin_memory(), out=torch.empty(dev.shape, dtype=torch.complex64).pin_memory())
    torch.cuda.synchronize()
    assert oracle.rel_l2(host.numpy().astype(np.complex128).ravel(), dev.numpy().astype(np.complex128).ravel()) < 1e-6


@pytest.mark.parametrize("name,cfg", CASES)
def test_fast_traj_gradient_matches_oracle(hh, name, cfg):
    s = synth.CONFIGS[name]()
    g = s.grid
    e = _echo(name, s)
    idx, gv, gimg = _image_values(name, g, 24)
    plan = hh.Plan(s.traj, s.freqs, g, **cfg)
    got = plan.traj_gradient(e, gimg).cpu().numpy()
    cnt = plan.counters()
    assert cnt["gate_miss"] == 0 and cnt["errors"] == 0, cnt
    ref = oracle.Plan(s.traj, s.freqs, g, **cfg).hhffbpa_traj_grad(e.cpu().numpy(), gv, g.points(idx))
    assert got.shape == (len(s.traj), 3)
    rel = oracle.rel_l2(got.ravel(), ref.ravel())
    assert rel < REL_TOL, (name, cfg, rel)


def _entropy(img):
    img = img.to(torch.complex128)  # the loss in FP64: differences of nearby losses stay resolved
    p = img.real ** 2 + img.imag ** 2
    q = p / p.sum()
    return -(q * torch.log(q + 1e-30)).sum()


@pytest.mark.parametrize("name,cfg", [("small", dict(leaf_size=16)), ("diff", dict(leaf_size=64))])
def test_fast_autofocus_loss_gradient_matches_finite_differences(hh, name, cfg):
    """Image entropy of the fast method's differentiable image of positions nominal + offsets,
    the plan held fixed: the backward pass (the adjoint traversal's kernels) against a central
    difference along a smooth random direction, both through the same fixed plan."""
    s = synth.CONFIGS[name]()
    n = len(s.traj)
    offs_true = synth.diff_offsets(n, seed=5, sigma_t=16.0 if n < 4096 else 128.0, rms=5e-4)
    e = synth.diff_echo(s, offs_true, device="cuda")
    plan = hh.Plan(s.traj, s.freqs, s.grid, **cfg)
    nominal = np.array(s.traj, np.float64)
    offsets = torch.zeros((n, 3), dtype=torch.float64, requires_grad=True)
    loss = _entropy(hh.hhffbpa_image_with_offsets(offsets, plan, e, nominal=nominal))
    loss.backward()
    grad = offsets.grad.numpy()
    assert np.isfinite(grad).all() and np.abs(grad).max() > 0
    v = synth.diff_offsets(n, seed=6, sigma_t=16.0 if n < 4096 else 128.0, rms=1.0)
    h = 2e-6
    with torch.no_grad():
        plan.update_positions(nominal + h * v)
        lp = _entropy(plan.form_image(e)).item()
        plan.update_positions(nominal - h * v)
        lm = _entropy(plan.form_image(e)).item()
    cnt = plan.counters()
    assert cnt["gate_miss"] == 0 and cnt["errors"] == 0, cnt
    fd = (lp - lm) / (2 * h)
    an = float((grad * v).sum())
    assert abs(fd - an) <= 2e-2 * abs(an), (fd, an)
