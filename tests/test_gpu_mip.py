"""The maximum-intensity projection kernel (hh_mip) against the plain definition on the CPU:
max over one axis of |f|, on a ragged image (sizes not multiples of a warp or tile)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_23568_gb300 as m

    m.lib()
    return m


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mip_matches_definition(hh, axis):
    rng = np.random.default_rng(7)
    f = (rng.normal(size=(7, 13, 45)) + 1j * rng.normal(size=(7, 13, 45))).astype(np.complex64)
    got = hh.mip(torch.as_tensor(f, device="cuda"), axis=axis).cpu().numpy()
    ref = np.abs(f.astype(np.complex128)).max(axis=axis)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=2e-7, atol=0)
