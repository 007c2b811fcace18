"""The maximum-intensity projection kernel (hh_mip) against the plain definition on the CPU:
max over one axis of |f|, on a ragged image (sizes not multiples of a warp or tile); and the
MUFU throughput probe that gives the MUFU rooflines their measured denominator."""
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


@pytest.mark.parametrize("op", ["rsqrt", "sin", "cos", "update_mix"])
def test_mufu_probe_counts_and_rate(hh, op):
    """The MUFU probe counts the results its grid computes and times them: 2048 threads per
    SM, eight chains each, three results per step for the update mix; the rate per SM and
    clock is within a factor of four of the 16 results/clk/SM of the sm_100 family."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rate, ops, ms = hh.mufu_throughput(op, 512)
    assert ops == sms * 2048 * 8 * 512 * (3 if op == "update_mix" else 1)
    assert ms > 0
    per_clk = rate / (sms * 2.07e9)
    assert 4.0 <= per_clk <= 64.0
