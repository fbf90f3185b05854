"""CPU pins of the E4M3 emulation that the precision-8 parity test compares against.

The rounding helper is checked against PyTorch's own float8_e4m3fn conversion (an
independent implementation) over every representable magnitude and the midpoints
between them, and the scale helper against its definition."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests.test_gpu_stages import _e4m3, _pow2_scale  # noqa: E402


def test_e4m3_rounding_matches_torch():
    codes = torch.arange(0, 127, dtype=torch.uint8)  # 0x7f is NaN
    grid = codes.view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert grid.max() == 448.0 and grid[1] == 2.0**-9
    # FP32 inputs, as in the kernel (PyTorch converts through FP32, so FP64 values one
    # FP64 ulp off a midpoint would round twice)
    mids = ((grid[:-1] + grid[1:]) / 2).astype(np.float32)
    rng = np.random.default_rng(0)
    v = np.concatenate([grid.astype(np.float32), mids, np.nextafter(mids, np.float32(0)),
                        np.nextafter(mids, np.float32(1e9)),
                        rng.uniform(0, 448, 100_000).astype(np.float32),
                        rng.uniform(0, 2.0**-5, 10_000).astype(np.float32)]).astype(np.float64)
    v = np.concatenate([v, -v])
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(_e4m3(v), ref)
    # saturation above the largest finite value
    assert _e4m3(np.array([470.0, -1e9]))[0] == 448.0
    assert _e4m3(np.array([470.0, -1e9]))[1] == -448.0


@pytest.mark.parametrize("amax", [1e-14, 0.013, 0.5, 1.0, 7.0, 224.0, 448.0, 449.0, 3e5])
def test_pow2_scale(amax):
    s = _pow2_scale(amax)
    assert s == 2.0 ** np.round(np.log2(s))
    assert 224.0 < s * amax <= 448.0
    assert _pow2_scale(0.0) == 1.0
    assert _pow2_scale(1e-30) == 2.0**60  # exponent clamped
