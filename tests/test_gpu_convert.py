"""The precision form's binary64 <-> binary32 conversions (integer-pipe forms
of the IEEE-754 layouts) against the hardware conversions: bit-exact over the
binary32 normal range, including ties, carries into the exponent, zeros,
infinities and NaNs; the documented flush of values below the normal range."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _cases(rng, n=1 << 20):
    mags = 10.0 ** rng.uniform(-37.5, 38.2, n)
    x = np.where(rng.random(n) < 0.5, -mags, mags)
    # exact ties between two binary32 neighbours and values next to them
    f = rng.standard_normal(4096).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + up.astype(np.float64)) / 2.0
    special = np.concatenate([mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf),
                              [0.0, -0.0, np.inf, -np.inf, 1.0, -1.0, 3.4028234663852886e38,
                               3.4028235677973366e38, 1.1754943508222875e-38, 2.0 ** -126 * (1 - 2.0 ** -25),
                               1.9999999403953552, 16777217.0, 0.1, 1e-30]])
    return np.concatenate([x, special])


def test_narrow_matches_hardware_rounding():
    import torch
    import paper_2301_02387_gb300 as pkg
    x = torch.from_numpy(_cases(np.random.default_rng(0))).cuda()
    y = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    pkg.convert(x, y)
    ref = x.float()
    normal = (x.abs() >= 2.0 ** -126) | (x == 0)
    assert torch.equal(y[normal].view(torch.int32), ref[normal].view(torch.int32))
    tiny = ~normal & torch.isfinite(x)
    assert torch.all(y[tiny] == 0) and torch.equal(torch.signbit(y[tiny]), torch.signbit(x[tiny]))
    nan = torch.tensor([float("nan"), -float("nan")], dtype=torch.float64, device="cuda")
    yn = torch.empty(2, dtype=torch.float32, device="cuda")
    pkg.convert(nan, yn)
    assert torch.all(torch.isnan(yn))


def test_widen_is_exact():
    import torch
    import paper_2301_02387_gb300 as pkg
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2 ** 32, 1 << 20, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    f = f[np.isfinite(f)]
    x = torch.from_numpy(np.concatenate([f, np.array([0.0, -0.0, np.inf, -np.inf], np.float32)])).cuda()
    y = torch.empty(x.shape, dtype=torch.float64, device="cuda")
    pkg.convert(x, y)
    ref = x.double()
    normal = (x.abs() >= 2.0 ** -126) | (x == 0) | torch.isinf(x)
    assert torch.equal(y[normal].view(torch.int64), ref[normal].view(torch.int64))
    assert torch.all(y[~normal] == 0)
