"""The integer -> FP64 conversions of the fixed-point reverse pass (written
from the IEEE 754 binary64 encoding, round to nearest, ties to even) against
exactly rounded references: Python's int -> float conversion (correctly
rounded, ties to even) for 128-bit values, and CUDA's own int64 -> float64
conversion for 64-bit ones.  Bit for bit, including ties, carries out of the
significand, the extreme magnitudes and zero."""
import numpy as np
import pytest
import torch

from paper_2309_02825_gb300 import lb

pytestmark = pytest.mark.gpu


def _values(rng):
    vals = [0, 1, -1, 2 ** 53 - 1, 2 ** 53, 2 ** 53 + 1, 2 ** 53 + 3, -(2 ** 53 + 1), 2 ** 63 - 1, -(2 ** 63),
            2 ** 64 - 1, 2 ** 64, 2 ** 64 + 1, 2 ** 127 - 1, -(2 ** 127), -(2 ** 127) + 1, (2 ** 53 - 1) * 2 ** 70,
            (2 ** 54 - 1) * 2 ** 60, -(2 ** 54 - 1) * 2 ** 12]
    for bits in range(1, 128):
        for _ in range(24):
            v = int(rng.integers(0, 2 ** 62)) << 66 | int(rng.integers(0, 2 ** 62)) << 4 | int(rng.integers(0, 16))
            v &= (1 << bits) - 1
            v |= 1 << (bits - 1)
            vals.append(-v if rng.random() < 0.5 else v)
        if bits > 54:  # exact ties: 53 significant bits and a lone half below them
            for _ in range(8):
                m = int(rng.integers(2 ** 52, 2 ** 53))
                k = bits - 53
                v = (m << k) | (1 << (k - 1))
                vals.append(-v if rng.random() < 0.5 else v)
    return [v for v in vals if -(2 ** 127) <= v < 2 ** 127]


def test_int128_and_int64_conversions_are_correctly_rounded():
    rng = np.random.default_rng(12)
    vals = _values(rng)
    hi = [v >> 64 for v in vals]
    lo = [v & (2 ** 64 - 1) for v in vals]
    lo_s = [x - 2 ** 64 if x >= 2 ** 63 else x for x in lo]
    hi_t = torch.tensor(hi, dtype=torch.int64).cuda()
    lo_t = torch.tensor(lo_s, dtype=torch.int64).cuda()
    o128, o64 = lb.lb_selftest_int_to_f64(hi_t, lo_t)
    torch.cuda.synchronize()
    want128 = np.array([float(v) for v in vals])
    want64 = np.array([float(x) for x in lo_s])
    got128, got64 = o128.cpu().numpy(), o64.cpu().numpy()
    bad = np.nonzero(got128.view(np.int64) != want128.view(np.int64))[0]
    assert bad.size == 0, [(vals[i], got128[i], want128[i]) for i in bad[:5]]
    assert np.array_equal(got64.view(np.int64), want64.view(np.int64))
    # CUDA's own conversion of the same int64 values
    assert torch.equal(o64.view(torch.int64), lo_t.to(torch.float64).view(torch.int64))


def test_selftest_argument_errors():
    lib = lb.load()
    assert lib.lb_selftest_int_to_f64(None, None, -1, None, None, None) == lb.LB_EINVAL
    assert lib.lb_selftest_int_to_f64(None, None, 4, None, None, None) == lb.LB_EINVAL
    assert lib.lb_selftest_int_to_f64(None, None, 0, None, None, None) == lb.LB_OK
