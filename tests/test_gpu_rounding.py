"""The library's FP64 -> FP32 rounding on the integer pipe (used for the FP32
copies of the FP32-mixed contexts) against the hardware conversion, bit for
bit: random values over the whole normal FP32 range, exact halfway cases of
both parities, the overflow and underflow boundaries, and the special
values that take the hardware path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _bits(hi, lo):
    return ((np.asarray(hi, dtype=np.uint64) << np.uint64(32)) | np.asarray(lo, dtype=np.uint64)).view(np.float64)


def test_round_f32_matches_hardware():
    from paper_2209_15095_gb300 import build

    build.build()
    from paper_2209_15095_gb300 import etd

    rng = np.random.default_rng(41)
    n = 1 << 20
    # random signs, FP64 exponents from below the FP32 subnormals to above FP32 overflow, random mantissas
    sign = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(31)
    ex = rng.integers(860, 1160, n, dtype=np.uint64)
    mhi = rng.integers(0, 1 << 20, n, dtype=np.uint64)
    lo = rng.integers(0, 1 << 32, n, dtype=np.uint64)
    vals = [_bits(sign | (ex << np.uint64(20)) | mhi, lo)]
    # exact halfway cases (dropped bits 1000...0) with odd and even kept mantissas
    ex2 = rng.integers(897, 1151, 4096, dtype=np.uint64)
    mhi2 = rng.integers(0, 1 << 20, 4096, dtype=np.uint64)
    keep_lo = rng.integers(0, 8, 4096, dtype=np.uint64) << np.uint64(29)
    vals.append(_bits((ex2 << np.uint64(20)) | mhi2, keep_lo | np.uint64(0x10000000)))
    vals.append(_bits((ex2 << np.uint64(20)) | mhi2, keep_lo | np.uint64(0x0FFFFFFF)))
    vals.append(_bits((ex2 << np.uint64(20)) | mhi2, keep_lo | np.uint64(0x10000001)))
    f32max = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    ulp_max = 2.0 ** 104
    edge = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, f32max, -f32max, f32max + 0.5 * ulp_max,
            f32max + 0.49 * ulp_max, f32max + 0.51 * ulp_max, np.nextafter(f32max + 0.5 * ulp_max, 0.0), 1e300,
            -1e300, tiny, -tiny, np.nextafter(tiny, 0.0), tiny * (1 - 2.0 ** -25), tiny * (1 - 2.0 ** -24),
            tiny * 0.5, 1e-300, 5e-324, 2.0 ** 127, 2.0 ** 128, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24,
            1.0 - 2.0 ** -25, 3.0 * 2.0 ** -150]
    vals.append(np.array(edge, dtype=np.float64))
    x = np.concatenate(vals)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    lib, hw = etd.selfcheck_round_f32(xd)
    a = lib.cpu().numpy().view(np.uint32)
    b = hw.cpu().numpy().view(np.uint32)
    bad = np.flatnonzero(a != b)
    assert bad.size == 0, [(float(x[i]).hex(), hex(int(a[i])), hex(int(b[i]))) for i in bad[:8]]
    # and the hardware conversion is numpy's rounding
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32).view(np.uint32)
    fin = np.isfinite(x) | np.isinf(x)
    assert np.all(b[fin] == ref[fin])
