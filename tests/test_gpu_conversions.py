"""The solve kernels convert between FP32 and FP64 with integer instructions;
check them bit for bit against the hardware conversions (round to nearest,
ties to even) on adversarial values."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _values():
    rng = np.random.default_rng(7)
    n = 1 << 20
    # random signs, mantissas and exponents spanning beyond the FP32 range
    mant = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    expo = rng.integers(1023 - 160, 1023 + 140, size=n).astype(np.uint64)
    sign = rng.integers(0, 2, size=n).astype(np.uint64)
    bits = [(sign << np.uint64(63)) | (expo << np.uint64(52)) | mant]
    # exact ties and their neighbours: low 29 mantissa bits = 2^28 (+-1), odd and even kept bits
    kept = rng.integers(0, 1 << 23, size=4096, dtype=np.uint64) << np.uint64(29)
    e2 = rng.integers(1023 - 126, 1023 + 128, size=4096).astype(np.uint64) << np.uint64(52)
    for low in (0x10000000, 0x0FFFFFFF, 0x10000001, 0x1FFFFFFF, 0):
        bits.append(e2 | kept | np.uint64(low))
        bits.append(e2 | kept | np.uint64(1 << 29) | np.uint64(low))
    x = np.concatenate([b.view(np.float64) for b in bits])
    f32 = np.finfo(np.float32)
    special = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, float(f32.max), -float(f32.max),
               float(f32.max) * (1 + 2.0 ** -25), float(f32.max) * (1 + 2.0 ** -24), float(f32.tiny),
               float(f32.tiny) * (1 - 2.0 ** -30), float(f32.tiny) * 0.5, 2.0 ** -149, 2.0 ** -150, 1e-300,
               1e300, np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0)]
    return np.concatenate([x, np.array(special, dtype=np.float64)])


def test_integer_pipe_conversions_match_hardware():
    from paper_2606_04864_gb300._lib import check, lib
    x = torch.as_tensor(_values(), device="cuda")
    nb, wb = C.c_int64(-1), C.c_int64(-1)
    check(lib().ams_check_conversions(C.c_void_p(x.data_ptr()), x.numel(), C.byref(nb), C.byref(wb)),
          "ams_check_conversions")
    assert nb.value == 0 and wb.value == 0, (nb.value, wb.value)
