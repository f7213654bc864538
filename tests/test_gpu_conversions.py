"""The library's integer-pipe IEEE 754 conversions (binary64 to binary32,
round to nearest even; binary32 to binary64, exact) give the hardware
conversions' bit patterns: on random bit patterns over every exponent, on
exact ties between neighbouring floats and one binary64 ulp either side of
them, at the ends of the normal binary32 range, and on zeros, subnormals,
infinities and NaNs."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("conv") / "libconvcheck.so")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "--expt-relaxed-constexpr", "-shared", "-o", out, os.path.join(HERE, "conversions_check.cu")]
    subprocess.run(cmd, check=True, capture_output=True)
    return ctypes.CDLL(out)


def _d2f_inputs():
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2**64, size=400000, dtype=np.uint64)
    parts = [bits.view(np.float64)]
    # exponents around the binary32 range, random fractions and signs
    e = rng.integers(1023 - 160, 1023 + 140, size=400000, dtype=np.uint64)
    f = rng.integers(0, 2**52, size=400000, dtype=np.uint64)
    s = rng.integers(0, 2, size=400000, dtype=np.uint64)
    parts.append(((s << np.uint64(63)) | (e << np.uint64(52)) | f).view(np.float64))
    # exact ties between neighbouring floats, and one binary64 ulp either side
    fl = (rng.integers(1, 0x7F7FFFFF, size=200000, dtype=np.uint32)).view(np.float32)
    lo = fl.astype(np.float64)
    hi = np.nextafter(fl, np.float32(np.inf)).astype(np.float64)
    mid = (lo + hi) / 2
    parts += [mid, -mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf)]
    fmax = float(np.finfo(np.float32).max)
    ulp = fmax - float(np.nextafter(np.float32(fmax), np.float32(0)))   # 2^104, the spacing at the top binade
    tiny = float(np.finfo(np.float32).tiny)
    edge = [0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, fmax + ulp / 2, np.nextafter(fmax + ulp / 2, 0.0),
            np.nextafter(fmax + ulp / 2, np.inf), tiny, -tiny, np.nextafter(tiny, 0.0), np.nextafter(tiny, 1.0),
            tiny / 2, 1e-45, 5e-324, 1.0, -1.0, 2.0 ** -126, 2.0 ** 127, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24]
    parts.append(np.array(edge, dtype=np.float64))
    return np.ascontiguousarray(np.concatenate(parts))


def test_f64_to_f32_matches_hardware(lib):
    x = _d2f_inputs()
    n = x.size
    got = np.empty(n, np.uint32)
    ref = np.empty(n, np.uint32)
    st = lib.check_d2f(x.ctypes.data_as(ctypes.c_void_p), got.ctypes.data_as(ctypes.c_void_p),
                       ref.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(n))
    assert st == 0
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, [(x[i], hex(got[i]), hex(ref[i])) for i in bad[:5]]
    # and the hardware is IEEE round-to-nearest-even, as numpy's cast
    fin = np.isfinite(x)
    with np.errstate(over="ignore"):
        assert np.array_equal(ref[fin], x[fin].astype(np.float32).view(np.uint32))


def test_f32_to_f64_matches_hardware(lib):
    rng = np.random.default_rng(12)
    bits = np.concatenate([rng.integers(0, 2**32, size=400000, dtype=np.uint32),
                           np.array([0, 0x80000000, 1, 0x807FFFFF, 0x00800000, 0x7F7FFFFF, 0x7F800000,
                                     0xFF800000, 0x7FC00000, 0x7FA00001], dtype=np.uint32)])
    x = np.ascontiguousarray(bits.view(np.float32))
    n = x.size
    got = np.empty(n, np.uint64)
    ref = np.empty(n, np.uint64)
    st = lib.check_f2d(x.ctypes.data_as(ctypes.c_void_p), got.ctypes.data_as(ctypes.c_void_p),
                       ref.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(n))
    assert st == 0
    assert np.array_equal(got, ref)
