"""The quotients cx / w and cy / w of quad setup come from the correctly rounded 1/w by
Markstein's correction instead of a full IEEE division (Sec. 2, "Stage 1: quad setup"; the
snapped coordinates must equal those of the plain fp32 definition bit for bit). This checks
the device routine against CUDA's IEEE division on every mantissa of w in [1, 2) times
thousands of numerators over the exponent range the fast path accepts, at several scales
of w, and on the edges of that range and special values (which take the IEEE division)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2405_13364_gb300 import _build
    out = str(tmp_path_factory.mktemp("divcheck") / "division_check.so")
    cmd = [_build._nvcc(), *_build.ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
           "-I", _build.CSRC, "-I", _build.INCLUDE, "-shared", "-o", out, os.path.join(HERE, "cuda", "division_check.cu")]
    subprocess.run(cmd, check=True)
    lib = ctypes.CDLL(out)
    lib.lr_test_div_check.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return lib


def _run(lib, a: np.ndarray, w_exp: int):
    at = torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    assert lib.lr_test_div_check(at.data_ptr(), at.numel(), w_exp, res.data_ptr(), res.data_ptr() + 8) == 0
    torch.cuda.synchronize()
    first = int(res[1]) & 0xFFFFFFFFFFFFFFFF
    return int(res[0]), first


def _numerators(rng, n, e_lo, e_hi):
    mant = rng.integers(0, 1 << 23, n, dtype=np.uint32)
    expo = rng.integers(127 + e_lo, 127 + e_hi + 1, n, dtype=np.uint32)
    sign = rng.integers(0, 2, n, dtype=np.uint32) << np.uint32(31)
    return (sign | (expo << np.uint32(23)) | mant).view(np.float32)


def test_all_mantissas_of_w(checker):
    rng = np.random.default_rng(7)
    a = _numerators(rng, 4096, -60, 60)
    a[:6] = [1.0, -1.0, 3.0, 1.9999999, 0.1, 7.0]
    bad, first = _run(checker, a, 0)
    assert bad == 0, f"{bad} mismatches, first (a bits << 32 | w bits) = {first:#x}"


@pytest.mark.parametrize("w_exp", [-60, -20, 7, 30, 59])
def test_scaled_w(checker, w_exp):
    rng = np.random.default_rng(100 + w_exp)
    # numerators whose quotient stays inside the fast path's range and just outside it
    a = _numerators(rng, 512, max(-90, w_exp - 62), min(60, w_exp + 62))
    bad, first = _run(checker, a, w_exp)
    assert bad == 0, f"{bad} mismatches, first = {first:#x}"


def test_range_edges_and_specials(checker):
    f = np.float32
    edges = [0.0, -0.0, 2.0 ** 60, -(2.0 ** 60), np.nextafter(f(2.0 ** 60), f(np.inf)), 2.0 ** -90,
             np.nextafter(f(2.0 ** -90), f(0)), 2.0 ** -100, 1e-38, 1e-45, 3.0e38, np.inf, -np.inf, np.nan,
             2.0 ** -60, 1.5 * 2.0 ** -60, np.nextafter(f(2.0 ** -60), f(0))]
    a = np.array(edges, np.float32)
    for w_exp in (-61, -60, 0, 59, 60, 61):
        bad, first = _run(checker, a, w_exp)
        assert bad == 0, f"w_exp {w_exp}: {bad} mismatches, first = {first:#x}"
