"""The tcgen05 / TMA tensor-core GEMM behind the mixed-precision modes,
through the C ABI, against an FP64 product of the same rounded operands."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build
    build.build()


def round_tf32(a):
    """Round to nearest, ties away from zero, keeping 10 mantissa bits."""
    b = a.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32)


def round_bf16(a):
    """Round to nearest even, keeping 7 mantissa bits."""
    b = a.astype(np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("M,N,K,splits", [(128, 64, 64, 1), (300, 48, 513, 1), (77, 16, 32, 1),
                                          (1000, 64, 2000, 4), (256, 256, 128, 1),
                                          (129, 200, 700, 3), (640, 96, 4096, 7)])
def test_tensor_core_gemm(kind, M, N, K, splits):
    from paper_2111_10105_gb300.codec import selftest_gemm
    r = np.random.default_rng(M * 7 + N + K + kind)
    A = r.normal(size=(M, K)).astype(np.float32)
    B = r.normal(size=(N, K)).astype(np.float32)
    rnd = round_tf32 if kind == 0 else round_bf16
    Ar, Br = rnd(A).astype(np.float64), rnd(B).astype(np.float64)
    want = Ar @ Br.T
    got = selftest_gemm(kind, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                        splits=splits).cpu().numpy()
    bound = 2.0 * K * 2.0 ** -24 * (np.abs(Ar) @ np.abs(Br).T) + 1e-30
    err = np.abs(got - want)
    assert np.all(err <= bound), (err / bound).max()
