"""Learned displacement model on the tensor cores vs the FP64 CPU oracle.

The tensor-core tile (tcgen05 MMAs on BF16 operands, FP32 accumulation in
tensor memory) must equal the exact product of the same BF16 values up to
FP32 accumulation rounding.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_2309_13824_gb300 as g

    g.build()


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (256, 64, 48), (128, 256, 256), (384, 48, 64), (128, 80, 32)])
def test_tensor_core_tile(M, N, K):
    import paper_2309_13824_gb300 as g

    rng = np.random.default_rng(M + N + K)
    A = g.bf16_bits(rng.standard_normal((M, K)))
    B = g.bf16_bits(rng.standard_normal((N, K)))
    D = g.mesh_tc_gemm_bf16(A, B)
    a = g.bf16_to_float(A).astype(np.float64)
    b = g.bf16_to_float(B).astype(np.float64)
    exact = a @ b.T
    scale = np.abs(a) @ np.abs(b).T
    assert np.all(np.abs(D - exact) <= 2e-6 * scale + 1e-30), np.max(np.abs(D - exact) / scale)
