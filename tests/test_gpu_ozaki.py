"""The tensor-core FP64 product (spk_dense_gemm, engine "tensor": tcgen05 MMAs
on BF16 slices of the FP64 operands, Ozaki et al. 2012) against NumPy's FP64
product and the library's FP64 CUDA-core GEMM.  The splitting keeps 57 bits
of every row and column (relative to its largest entry) and every level sum
is exact in FP32, so the result carries FP64 GEMM accuracy: the bound
checked is |C - C_ref| <= 4 K u max|A row| max|B col| entry by entry."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_16019_gb300 import build, spk
    build.build()
    return spk.load()


def spk():
    from paper_2311_16019_gb300 import spk as s
    return s


U = 2.0 ** -53


def _check(A, B, ta, tb, alpha=1.0, beta=0.0, Cin=None):
    opA = A if ta == "N" else A.T
    opB = B if tb == "N" else B.T
    ref = alpha * (opA @ opB) + (beta * Cin if Cin is not None else 0.0)
    got = spk().dense_gemm(A, B, ta=ta, tb=tb, alpha=alpha, beta=beta, Cin=Cin, engine="tensor")
    fp = spk().dense_gemm(A, B, ta=ta, tb=tb, alpha=alpha, beta=beta, Cin=Cin, engine="fp64")
    K = opA.shape[1]
    scale = np.abs(alpha) * np.outer(np.abs(opA).max(axis=1), np.abs(opB).max(axis=0)) * K
    if Cin is not None:
        scale = scale + np.abs(beta * Cin)
    bound = 4 * U * scale + 1e-300
    err = np.abs(got - ref) / bound
    err_fp = np.abs(fp - ref) / bound
    print(f"{opA.shape} x {opB.shape} {ta}{tb}: max err / bound tensor {err.max():.3f}, "
          f"fp64 gemm {err_fp.max():.3f}, relative Frobenius "
          f"{np.linalg.norm(got - ref) / np.linalg.norm(ref):.2e}")
    assert err.max() <= 1.0


@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (300, 257, 130), (640, 700, 128),
                                   (1000, 300, 1000), (129, 65, 33)])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_tensor_gemm_random(M, N, K, ta, tb):
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    A = rng.standard_normal((M, K) if ta == "N" else (K, M))
    B = rng.standard_normal((K, N) if tb == "N" else (N, K))
    _check(A, B, ta, tb)


def test_tensor_gemm_dynamic_range_alpha_beta():
    """Rows and columns spanning 60 orders of magnitude (each scaled by its
    own exponent), entries within a row spanning 1e-12..1, and the update
    form alpha op(A) op(B) + beta C of the Gauss-Jordan trailing updates."""
    rng = np.random.default_rng(5)
    M, N, K = 384, 320, 200
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-30, 30, (M, 1))
    A *= 10.0 ** rng.uniform(-12, 0, (1, K))
    B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-30, 30, (1, N))
    Cin = rng.standard_normal((M, N)) * np.abs(A).max(axis=1)[:, None]
    _check(A, B, "N", "N", alpha=-1.5, beta=1.0, Cin=Cin)


def test_tensor_gemm_integers_exact():
    """Integer operands of 20 bits: every product and sum is exact in FP64,
    and the splitting reproduces them exactly."""
    rng = np.random.default_rng(9)
    A = rng.integers(-2 ** 20, 2 ** 20, (512, 256)).astype(np.float64)
    B = rng.integers(-2 ** 10, 2 ** 10, (256, 384)).astype(np.float64)
    got = spk().dense_gemm(A, B, engine="tensor")
    assert np.array_equal(got, A @ B)
