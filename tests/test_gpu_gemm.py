"""Batched complex GEMM of the band step (FP64 CUDA cores and the tensor-core digit-plane
method) against numpy complex128 products (GPU only)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4247_gb300.nao import Context
    c = Context(0)
    yield c
    c.close()


def _op(X, t):
    return X if t == 0 else (np.swapaxes(X, 1, 2) if t == 1 else np.conj(np.swapaxes(X, 1, 2)))


def _run(ctx, A, B, tA, tB, method, alpha=1.0, beta=0.0, C0=None):
    from paper_1402_4247_gb300.nao import NAO_GEMM_TC  # noqa: F401
    At = torch.from_numpy(A).to(DEV)
    Bt = torch.from_numpy(B).to(DEV)
    Ct = None if C0 is None else torch.from_numpy(C0.copy()).to(DEV)
    out = ctx.nao_zgemm(At, Bt, C=Ct, alpha=alpha, beta=beta, transA=tA, transB=tB, method=method)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _bound(A, B, tA, tB):
    """FP64-level elementwise bound: 16 K 2^-53 (|op(A)| |op(B)|)_ij plus the same factor times
    the row-maximum / column-maximum product (the tensor-core method scales rows and columns)."""
    a, b = np.abs(_op(A, tA)), np.abs(_op(B, tB))
    K = a.shape[2]
    amax = a.max(axis=2, keepdims=True)
    bmax = b.max(axis=1, keepdims=True)
    return 16 * K * 2.0 ** -53 * (np.einsum("pik,pkj->pij", a, b) + amax * bmax)


@pytest.mark.parametrize("method", [0, 1], ids=["fp64", "tc"])
@pytest.mark.parametrize("nprob,M,N,K,tA,tB", [
    (1, 1, 1, 1, 0, 0), (2, 7, 5, 3, 0, 0), (3, 128, 40, 16, 0, 0), (2, 130, 41, 17, 2, 0),
    (2, 33, 129, 95, 0, 2), (1, 257, 81, 300, 1, 1), (1, 568, 568, 568, 2, 0), (2, 64, 48, 896, 0, 0)])
def test_zgemm_random(ctx, method, nprob, M, N, K, tA, tB):
    rng = np.random.Generator(np.random.PCG64(M * 1000 + N * 10 + K))
    shA = (nprob, K, M) if tA else (nprob, M, K)
    shB = (nprob, N, K) if tB else (nprob, K, N)
    A = rng.normal(size=shA) + 1j * rng.normal(size=shA)
    B = rng.normal(size=shB) + 1j * rng.normal(size=shB)
    A[:, :1] *= 1e-9  # rows / columns of very different scale
    ref = np.einsum("pik,pkj->pij", _op(A, tA), _op(B, tB))
    got = _run(ctx, A, B, tA, tB, method)
    bnd = _bound(A, B, tA, tB)
    assert np.all(np.abs(got - ref) <= bnd), np.max(np.abs(got - ref) / bnd)


@pytest.mark.parametrize("method", [0, 1], ids=["fp64", "tc"])
def test_zgemm_alpha_beta(ctx, method):
    rng = np.random.Generator(np.random.PCG64(77))
    A = rng.normal(size=(2, 50, 60)) + 1j * rng.normal(size=(2, 50, 60))
    B = rng.normal(size=(2, 60, 70)) + 1j * rng.normal(size=(2, 60, 70))
    C0 = rng.normal(size=(2, 50, 70)) + 1j * rng.normal(size=(2, 50, 70))
    got = _run(ctx, A, B, 0, 0, method, alpha=-1.0, beta=1.0, C0=C0)
    ref = C0 - A @ B
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_tc_exact_on_integers(ctx):
    """Small-integer operands have exact products: both methods must return them exactly."""
    rng = np.random.Generator(np.random.PCG64(5))
    A = (rng.integers(-50, 50, size=(2, 100, 200)) + 1j * rng.integers(-50, 50, size=(2, 100, 200))).astype(complex)
    B = (rng.integers(-50, 50, size=(2, 200, 90)) + 1j * rng.integers(-50, 50, size=(2, 200, 90))).astype(complex)
    ref = A @ B
    for method in (0, 1):
        assert np.array_equal(_run(ctx, A, B, 0, 0, method), ref)


@pytest.mark.parametrize("K", [897, 2000])
def test_tc_long_k_in_chunks(ctx, K):
    """Contractions past one exact chunk (896) run as several, summed in FP64: as accurate as
    the FP64 product against extended precision, and within the FP64 error bound."""
    rng = np.random.Generator(np.random.PCG64(K))
    A = rng.normal(size=(2, 70, K)) + 1j * rng.normal(size=(2, 70, K))
    B = rng.normal(size=(2, K, 50)) + 1j * rng.normal(size=(2, K, 50))
    A[:, :, :5] *= 1e-7
    ref = np.matmul(A.astype(np.clongdouble), B.astype(np.clongdouble))
    got = _run(ctx, A, B, 0, 0, 1)
    e_fp64 = np.linalg.norm((_run(ctx, A, B, 0, 0, 0) - ref).astype(np.complex128))
    e_tc = np.linalg.norm((got - ref).astype(np.complex128))
    assert e_tc <= 2.0 * e_fp64 + 1e-300, (e_tc, e_fp64)
    assert np.all(np.abs(got - ref.astype(np.complex128)) <= _bound(A, B, 0, 0))


@pytest.mark.parametrize("M,N,K,tA", [(96, 64, 568, 2), (130, 50, 890, 0), (64, 130, 300, 1)])
def test_tc_error_not_above_fp64_error(ctx, M, N, K, tA):
    """Against an extended-precision reference, the tensor-core product must be at least
    about as accurate as the FP64 product (Frobenius error at most 2x)."""
    rng = np.random.Generator(np.random.PCG64(9000 + M + K))
    shA = (1, K, M) if tA else (1, M, K)
    A = rng.normal(size=shA) + 1j * rng.normal(size=shA)
    B = rng.normal(size=(1, K, N)) + 1j * rng.normal(size=(1, K, N))
    A[0, :, :3] *= 1e-6  # entries far below their row maximum
    opA = _op(A, tA)
    ref = np.matmul(opA.astype(np.clongdouble), B.astype(np.clongdouble))
    e_fp64 = np.linalg.norm((_run(ctx, A, B, tA, 0, 0) - ref).astype(np.complex128))
    e_tc = np.linalg.norm((_run(ctx, A, B, tA, 0, 1) - ref).astype(np.complex128))
    assert e_tc <= 2.0 * e_fp64 + 1e-300, (e_tc, e_fp64)


def test_tc_gram_of_reflectors_as_accurate_as_fp64(ctx):
    """V^H V for unit lower-trapezoidal reflector blocks (the compact-WY Gram matrix): row and
    column maxima are 1 while most entries are small, the hardest case for row scaling."""
    rng = np.random.Generator(np.random.PCG64(4242))
    n, nb = 567, 128
    V = (rng.normal(size=(2, n, nb)) + 1j * rng.normal(size=(2, n, nb))) * 0.05
    for c in range(nb):
        V[:, :c, c] = 0.0
        V[:, c, c] = 1.0
    ref = np.matmul(np.conj(np.swapaxes(V, 1, 2)).astype(np.clongdouble), V.astype(np.clongdouble))
    e_fp64 = np.linalg.norm((_run(ctx, V, V, 2, 0, 0) - ref).astype(np.complex128))
    e_tc = np.linalg.norm((_run(ctx, V, V, 2, 0, 1) - ref).astype(np.complex128))
    assert e_tc <= 2.0 * e_fp64 + 1e-300, (e_tc, e_fp64)
