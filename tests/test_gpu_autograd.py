"""Differentiable GEMM (paper_2302_08417_gb300.autograd): gradcheck by central finite
differences in FP64, and both gradients against the CPU oracle."""
import itertools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2302_08417_gb300 import autograd as ag  # noqa: E402
from paper_2302_08417_gb300 import inputs  # noqa: E402

FLIP = {"N": "T", "T": "N"}


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


def stored(rows, cols, dtype, dev, gen):
    """A column-major rows x cols leaf-derived view (the leaf is its cols x rows transpose)."""
    leaf = (torch.rand((cols, rows), generator=gen, dtype=dtype, device=dev) * 2 - 1)
    return leaf


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_gradcheck_fp64(dev, ta, tb):
    m, n, k = 64, 48, 32
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    ra, ca = (m, k) if ta == "N" else (k, m)
    rb, cb = (k, n) if tb == "N" else (n, k)
    At = stored(ra, ca, torch.float64, dev, gen).requires_grad_()
    Bt = stored(rb, cb, torch.float64, dev, gen).requires_grad_()
    for alpha in (1.0, -0.5):
        def f(At, Bt):
            return ag.gemm(At.t(), Bt.t(), ta, tb, alpha)
        assert torch.autograd.gradcheck(f, (At, Bt), eps=1e-6, atol=1e-8, rtol=1e-6)


def _np_colmajor(X):
    """Flat column-major buffer and leading dimension of a column-major torch view."""
    rows, cols = X.shape
    ld = rows
    buf = X.detach().t().contiguous().cpu().numpy().astype(np.float64).reshape(-1)
    return buf, ld


def _ref_grads(At, Bt, dC, ta, tb, alpha, m, n, k):
    """Oracle dA (stored shape) and dB, plus the bound terms, from the definitions
    d op(A) = alpha dC op(B)^T and d op(B) = alpha op(A)^T dC."""
    A, lda = _np_colmajor(At.t())
    B, ldb = _np_colmajor(Bt.t())
    G, ldg = _np_colmajor(dC)
    out = {}
    if ta == "N":   # dA (m x k) = alpha * dC * op(B)^T
        args = ("N", FLIP[tb], m, k, n, alpha, G, ldg, B, ldb)
        rows = m
    else:           # dA (k x m) = alpha * op(B) * dC^T
        args = (tb, "T", k, m, n, alpha, B, ldb, G, ldg)
        rows = k
    cols = k if ta == "N" else m
    z = np.zeros(rows * cols)
    out["A"] = (oracle.gemm_result(*args, 0.0, z, rows, nthreads=8),
                oracle.abs_bound(*args, 0.0, z, rows, nthreads=8), rows, cols, n)
    if tb == "N":   # dB (k x n) = alpha * op(A)^T * dC
        args = (FLIP[ta], "N", k, n, m, alpha, A, lda, G, ldg)
        rows = k
    else:           # dB (n x k) = alpha * dC^T * op(A)
        args = ("T", ta, n, k, m, alpha, G, ldg, A, lda)
        rows = n
    cols = n if tb == "N" else k
    z = np.zeros(rows * cols)
    out["B"] = (oracle.gemm_result(*args, 0.0, z, rows, nthreads=8),
                oracle.abs_bound(*args, 0.0, z, rows, nthreads=8), rows, cols, m)
    return out


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_gradients_match_oracle(dev, dtype, ta, tb):
    m, n, k = 260, 190, 130
    gen = torch.Generator(device=dev)
    gen.manual_seed(17)
    ra, ca = (m, k) if ta == "N" else (k, m)
    rb, cb = (k, n) if tb == "N" else (n, k)
    At = stored(ra, ca, dtype, dev, gen).requires_grad_()
    Bt = stored(rb, cb, dtype, dev, gen).requires_grad_()
    alpha = -1.5
    C = ag.gemm(At.t(), Bt.t(), ta, tb, alpha)
    dC = (torch.rand((m, n), generator=gen, dtype=dtype, device=dev) * 2 - 1)
    C.backward(dC)
    u = inputs.unit_roundoff(np.float64 if dtype == torch.float64 else np.float32)
    ref = _ref_grads(At, Bt, dC, ta, tb, alpha, m, n, k)
    for name, grad in (("A", At.grad.t()), ("B", Bt.grad.t())):
        want, bound, rows, cols, inner = ref[name]
        got = grad.detach().double().cpu().numpy()
        want = inputs.as_matrix(want, rows, cols, rows)
        bound = bound.reshape(rows, cols) if bound.ndim == 2 else bound
        tol = 2 * max(inner, 2) * u * bound
        assert got.shape == want.shape
        assert np.all(np.abs(got - want) <= tol), (name, np.abs(got - want).max())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("m,n,k", [(4096, 4096, 1024), (1024, 8192, 4096)])
def test_config_shapes_sampled(dev, dtype, m, n, k):
    """The differentiable-GEMM workload shapes, N/N: sampled gradient entries against the
    oracle's dot products (d op(A)[i,p] = alpha * sum_j dC[i,j] B[p,j], etc.)."""
    gen = torch.Generator(device=dev)
    gen.manual_seed(23)
    At = stored(m, k, dtype, dev, gen).requires_grad_()
    Bt = stored(k, n, dtype, dev, gen).requires_grad_()
    C = ag.gemm(At.t(), Bt.t(), "N", "N", 1.0)
    dC = torch.rand((m, n), generator=gen, dtype=dtype, device=dev) * 2 - 1
    C.backward(dC)
    torch.cuda.synchronize()
    u = inputs.unit_roundoff(np.float64 if dtype == torch.float64 else np.float32)
    A, lda = _np_colmajor(At.t())
    B, ldb = _np_colmajor(Bt.t())
    G, ldg = _np_colmajor(dC)
    rng = np.random.Generator(np.random.PCG64(3))
    # dA = dC * B^T  (m x k), inner dimension n
    ii, jj = inputs.sample_indices(rng, m, k, 2048)
    want = oracle.entries("N", "T", m, k, n, 1.0, G, ldg, B, ldb, 0.0, None, m, ii, jj,
                          nthreads=8)
    bnd = oracle.entries("N", "T", m, k, n, 1.0, G, ldg, B, ldb, 0.0, None, m, ii, jj,
                         absval=True, nthreads=8)
    got = At.grad.t().detach().double().cpu().numpy()[ii, jj]
    assert np.all(np.abs(got - want) <= 2 * n * u * bnd)
    # dB = A^T * dC  (k x n), inner dimension m
    ii, jj = inputs.sample_indices(rng, k, n, 2048)
    want = oracle.entries("T", "N", k, n, m, 1.0, A, lda, G, ldg, 0.0, None, k, ii, jj,
                          nthreads=8)
    bnd = oracle.entries("T", "N", k, n, m, 1.0, A, lda, G, ldg, 0.0, None, k, ii, jj,
                         absval=True, nthreads=8)
    got = Bt.grad.t().detach().double().cpu().numpy()[ii, jj]
    assert np.all(np.abs(got - want) <= 2 * m * u * bnd)
