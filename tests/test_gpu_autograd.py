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


def _uneven_batch(seed, count, lo, hi, dtype, dev):
    """count problems, m, n, k log-uniform in [lo, hi], random trans; stored operands are
    leaves (their transposes are the column-major matrices passed to the GEMM)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    probs = []
    for _ in range(count):
        m, n, k = (int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for _ in range(3))
        ta, tb = str(rng.choice(["N", "T"])), str(rng.choice(["N", "T"]))
        ra, ca = (m, k) if ta == "N" else (k, m)
        rb, cb = (k, n) if tb == "N" else (n, k)
        At = stored(ra, ca, dtype, dev, gen).requires_grad_()
        Bt = stored(rb, cb, dtype, dev, gen).requires_grad_()
        probs.append((m, n, k, ta, tb, At, Bt))
    return probs


def test_grouped_gradcheck_fp64(dev):
    probs = _uneven_batch(41, 4, 3, 12, torch.float64, dev)
    ta = [p[3] for p in probs]
    tb = [p[4] for p in probs]
    leaves = [p[5] for p in probs] + [p[6] for p in probs]

    def f(*xs):
        As, Bs = xs[:len(probs)], xs[len(probs):]
        return tuple(ag.grouped_gemm([a.t() for a in As], [b.t() for b in Bs], ta, tb, -0.75,
                                     tile=0))
    assert torch.autograd.gradcheck(f, tuple(leaves), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_grouped_gradients_match_oracle(dev, dtype):
    """A batch of uneven problems (m, n, k log-uniform in [8, 128], random trans): forward
    and both gradients of every problem against the oracle."""
    probs = _uneven_batch(43, 96, 8, 128, dtype, dev)
    alpha = 1.25
    Cs = ag.grouped_gemm([p[5].t() for p in probs], [p[6].t() for p in probs],
                         [p[3] for p in probs], [p[4] for p in probs], alpha)
    gen = torch.Generator(device=dev)
    gen.manual_seed(44)
    dCs = [torch.rand(C.shape, generator=gen, dtype=dtype, device=dev) * 2 - 1 for C in Cs]
    torch.autograd.backward(Cs, dCs)
    u = inputs.unit_roundoff(np.float64 if dtype == torch.float64 else np.float32)
    for (m, n, k, ta, tb, At, Bt), C, dC in zip(probs, Cs, dCs):
        # forward
        A, lda = _np_colmajor(At.t())
        B, ldb = _np_colmajor(Bt.t())
        z = np.zeros(m * n)
        want = oracle.gemm_result(ta, tb, m, n, k, alpha, A, lda, B, ldb, 0.0, z, m)
        bound = oracle.abs_bound(ta, tb, m, n, k, alpha, A, lda, B, ldb, 0.0, z, m)
        got = C.detach().double().cpu().numpy()
        assert np.all(np.abs(got - inputs.as_matrix(want, m, n, m))
                      <= 2 * max(k, 2) * u * bound)   # abs_bound is already m x n
        # gradients
        ref = _ref_grads(At, Bt, dC, ta, tb, alpha, m, n, k)
        for name, grad in (("A", At.grad.t()), ("B", Bt.grad.t())):
            want, bound, rows, cols, inner = ref[name]
            got = grad.detach().double().cpu().numpy()
            want = inputs.as_matrix(want, rows, cols, rows)
            assert got.shape == want.shape == bound.shape
            assert np.all(np.abs(got - want) <= 2 * max(inner, 2) * u * bound), (
                name, m, n, k, ta, tb)
