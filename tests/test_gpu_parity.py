"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bounds: |C - C_oracle| <= 2*max(k,2)*u*(|alpha||op(A)||op(B)| + |beta||C0|) elementwise with
u = 2^-53 (FP64) or 2^-24 (FP32); bit-exact on small-integer inputs; bit-identical across
the fused, direct and pack-then-compute variants and across pack policies."""
import itertools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_08417_gb300 import gemmfip as g  # noqa: E402
from paper_2302_08417_gb300 import inputs  # noqa: E402
from tests import gpu_util as gu  # noqa: E402

DTYPES = (np.float64, np.float32)
TINY = (0, 1, 2, 3, 5, 7, 8, 15, 16, 17, 33)


@pytest.fixture(scope="module")
def runner():
    import __graft_entry__
    __graft_entry__.build()
    return gu.Runner()


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_tiny_bruteforce_all_shapes(runner, dtype, ta, tb):
    """Every m, n, k in {0,1,2,3,5,7,8,15,16,17,33} x ld in {rows, rows+7} x beta in {0, 0.5},
    fused variant, against the oracle; C gap rows and the guard stay untouched."""
    seed = 0
    for m, n, k in itertools.product(TINY, TINY, TINY):
        for pad, beta in itertools.product((0, 7), (0.0, 0.5)):
            seed += 1
            p = inputs.problem(seed, ta, tb, m, n, k, 1.0, beta, pad, pad, pad, dtype=dtype)
            got, guard = runner.run(p, "fused")
            gu.assert_close(p, got, label="fused")
            gu.assert_gap_untouched(p, got, guard)


MEDIUM = [(200, 190, 150), (257, 129, 300), (1000, 70, 33), (33, 1000, 500), (130, 130, 1),
          (64, 64, 64), (129, 255, 17)]


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
@pytest.mark.parametrize("variant", gu.VARIANTS)
def test_medium_ragged_all_trans(runner, dtype, variant):
    """Several tiles with ragged tails, every trans combination, ld padded or not."""
    seed = 1000
    for (m, n, k), (ta, tb), pad, beta in itertools.product(
            MEDIUM, itertools.product("NT", "NT"), (0, 7), (0.0, 0.5)):
        seed += 1
        p = inputs.problem(seed, ta, tb, m, n, k, 1.0, beta, pad, pad, pad, dtype=dtype)
        got, guard = runner.run(p, variant)
        gu.assert_close(p, got, label=variant)
        gu.assert_gap_untouched(p, got, guard)


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_integer_inputs_bit_exact(runner, dtype):
    """Small integers: partial sums stay far below 2^24, so every variant is exact."""
    for (m, n, k), (ta, tb) in itertools.product(
            [(300, 200, 1000), (77, 513, 129), (1, 1, 4000)], itertools.product("NT", "NT")):
        for alpha, beta in ((1.0, 0.0), (2.0, 0.5), (-1.0, 1.0)):
            p = inputs.problem(7, ta, tb, m, n, k, alpha, beta, 3, 5, 1, dtype=dtype,
                               dist="int", int_lim=4)
            ref, _ = gu.reference(p)
            for variant in gu.VARIANTS:
                got, _ = runner.run(p, variant)
                a = inputs.as_matrix(got.astype(np.float64), m, n, p.ldc)
                b = inputs.as_matrix(ref, m, n, p.ldc)
                assert np.array_equal(a, b), (variant, ta, tb, m, n, k, alpha, beta)


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_variants_and_policies_bitwise_identical(runner, dtype):
    """Packing changes where a tile is read from, never its value: all three variants, all
    five pack policies and both packers (first tile line, shared by all CTAs) give the same
    bits."""
    for (m, n, k), (ta, tb) in itertools.product(
            [(520, 300, 700), (96, 1100, 260), (2048, 64, 48)], itertools.product("NT", "NT")):
        p = inputs.problem(3, ta, tb, m, n, k, -1.5, 0.5, 7, 0, 7, dtype=dtype)
        base, _ = runner.run(p, "direct")
        for variant in ("fused", "pack_then_compute"):
            got, _ = runner.run(p, variant)
            assert np.array_equal(got.view(np.uint8), base.view(np.uint8)), variant
        for policy, packer in itertools.product(
                (g.GFIP_PACK_AUTO, g.GFIP_PACK_NONE, g.GFIP_PACK_A, g.GFIP_PACK_B,
                 g.GFIP_PACK_BOTH), (g.GFIP_PACKER_LINE, g.GFIP_PACKER_SHARED)):
            got, _ = runner.run(p, "fused", policy=policy, packer=packer)
            assert np.array_equal(got.view(np.uint8), base.view(np.uint8)), (policy, packer)
        gu.assert_close(p, base)


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
def test_shared_packer_sizes_and_codes(runner, dtype):
    """The shared packer on shapes whose pack units do not divide over the CTAs (fewer units
    than CTAs, several rounds, ragged k), against the oracle and bitwise against direct;
    an unknown packer value is refused."""
    for (m, n, k), (ta, tb) in itertools.product(
            [(70, 300, 33), (1000, 900, 1000), (3000, 260, 900)], (("N", "N"), ("T", "T"))):
        p = inputs.problem(5, ta, tb, m, n, k, 0.75, 0.5, 7, 3, 7, dtype=dtype)
        base, _ = runner.run(p, "direct")
        got, guard = runner.run(p, "fused", policy=g.GFIP_PACK_BOTH,
                                packer=g.GFIP_PACKER_SHARED)
        assert np.array_equal(got.view(np.uint8), base.view(np.uint8)), (m, n, k, ta, tb)
        gu.assert_gap_untouched(p, got, guard)
        gu.assert_close(p, got, label="shared packer")
        assert runner.h.status() == 0
    assert g.gfip_set_packer(runner.h.h, 3) == g.GFIP_ERR_ARG
    assert g.gfip_set_packer(runner.h.h, -1) == g.GFIP_ERR_ARG


@pytest.mark.parametrize("variant", gu.VARIANTS)
def test_blas_special_values(runner, variant):
    """beta == 0 never reads C (NaN C gives no NaN); alpha == 0 and k == 0 never read A or
    B (NaN operands); alpha == 0 with beta == 1 leaves C bit for bit."""
    for dtype in DTYPES:
        p = inputs.problem(11, "N", "T", 70, 90, 40, 1.0, 0.0, 7, 7, 7, dtype=dtype)
        nanC = np.full_like(p.C0, np.nan)
        got, _ = runner.run(p, variant, C_init=nanC)
        assert not np.isnan(inputs.as_matrix(got, p.m, p.n, p.ldc)).any()
        gu.assert_close(p, got)
        for k in (0, 40):
            q = inputs.problem(12, "T", "N", 70, 90, k, 0.0 if k else 1.0, -2.0, 1, 1, 1,
                               dtype=dtype)
            q.A = np.full_like(q.A, np.nan)
            q.B = np.full_like(q.B, np.nan)
            got, guard = runner.run(q, variant)
            want = np.float64(-2.0) * inputs.as_matrix(q.C0.astype(np.float64), 70, 90, q.ldc)
            assert np.array_equal(inputs.as_matrix(got.astype(np.float64), 70, 90, q.ldc), want)
            gu.assert_gap_untouched(q, got, guard)
        q = inputs.problem(13, "N", "N", 33, 17, 9, 0.0, 1.0, 2, 2, 2, dtype=dtype)
        C0 = q.C0.copy()
        C0[5] = np.nan
        got, _ = runner.run(q, variant, C_init=C0)
        assert np.array_equal(got.view(np.uint8), C0.view(np.uint8))


def test_operands_unchanged_and_status_clean(runner):
    p = inputs.problem(21, "T", "T", 300, 260, 270, 1.0, 0.5, 7, 7, 7)
    A = torch.from_numpy(p.A).to(runner.dev)
    B = torch.from_numpy(p.B).to(runner.dev)
    for variant in gu.VARIANTS:
        runner.run(p, variant, A_dev=A, B_dev=B)
    assert np.array_equal(A.cpu().numpy().view(np.uint8), p.A.view(np.uint8))
    assert np.array_equal(B.cpu().numpy().view(np.uint8), p.B.view(np.uint8))
    assert runner.h.status() == 0


def test_workspace_reuse_across_shapes_and_garbage(runner):
    """One handle, a workspace first filled with random bytes, then a sequence of different
    shapes and variants: stale control words and packed tiles never leak into a result."""
    h = g.Handle()
    h.bind_stream()
    h.ensure_workspace("N", "N", 1500, 1500, 1500, 8)
    h.workspace.random_(0, 256)
    r = gu.Runner.__new__(gu.Runner)
    r.dev, r.h = runner.dev, h
    shapes = [(700, 650, 300, "N", "T"), (1500, 33, 999, "T", "N"), (64, 1400, 260, "T", "T"),
              (700, 650, 300, "N", "T"), (257, 257, 257, "N", "N")]
    for it, (m, n, k, ta, tb) in enumerate(shapes * 2):
        for dtype in DTYPES:
            p = inputs.problem(40 + it, ta, tb, m, n, k, 1.0, 0.5, 7, 7, 7, dtype=dtype)
            got, _ = r.run(p, gu.VARIANTS[it % 3])
            gu.assert_close(p, got, label=f"seq{it}")
    assert h.status() == 0


def test_repeated_calls_identical(runner):
    p = inputs.problem(31, "N", "N", 900, 700, 500, 1.0, 0.5, 7, 7, 7)
    first, _ = runner.run(p, "fused")
    for _ in range(5):
        again, _ = runner.run(p, "fused")
        assert np.array_equal(again.view(np.uint8), first.view(np.uint8))


def test_config_256_cube_fp64(runner):
    """The 256^3 FP64 N/N workload with lda = ldb = ldc = 256, alpha 1, beta 0.5, seeds 0-2,
    full comparison with the oracle triple loop."""
    for seed in (0, 1, 2):
        p = inputs.problem(seed, "N", "N", 256, 256, 256, 1.0, 0.5)
        for variant in gu.VARIANTS:
            got, guard = runner.run(p, variant)
            gu.assert_close(p, got, label=variant)


@pytest.mark.parametrize("dtype", DTYPES, ids=["f64", "f32"])
@pytest.mark.parametrize("n", [16, 48, 96, 192, 384, 768, 1536])
def test_size_spectrum_full_compare(runner, dtype, n):
    """Sizes of the 16..16384 sweep small enough for a full oracle product, ld = m + 7 and
    ld = m, both betas, the two trans extremes."""
    for (ta, tb), pad, beta in itertools.product((("N", "N"), ("T", "T")), (7, 0), (0.0, 0.5)):
        p = inputs.problem(n + pad, ta, tb, n, n, n, 1.0, beta, pad, pad, pad, dtype=dtype)
        ref, ab = gu.reference(p)
        for variant in gu.VARIANTS:
            got, _ = runner.run(p, variant)
            gu.assert_close(p, got, ref, ab, label=variant)
