"""Grouped GEMM (gfip_?gemm_grouped, gfip_?gemm_grouped_plan): a batch of uneven problems in
one launch, through the C ABI, against the oracle per problem: every warp-tile shape, plans
with k-splits, the tuned plan, the full 4096-problem workload; CUDA-graph replay; tuning that
leaves C untouched; invalid problems skipped with a status bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_08417_gb300 import gemmfip as g  # noqa: E402
from paper_2302_08417_gb300 import grouped as gr  # noqa: E402
from paper_2302_08417_gb300 import inputs  # noqa: E402
from tests import gpu_util as gu  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


def make_problems(seed, count, dtype, lo=4, hi=256):
    """Sizes log-uniform in [lo, hi], random operand orders, leading dims rows + {0..7}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    probs = []
    for q in range(count):
        m, n, k = (int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for _ in range(3))
        ta, tb = rng.choice(["N", "T"]), rng.choice(["N", "T"])
        pa, pb, pc = (int(x) for x in rng.integers(0, 8, 3))
        alpha = float(rng.choice([1.0, -0.5, 2.0]))
        beta = float(rng.choice([0.0, 0.5, 1.0]))
        probs.append(inputs.problem(seed * 10000 + q, ta, tb, m, n, k, alpha, beta, pa, pb, pc,
                                    dtype=dtype))
    return probs


def to_device(p, dev):
    def view(flat, rows, cols, ld):
        t = torch.from_numpy(flat).to(dev)
        return torch.as_strided(t, (rows, cols), (1, ld)), t
    A, a_buf = view(p.A, p.rows_a, p.cols_a, p.lda)
    B, b_buf = view(p.B, p.rows_b, p.cols_b, p.ldb)
    C, c_buf = view(p.C0, p.m, p.n, p.ldc)
    return A, B, C, c_buf


def build_batch(probs, dev):
    A, B, C, bufs = [], [], [], []
    for p in probs:
        a, b, c, cb = to_device(p, dev)
        A.append(a)
        B.append(b)
        C.append(c)
        bufs.append(cb)
    batch = gr.Batch([p.transa for p in probs], [p.transb for p in probs], A, B, C,
                     [p.alpha for p in probs], [p.beta for p in probs])
    return batch, bufs


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_batch_matches_oracle(dev, dtype):
    probs = make_problems(3, 300, dtype)
    tiles = gr.TILES[np.dtype(dtype).itemsize]
    for tile in tiles:
        batch, bufs = build_batch(probs, dev)
        gr.run(batch, tile)
        torch.cuda.synchronize()
        for p, buf in zip(probs, bufs):
            got = buf.cpu().numpy()
            gu.assert_close(p, got, label=f"grouped tile {tile}")
        assert g.default_handle().status() == 0


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("splits", [2, 3, 4, 8])
def test_split_plans_match_oracle(dev, dtype, splits):
    """Every problem split along k (the split tiles' partial sums added in order by the last
    warp to arrive), with the tile shapes mixed across the batch."""
    probs = make_problems(11 + splits, 160, dtype, hi=300)
    batch, bufs = build_batch(probs, dev)
    codes = [g.GFIP_GROUP_PLAN(q % 5, splits) for q in range(len(probs))]
    plan = gr.Plan(batch, codes)
    gr.run(batch, plan)
    torch.cuda.synchronize()
    for p, buf in zip(probs, bufs):
        gu.assert_close(p, buf.cpu().numpy(), label=f"split {splits}")
    assert g.default_handle().status() == 0


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_split_plan_beyond_capacity_runs_unsplit(dev, dtype):
    """A plan whose partial sums do not fit the provisioned space: the problems past the
    capacity run unsplit and the results are still right."""
    probs = make_problems(21, 64, dtype, lo=64, hi=200)
    batch, bufs = build_batch(probs, dev)
    plan = gr.Plan.uniform(batch, g.GFIP_GROUP_TILE_SMALL, 4)
    plan.split_elems //= 3
    gr.run(batch, plan)
    torch.cuda.synchronize()
    for p, buf in zip(probs, bufs):
        gu.assert_close(p, buf.cpu().numpy(), label="capacity")


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_tuning_leaves_c_untouched_whatever_beta(dev, dtype):
    probs = make_problems(31, 120, dtype)
    batch, bufs = build_batch(probs, dev)
    gr._tuned.clear()
    plan = gr.autotune_plan(batch)
    torch.cuda.synchronize()
    for p, buf in zip(probs, bufs):
        assert np.array_equal(buf.cpu().numpy().view(np.uint8), p.C0.view(np.uint8))
    assert all((c & 0xFF) in gr.TILES[np.dtype(dtype).itemsize] for c in plan.codes)
    gr.run(batch, plan)
    torch.cuda.synchronize()
    for p, buf in zip(probs, bufs):
        gu.assert_close(p, buf.cpu().numpy(), label="tuned plan")


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_full_batched_workload_matches_oracle(dev, dtype):
    """The batched workload itself: 4096 problems, m, n, k log-uniform in [4, 256], random
    operand orders, ld = rows + {0..7}, with the tuned plan, one launch replayed from a graph."""
    probs = make_problems(41, 4096, dtype)
    batch, bufs = build_batch(probs, dev)
    plan = gr.autotune_plan(batch)
    for p, buf in zip(probs, bufs):
        buf.copy_(torch.from_numpy(p.C0))
    runner = gr.GraphRunner(batch, plan)
    for p, buf in zip(probs, bufs):
        buf.copy_(torch.from_numpy(p.C0))
    runner.replay()
    torch.cuda.synchronize()
    for p, buf in zip(probs, bufs):
        gu.assert_close(p, buf.cpu().numpy(), label="4096-problem batch")
    assert runner.handle.status() == 0


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_graph_replay_and_autotune(dev, dtype):
    probs = make_problems(5, 200, dtype)
    batch, bufs = build_batch(probs, dev)
    tile = gr.autotune(batch)
    assert isinstance(tile, gr.Plan)
    # restore C, then capture one call and replay it: same result as the oracle
    for p, buf in zip(probs, bufs):
        buf.copy_(torch.from_numpy(p.C0))
    runner = gr.GraphRunner(batch, tile)      # runs once eagerly to size the workspace
    for p, buf in zip(probs, bufs):
        buf.copy_(torch.from_numpy(p.C0))
    runner.replay()
    torch.cuda.synchronize()
    for p, buf in zip(probs, bufs):
        gu.assert_close(p, buf.cpu().numpy(), label="graph replay")


def test_special_and_invalid_problems(dev):
    ps = [inputs.problem(1, "N", "T", 40, 30, 0, 1.0, -2.0),          # k == 0: C := beta C
          inputs.problem(2, "T", "N", 40, 30, 20, 0.0, 0.5),          # alpha == 0
          inputs.problem(3, "N", "N", 40, 30, 20, 0.0, 1.0),          # C unchanged
          inputs.problem(4, "N", "N", 0, 30, 20, 1.0, 0.5),           # m == 0
          inputs.problem(5, "T", "T", 33, 17, 65, 1.5, 0.0)]          # ordinary
    ps[1].A = np.full_like(ps[1].A, np.nan)                           # must not be read
    batch, bufs = build_batch(ps, dev)
    gr.run(batch, 0)
    torch.cuda.synchronize()
    for p, buf in zip(ps, bufs):
        gu.assert_close(p, buf.cpu().numpy(), label="special")
    assert g.default_handle().status() == 0
    # an invalid problem (ldc < m) is skipped and reported; the others still run
    bad = inputs.problem(6, "N", "N", 20, 10, 10, 1.0, 0.0)
    good = inputs.problem(7, "N", "N", 20, 10, 10, 1.0, 0.0)
    batch, bufs = build_batch([bad, good], dev)
    batch.ldc[0] = 5
    gr.run(batch, 0)
    torch.cuda.synchronize()
    assert np.array_equal(bufs[0].cpu().numpy().view(np.uint8), bad.C0.view(np.uint8))
    gu.assert_close(good, bufs[1].cpu().numpy())
    assert g.default_handle().status() & g.GFIP_STATUS_BAD_PROBLEM
