"""Host-side logic of the grouped GEMM (grouped.py), on CPU tensors, no GPU: size buckets,
the processing order of a plan, the partial-sum space a plan asks for, the least-padded start
of the tuner, and the balance of the kernel's dealing of work units to warps (bands of all
warps, alternately forwards and backwards) under the plan's order."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2302_08417_gb300 import gemmfip as g  # noqa: E402
from paper_2302_08417_gb300 import grouped as gr  # noqa: E402

# what the kernel source fixes (gfip_grouped.cu): k rows per chunk, the largest split factor
KC, MAX_SPLITS = 8, 8


def cpu_batch(sizes, dtype=torch.float64):
    """A Batch over CPU tensors of the given (m, n, k), operands 'N'/'N', ld = rows."""
    A = [torch.zeros((k, m), dtype=dtype).t() for m, n, k in sizes]
    B = [torch.zeros((n, k), dtype=dtype).t() for m, n, k in sizes]
    C = [torch.zeros((n, m), dtype=dtype).t() for m, n, k in sizes]
    count = len(sizes)
    return gr.Batch(["N"] * count, ["N"] * count, A, B, C, [1.0] * count, [0.0] * count)


def batched_sizes(count=4096, seed=11):
    """The batched workload's problem sizes: m, n, k log-uniform in [4, 256]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [tuple(int(x) for x in row)
            for row in np.exp(rng.uniform(np.log(4), np.log(256), (count, 3))).round()]


def test_bucket_boundaries():
    assert gr.bucket_of(16, 3, 31) == (0, 0)
    assert gr.bucket_of(17, 3, 32) == (1, 1)
    assert gr.bucket_of(5, 64, 127) == (2, 1)
    assert gr.bucket_of(65, 1, 128) == (3, 2)
    assert gr.bucket_of(129, 200, 4) == (4, 0)


def test_shapes_cover_every_tile_code():
    for esz in (4, 8):
        assert set(gr.TILES[esz]) == {0, 1, 2, 3, 4}
        for t in gr.TILES[esz]:
            bm, bn = gr.SHAPES[(esz, t)]
            assert bm * bn % 32 == 0 and bm in (8, 16, 32) and bn in (8, 16, 32)


def test_order_puts_costliest_units_first():
    sizes = [(4, 4, 256), (256, 256, 8), (64, 64, 64), (32, 16, 200), (200, 3, 3)]
    b = cpu_batch(sizes)
    codes = [g.GFIP_GROUP_PLAN(t, 1) for t in (0, 0, 2, 1, 4)]
    order = b.order_for(codes).tolist()
    cost = [gr.unit_cost(8, c & 0xFF, c >> 8, *s) for s, c in zip(sizes, codes)]
    assert sorted(order) == list(range(len(sizes)))
    assert [cost[q] for q in order] == sorted(cost, reverse=True)
    # a unit's cost follows its k range: the k = 256 problem's units come first
    assert order[0] == 0


def test_plan_split_space_covers_what_the_kernel_uses():
    """The partial-sum elements a Plan provisions are at least what the prepare kernel gives
    each split problem (splits clamped to the chunks and to MAX_SPLITS, no empty k-range)."""
    rng = np.random.Generator(np.random.PCG64(3))
    sizes = [tuple(int(x) for x in rng.integers(1, 300, 3)) for _ in range(400)]
    b = cpu_batch(sizes)
    codes = [g.GFIP_GROUP_PLAN(int(rng.integers(0, 5)), int(rng.choice([1, 2, 3, 4, 8])))
             for _ in sizes]
    plan = gr.Plan(b, codes)
    need = 0
    for (m, n, k), c in zip(sizes, codes):
        bm, bn = gr.SHAPES[(8, c & 0xFF)]
        chunks = math.ceil(k / KC)
        s = max(1, min(c >> 8, MAX_SPLITS, chunks))
        ks = math.ceil(chunks / s)
        s = math.ceil(chunks / ks)
        if s > 1:
            need += math.ceil(m / bm) * math.ceil(n / bn) * s * bm * bn
    assert plan.split_elems >= need


def test_tuner_starts_from_the_least_padded_tile():
    b = cpu_batch([(5, 9, 40), (6, 7, 40), (200, 250, 40), (30, 30, 300)])
    start = gr._initial_tiles(b)
    for bucket, tile in start.items():
        members = [s for s in b.sizes if gr.bucket_of(*s) == bucket]
        work = {t: sum(gr.padded_work(8, t, *s) for s in members) for t in gr.TILES[8]}
        assert work[tile] == min(work.values())
    assert start[gr.bucket_of(5, 9, 40)] in (3, 4)      # 16 x 8 or 8 x 16 for tiny problems


def deal(units, nwarps):
    """The kernel's dealing of units (in processing order) to warps: bands of nwarps units,
    alternately forwards and backwards; returns each warp's summed cost."""
    load = np.zeros(nwarps)
    for band, u0 in enumerate(range(0, len(units), nwarps)):
        seg = units[u0:u0 + nwarps]
        if band % 2 == 0:
            load[:len(seg)] += seg
        else:
            load[nwarps - len(seg):] += seg[::-1]
    return load


def units_in_order(b, plan, esz):
    out = []
    for q in plan.order.tolist():
        (m, n, k), c = b.sizes[q], plan.codes[q]
        bm, bn = gr.SHAPES[(esz, c & 0xFF)]
        tiles = math.ceil(m / bm) * math.ceil(n / bn)
        out += [gr.unit_cost(esz, c & 0xFF, c >> 8, m, n, k)] * (tiles * max(1, c >> 8))
    return np.array(out, dtype=np.float64)


@pytest.mark.parametrize("tile", [0, 2, 4])
def test_dealing_under_the_plan_order_is_balanced(tile):
    """On the batched workload the busiest of 3040 warps (152 SMs x 2 CTAs x 10 warps) gets
    at most 6 % above the mean cost under the plan's order (1.05, 1.02, 1.02 for these
    shapes); dealing the same units in order of m n k, round-robin, leaves the busiest warp
    at least 20 % above it (2.1, 1.5, 1.3)."""
    sizes = batched_sizes()
    b = cpu_batch(sizes, torch.float32)
    plan = gr.Plan.uniform(b, tile)
    units = units_in_order(b, plan, 4)
    nwarps = 3040
    load = deal(units, nwarps)
    assert load.max() / load.mean() <= 1.06
    by_mnk = sorted(range(len(sizes)), key=lambda q: -sizes[q][0] * sizes[q][1] * sizes[q][2])
    rr = []
    for q in by_mnk:
        m, n, k = sizes[q]
        bm, bn = gr.SHAPES[(4, tile)]
        rr += [gr.unit_cost(4, tile, 1, m, n, k)] * (math.ceil(m / bm) * math.ceil(n / bn))
    rr = np.array(rr, dtype=np.float64)
    load_rr = np.zeros(nwarps)
    for u0 in range(0, len(rr), nwarps):
        seg = rr[u0:u0 + nwarps]
        load_rr[:len(seg)] += seg
    assert load_rr.max() / load_rr.mean() >= 1.2 * load.max() / load.mean()
