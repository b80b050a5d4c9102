"""The column blocks of the pipelined end-to-end path (CPU only): they tile [0, n) in order,
each at least HOST_BLOCK_COLS wide, one range for op(B) = B^T or short C; the storage spans
the blocks copy are disjoint, lie inside the matrix's span and leave out exactly the gap
rows m..ld-1 of each block's last column."""
import itertools

import pytest

from paper_2302_08417_gb300 import gemmfip as g


@pytest.mark.parametrize("block", [64, 1024])
def test_blocks_tile_the_columns(monkeypatch, block):
    monkeypatch.setattr(g, "HOST_BLOCK_COLS", block)
    for n in (0, 1, block - 1, block, 2 * block - 1, 2 * block, 2 * block + 1, 7 * block + 5,
              8192):
        for tb in "NnTt":
            r = g.host_blocks(n, tb)
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            if tb in "Tt" or n < 2 * block:
                assert r == [(0, n)]
            else:
                assert len(r) == n // block
                assert all(j1 - j0 >= block for j0, j1 in r)
                assert max(j1 - j0 for j0, j1 in r) - min(j1 - j0 for j0, j1 in r) <= 1


def test_block_spans_disjoint_and_skip_boundary_gaps(monkeypatch):
    monkeypatch.setattr(g, "HOST_BLOCK_COLS", 16)
    for n, rows, pad in itertools.product((32, 50, 97), (1, 5, 16), (0, 3)):
        ld = rows + pad
        covered = set()
        for j0, j1 in g.host_blocks(n, "N"):
            span = set(range(j0 * ld, (j1 - 1) * ld + rows))
            assert not (span & covered)
            covered |= span
        whole = set(range(0, (n - 1) * ld + rows))
        assert covered <= whole
        # what no block copies: the gap rows after the last column of every block but the last
        boundary_cols = [j1 - 1 for _, j1 in g.host_blocks(n, "N")[:-1]]
        missing = {c * ld + r for c in boundary_cols for r in range(rows, ld)}
        assert whole - covered == missing
