"""Index arithmetic of the row tiles (common.cuh: warp_rows, tile_own_row,
tile_tree / tile_combine), restated in Python and checked for the properties
the CUDA kernels rely on: every row is owned by exactly one lane of exactly one
warp, the row extents a round reads come from the lane that owns that row, and
the transposed reduction leaves in each lane the sum of its own row, added in
the same tree as a per-row shuffle reduction (lanes W/2 apart first)."""
import itertools

import pytest


def ceil_div(a, b):
    return (a + b - 1) // b


def warp_rows(n, w, nwarps, W):
    G = 32 // W
    units = ceil_div(n, G)
    q, rem = divmod(units, nwarps)
    u0 = w * q + min(w, rem)
    u1 = u0 + q + (1 if w < rem else 0)
    return min(u0 * G, n), min(u1 * G, n)


def tile_own_row(lane, W):
    return (lane % W) * (32 // W) + lane // W


@pytest.mark.parametrize("W", [4, 8])
@pytest.mark.parametrize("n", [0, 1, 7, 31, 32, 33, 125, 1000, 4097, 262144])
@pytest.mark.parametrize("nwarps", [8, 24, 7296])
def test_warp_rows_partition_rows(W, n, nwarps):
    G = 32 // W
    seen = []
    lengths = []
    for w in range(nwarps):
        r0, r1 = warp_rows(n, w, nwarps, W)
        assert 0 <= r0 <= r1 <= n
        if r0 < r1:
            assert r0 % G == 0  # ranges start on a round boundary
            lengths.append(r1 - r0)
        seen.append((r0, r1))
    # consecutive, disjoint, covering [0, n)
    pos = 0
    for r0, r1 in seen:
        if r0 == r1:
            continue
        assert r0 == pos
        pos = r1
    assert pos == n
    if lengths:  # balanced to within one round (the last range may be short)
        assert max(lengths) - min(lengths) <= 2 * G


@pytest.mark.parametrize("W", [4, 8])
@pytest.mark.parametrize("rows", [1, 3, 4, 8, 17, 29, 32])
def test_tile_lanes_own_each_row_once_and_rounds_read_the_owner(W, rows):
    G = 32 // W
    own = [tile_own_row(l, W) for l in range(32)]
    assert sorted(own) == list(range(32))
    assert sorted(o for o in own if o < rows) == list(range(rows))
    for t in range(W):
        if t * G >= rows:
            continue  # the round is skipped by every lane (warp-uniform)
        for g in range(G):
            # round t's row of group g is t G + g; its extents are shuffled from lane g W + t
            assert own[g * W + t] == t * G + g


def transposed_reduction(W):
    """Symbolic run of tile_tree/tile_combine for one group: partial[l][t] is
    lane l's partial of round t; returns each lane's final expression."""
    def tree(O, t0):  # the same shape in every lane; leaves name rounds
        if O == W:
            return ("round", t0)
        return (tree(2 * O, t0), tree(2 * O, t0 + O), O)

    def evaluate(lane, node):
        if node[0] == "round":
            return ("p", lane, node[1])
        lo_node, hi_node, O = node
        lo_mine, hi_mine = evaluate(lane, lo_node), evaluate(lane, hi_node)
        partner = lane ^ O
        lo_p, hi_p = evaluate(partner, lo_node), evaluate(partner, hi_node)
        up = (lane & O) != 0
        keep, recv = (hi_mine, hi_p) if up else (lo_mine, lo_p)
        # the lower lane's value is added first on both sides
        return ("+", recv, keep) if up else ("+", keep, recv)

    return [evaluate(l, tree(1, 0)) for l in range(W)]


def row_reduce_tree(W, t):
    """row_reduce's result in lane 0 for round t: lanes W/2 apart first."""
    vals = [("p", l, t) for l in range(W)]
    o = W // 2
    while o > 0:
        vals = [("+", vals[l], vals[l + o]) for l in range(o)]
        o //= 2
    return vals[0]


@pytest.mark.parametrize("W", [4, 8])
def test_transposed_reduction_matches_row_reduce_tree(W):
    final = transposed_reduction(W)
    for lane in range(W):
        # lane `lane` of a group ends with round `lane`, summed exactly as row_reduce sums it
        assert final[lane] == row_reduce_tree(W, lane)


@pytest.mark.parametrize("W", [4, 8])
def test_lane_entry_count(W):
    # tile_nmax: lane `sub` of a row group takes entries beg + sub + j W < end;
    # their count is (len - sub + W - 1) / W, never negative
    for length, sub in itertools.product(range(0, 70), range(W)):
        cnt = (length - sub + W - 1) // W
        assert cnt >= 0
        assert cnt == len(range(sub, length, W))
