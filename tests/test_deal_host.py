"""The engine's launch-table dealing rule (csrc/deal.h), built here with g++:
every item placed exactly once, holes only in the last round, items ranked
by decreasing size, one system alone left in item order, and the block loads
of very uneven members balanced where a round-robin table is not."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        out = os.path.join(tempfile.mkdtemp(prefix="deal_host_"), "libdeal_host.so")
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                               "-I", os.path.join(ROOT, "paper_2510_27517_gb300", "csrc"),
                               os.path.join(ROOT, "tests", "deal_host.cpp"), "-o", out])
        _LIB = ctypes.CDLL(out)
        _LIB.deal_table.restype = ctypes.c_int64
    return _LIB


def deal(weights, grid):
    w = np.ascontiguousarray(weights, dtype=np.float64)
    npos = -(-len(w) // grid) * grid
    table = np.empty(max(npos, 1), dtype=np.int32)
    got = lib().deal_table(ctypes.c_void_p(w.ctypes.data), ctypes.c_int64(len(w)), ctypes.c_int(grid),
                           ctypes.c_void_p(table.ctypes.data))
    assert got == npos
    return table[:npos]


def block_loads(table, weights, grid):
    loads = np.zeros(grid)
    for p, item in enumerate(table):
        if item >= 0:
            loads[p % grid] += weights[item]
    return loads


@pytest.mark.parametrize("items,grid", [(1, 1), (7, 3), (445, 445), (446, 445), (1000, 455), (4842, 455),
                                        (5, 8)])
def test_every_item_once_holes_only_in_the_last_round(items, grid):
    rng = np.random.default_rng(items + grid)
    w = rng.lognormal(0.0, 1.5, items)
    t = deal(w, grid)
    placed = t[t >= 0]
    assert sorted(placed.tolist()) == list(range(items))
    holes = np.nonzero(t < 0)[0]
    assert len(holes) == len(t) - items
    if len(holes):
        assert holes.min() >= len(t) - grid  # all in the last round


def test_ranked_by_decreasing_size_in_a_snake():
    rng = np.random.default_rng(3)
    grid = 16
    w = rng.integers(1, 9, 70).astype(np.float64)
    t = deal(w, grid)
    order = np.argsort(-w, kind="stable")  # ties keep their order
    for j, item in enumerate(order):
        r, c = divmod(j, grid)
        pos = r * grid + (grid - 1 - c if r % 2 else c)
        assert t[pos] == item


def test_one_system_alone_keeps_item_order():
    # equal items except a short last one: one round is the identity, so a
    # system alone runs item v in block v
    w = np.full(445, 10.0)
    w[-1] = 3.0
    assert np.array_equal(deal(w, 445), np.arange(445))
    assert np.array_equal(deal(w[:300], 445)[:300], np.arange(300))


def test_uneven_members_balance_better_than_round_robin():
    # items of 512 members of log-uniform sizes (about the anisotropic batch):
    # each member's items are equal but members differ by two orders
    rng = np.random.default_rng(11)
    w = []
    for _ in range(512):
        groups = int(np.exp(rng.uniform(np.log(2), np.log(1100))))
        k = max(1, groups // 12)
        w += [float(min(k, groups - v * k)) for v in range(-(-groups // k))]
    w = np.array(w)
    grid = 455
    snake = block_loads(deal(w, grid), w, grid)
    rr = block_loads(np.arange(len(w)), w, grid)
    assert snake.max() / snake.mean() < 1.15  # about 1.10 here
    assert rr.max() / rr.mean() > 1.5 * snake.max() / snake.mean()  # round robin: about 2.2
