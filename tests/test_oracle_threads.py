"""The oracle's results do not depend on how many host threads run its row loops.

Independent rows may run on any thread without changing their arithmetic; whole-vector sums (inner
products and norms) are taken in a fixed block order: consecutive blocks of 4096 terms, each added
left to right, then the block sums left to right.  The block order is pinned here against a
restatement of that definition and against the exactly rounded sum; the whole set-up and solve are
compared bit for bit at one and at four threads."""
import math

import numpy as np
import pytest

import battery_system as bs
import oracle

BLOCK = 4096


def blocked_sum(a, b):
    parts = []
    for lo in range(0, len(a), BLOCK):
        s = 0.0
        for x, y in zip(a[lo:lo + BLOCK].tolist(), b[lo:lo + BLOCK].tolist()):
            s += x * y
        parts.append(s)
    t = 0.0
    for p in parts:
        t += p
    return t


@pytest.mark.parametrize("n", [0, 1, 17, 4096, 4097, 3 * 4096 + 5, 40_000])
def test_sum_prod_is_the_block_ordered_sum(n):
    rng = np.random.default_rng(n + 1)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    got = oracle.sum_prod(a, b)
    assert got == blocked_sum(a, b)
    exact = math.fsum((a * b).tolist()) if n else 0.0
    # a sum of n rounded products in any order: |error| <= (n + 1) eps sum |a b|
    assert abs(got - exact) <= (n + 1) * np.finfo(float).eps * float(np.abs(a * b).sum())


def _run(system, threads):
    oracle.set_threads(threads)
    o = oracle.bgs_for_system(system, opts=oracle.default_options(max_coarse=40))
    x, info = o.solve(system.b)
    levels = []
    for k in range(5):
        a = o.amg(k)
        lv = []
        for l in range(a.nlevels):
            A = a.level_matrix(l)
            item = [A.rowptr.copy(), A.col.copy(), A.val.copy()]
            if l + 1 < a.nlevels:
                P = a.prolongator(l)
                item += [a.aggregates(l).copy(), P.val.copy(), a.omega(l), a.cheb_bounds(l)]
            lv.append(item)
        levels.append(lv)
    return x, info.iters, levels


def _same(u, v):
    if isinstance(u, (list, tuple)):
        return len(u) == len(v) and all(_same(p, q) for p, q in zip(u, v))
    if isinstance(u, np.ndarray):
        return u.dtype == v.dtype and np.array_equal(u, v)
    return u == v


def test_setup_and_solve_are_bit_identical_at_any_thread_count():
    system = bs.assemble(grid=bs.Grid(3, 14, 12, 10), seed=3)    # 8400 DOFs: several sum blocks
    default = oracle.set_threads(0)
    try:
        x1, it1, lv1 = _run(system, 1)
        x4, it4, lv4 = _run(system, 4)
    finally:
        oracle.set_threads(default)
    assert it1 == it4
    assert np.array_equal(x1, x4)
    assert _same(lv1, lv4)
