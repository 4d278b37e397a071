"""Pins of the oracle's block Gauss-Seidel sweep, FGMRES and adjoint against dense linear algebra."""
import numpy as np
import pytest

import battery_system as bs
import oracle
from battery_system import spec


def small_system(grid=None, seed=1):
    return bs.assemble(grid=grid or bs.Grid(3, 6, 6, 6), seed=seed)


def lower_block_matrix(system, order):
    """Dense matrix of the blocks kept by the forward sweep (pos(j) <= pos(k))."""
    n = system.ncells
    pos = {f: p for p, f in enumerate(order)}
    M = np.zeros((system.ndof, system.ndof))
    for (r, c), blk in system.blocks.items():
        if pos[c] <= pos[r]:
            M[r * n:(r + 1) * n, c * n:(c + 1) * n] = blk.to_dense()
    return M


@pytest.mark.parametrize("order", [spec.WORKLOAD_ORDER, spec.PAPER_ORDER])
def test_bgs_with_exact_block_solves_is_the_block_triangular_inverse(order):
    s = small_system(bs.Grid(3, 4, 4, 4))
    opts = oracle.default_options(max_coarse=10_000)       # every block: one dense LU level
    o = oracle.bgs_for_system(s, order=list(order), opts=opts)
    for k in range(5):
        assert o.amg(k).nlevels == 1
    M = lower_block_matrix(s, order)
    v = np.random.default_rng(2).standard_normal(s.ndof)
    z = o.apply(v)
    ref = np.linalg.solve(M, v)
    assert np.abs(z - ref).max() <= 1e-10 * np.abs(ref).max()


def test_block_jacobi_with_exact_block_solves_is_the_block_diagonal_inverse():
    """Block Jacobi (couplings left out, Secs. 3.2 and 4): M^-1 = blockdiag(A_kk)^-1, in either
    direction (the adjoint of a block-diagonal M is blockdiag(A_kk^T)^-1)."""
    s = small_system(bs.Grid(3, 4, 4, 4))
    opts = oracle.default_options(max_coarse=10_000, jacobi=1)
    o = oracle.bgs_for_system(s, order=list(spec.WORKLOAD_ORDER), opts=opts)
    n = s.ncells
    D = np.zeros((s.ndof, s.ndof))
    for k in range(5):
        D[k * n:(k + 1) * n, k * n:(k + 1) * n] = s.blocks[(k, k)].to_dense()
    v = np.random.default_rng(4).standard_normal(s.ndof)
    ref = np.linalg.solve(D, v)
    assert np.abs(o.apply(v) - ref).max() <= 1e-10 * np.abs(ref).max()
    refT = np.linalg.solve(D.T, v)
    assert np.abs(o.apply_adjoint(v) - refT).max() <= 1e-10 * np.abs(refT).max()
    # with AMG blocks the Jacobi-preconditioned FGMRES still solves, in more iterations than GS
    gs = oracle.bgs_for_system(s, opts=oracle.default_options(max_coarse=20))
    jac = oracle.bgs_for_system(s, opts=oracle.default_options(max_coarse=20, jacobi=1))
    xg, ig = gs.solve(s.b)
    xj, ij = jac.solve(s.b)
    assert ig.converged and ij.converged and ij.iters >= ig.iters
    assert np.linalg.norm(xj - xg) <= 1e-6 * np.linalg.norm(xg)


def test_fgmres_converges_in_one_iteration_without_upper_blocks():
    s = small_system(bs.Grid(3, 4, 4, 4))
    order = list(spec.WORKLOAD_ORDER)
    pos = {f: p for p, f in enumerate(order)}
    blocks = [[s.blocks.get((r, c)) if pos[c] <= pos[r] else None for c in range(5)] for r in range(5)]
    o = oracle.BGS(blocks, s.field_sizes, order, oracle.default_options(max_coarse=10_000))
    assert o.setup() == 0
    x, info = o.solve(s.b)
    assert info.converged and info.iters == 1


@pytest.mark.parametrize("grid,mc", [(bs.Grid(3, 6, 6, 6), 20), (bs.Grid(2, 16, 16, 1), 30)])
def test_whole_solve_matches_dense_lu(grid, mc):
    s = small_system(grid)
    opts = oracle.default_options(max_coarse=mc, rtol=1e-12)
    o = oracle.bgs_for_system(s, opts=opts)
    assert max(o.amg(k).nlevels for k in range(5)) >= 2      # the AMG path is exercised
    x, info = o.solve(s.b)
    assert info.converged and info.rel_true_resid <= 1e-12
    xd = oracle.dense_solve(s.full_dense(), s.b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_paper_order_also_converges():
    s = small_system()
    o = oracle.bgs_for_system(s, order=list(spec.PAPER_ORDER), opts=oracle.default_options(max_coarse=20))
    x, info = o.solve(s.b)
    assert info.converged
    r = s.b - s.matvec(x)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(s.b)


def test_fgmres_terminates_within_n_and_residual_estimates_monotone():
    rng = np.random.default_rng(11)
    n = 20
    A = rng.standard_normal((n, n)) + 6 * np.eye(n)
    b = rng.standard_normal(n)
    ests = []

    def amul(x):
        return A @ x

    x, info = oracle.fgmres(n, amul, lambda v: v, b, restart=50, maxit=1000, rtol=1e-12)
    assert info.converged and info.iters <= n
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b) * 10
    # monotone residual estimates: run with growing maxit (no restarts inside)
    for it in range(1, info.iters + 1):
        _, inf2 = oracle.fgmres(n, amul, lambda v: v, b, restart=50, maxit=it, rtol=1e-12)
        ests.append(inf2.rel_est_resid)
    assert all(a >= b_ - 1e-15 for a, b_ in zip(ests, ests[1:]))
    # a varying (flexible) preconditioner is allowed
    calls = {"k": 0}

    def prec(v):
        calls["k"] += 1
        return v * (1.0 + 0.1 * (calls["k"] % 3))

    x, info = oracle.fgmres(n, amul, prec, b, restart=50, maxit=1000, rtol=1e-10)
    assert info.converged and np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b) * 10


def test_restarted_fgmres_true_residual():
    s = small_system()
    opts = oracle.default_options(max_coarse=20, restart=3)
    o = oracle.bgs_for_system(s, opts=opts)
    x, info = o.solve(s.b)
    assert info.converged and info.iters > 3
    assert np.linalg.norm(s.b - s.matvec(x)) <= 1e-8 * np.linalg.norm(s.b)


def test_nonconvergence_reported():
    s = small_system()
    o = oracle.bgs_for_system(s, opts=oracle.default_options(max_coarse=20, maxit=1))
    x, info = o.solve(s.b)
    assert not info.converged and info.status == 3 and info.iters == 1


def test_adjoint_solve_against_dense_and_duality():
    s = small_system()
    opts = oracle.default_options(max_coarse=20, rtol=1e-12)
    o = oracle.bgs_for_system(s, opts=opts)
    rng = np.random.default_rng(4)
    g = rng.standard_normal(s.ndof)
    lam, info = o.solve_adjoint(g)
    assert info.converged
    Ad = s.full_dense()
    lref = np.linalg.solve(Ad.T, g)
    assert np.linalg.norm(lam - lref) <= 1e-9 * np.linalg.norm(lref)
    x, _ = o.solve(s.b)
    # g^T x = lambda^T b
    assert abs(g @ x - lam @ s.b) <= 1e-9 * abs(g @ x)
    # the transposed sweep with exact block solves inverts the transposed upper block matrix
    ob = oracle.bgs_for_system(s, opts=oracle.default_options(max_coarse=10_000))
    M = lower_block_matrix(s, spec.WORKLOAD_ORDER)
    z = ob.apply_adjoint(g)
    assert np.abs(z - np.linalg.solve(M.T, g)).max() <= 1e-9 * np.abs(z).max()


def test_grad_values_is_minus_lambda_x_on_pattern():
    s = small_system(bs.Grid(3, 4, 4, 4))
    o = oracle.bgs_for_system(s, opts=oracle.default_options(max_coarse=20, rtol=1e-13))
    x, _ = o.solve(s.b)
    # loss = c^T x ; dL/dA = -lambda x^T with A^T lambda = c ; check by finite differences
    c = np.zeros(s.ndof)
    c[s.collector] = 1.0 / len(s.collector)
    lam, _ = o.solve_adjoint(c)
    blk = s.blocks[(0, 0)]
    rows = np.repeat(np.arange(blk.nrows), np.diff(blk.rowptr))
    g = -(lam[rows] * x[blk.col])
    Ad = s.full_dense()
    for e in [0, 5, blk.nnz // 2, blk.nnz - 1]:
        hstep = 1e-6 * abs(blk.val[e])
        Ap, Am = Ad.copy(), Ad.copy()
        Ap[rows[e], blk.col[e]] += hstep
        Am[rows[e], blk.col[e]] -= hstep
        fd = (c @ np.linalg.solve(Ap, s.b) - c @ np.linalg.solve(Am, s.b)) / (2 * hstep)
        # relative 1e-5, plus the rounding floor of the dense solves (|L| eps / h)
        assert abs(fd - g[e]) <= 1e-5 * abs(fd) + 1e-13 * abs(c @ x) / hstep


def group_lower_matrix(system, order, group_end):
    """Dense matrix of the blocks the nested preconditioner inverts: whole diagonal groups and the
    couplings from earlier groups to later ones."""
    n = system.ncells
    grp = {}
    start = 0
    for g, end in enumerate(group_end):
        for p in range(start, end):
            grp[order[p]] = g
        start = end
    M = np.zeros((system.ndof, system.ndof))
    for (r, c), blk in system.blocks.items():
        if grp[c] <= grp[r]:
            M[r * n:(r + 1) * n, c * n:(c + 1) * n] = blk.to_dense()
    return M


@pytest.mark.parametrize("order,group_end", [(spec.WORKLOAD_ORDER, [2, 5]), (spec.PAPER_ORDER, [3, 5])],
                         ids=["voltage-first", "paper-order"])
def test_nested_with_exact_inner_solves_is_the_group_triangular_inverse(order, group_end):
    """Nested variant (Sec. 2.2, Eq. hierarchical-bgs over the groups; inner FGMRES per group): with
    the inner solves converged to 1e-13, M^-1 = (group-block lower triangle of A)^-1."""
    s = small_system(bs.Grid(3, 5, 4, 4))
    opts = oracle.default_options(max_coarse=20, ngroups=2, group_end=group_end, inner_rtol=1e-13,
                                  inner_maxit=400, inner_restart=60)
    o = oracle.bgs_for_system(s, order=list(order), opts=opts)
    M = group_lower_matrix(s, list(order), group_end)
    v = np.random.default_rng(6).standard_normal(s.ndof)
    ref = np.linalg.solve(M, v)
    assert np.linalg.norm(o.apply(v) - ref) <= 1e-9 * np.linalg.norm(ref)
    refT = np.linalg.solve(M.T, v)
    assert np.linalg.norm(o.apply_adjoint(v) - refT) <= 1e-9 * np.linalg.norm(refT)


def test_nested_outer_converges_in_one_iteration_without_upper_group_couplings():
    """The paper's observation for the nested solver (outer FGMRES in one iteration) holds exactly
    when no coupling points from a later group to an earlier one and the inner solves are exact."""
    s = small_system(bs.Grid(3, 4, 4, 4))
    order = list(spec.WORKLOAD_ORDER)
    grp = {0: 0, 1: 0, 2: 1, 3: 1, 4: 1}
    blocks = [[s.blocks.get((r, c)) if grp[c] <= grp[r] else None for c in range(5)] for r in range(5)]
    opts = oracle.default_options(max_coarse=10, ngroups=2, group_end=[2, 5], inner_rtol=1e-13,
                                  inner_maxit=400, inner_restart=60, restart=5)
    o = oracle.BGS(blocks, s.field_sizes, order, opts)
    assert o.setup() == 0
    x, info = o.solve(s.b)
    assert info.converged and info.iters == 1


def test_nested_solve_matches_flattened_solve():
    s = small_system(bs.Grid(3, 8, 7, 6), seed=3)
    order = list(spec.WORKLOAD_ORDER)
    flat = oracle.bgs_for_system(s, order=order, opts=oracle.default_options(max_coarse=30))
    nest = oracle.bgs_for_system(s, order=order, opts=oracle.default_options(
        max_coarse=30, ngroups=2, group_end=[2, 5], restart=5))
    xf, inf_ = flat.solve(s.b)
    xn, inn = nest.solve(s.b)
    assert inf_.converged and inn.converged
    assert inn.iters < inf_.iters                     # each outer step holds inner solves
    assert np.linalg.norm(xn - xf) <= 1e-6 * np.linalg.norm(xf)
    assert np.linalg.norm(s.b - s.matvec(xn)) <= 1e-8 * np.linalg.norm(s.b)
    lf, _ = flat.solve_adjoint(s.b)
    ln, ia = nest.solve_adjoint(s.b)
    assert ia.converged and np.linalg.norm(ln - lf) <= 1e-6 * np.linalg.norm(lf)


def test_diagonal_field_solved_exactly_in_a_six_field_system():
    """A sixth field with a diagonal block (the solid species A_s of Sec. 2.2, inverted directly):
    subsolver 2 applies 1/diag exactly, so with dense-LU solves on the other blocks the sweep is the
    block-triangular inverse of the six-field system; with V-cycles the system solves."""
    from six_field import six_field, dense, SOLID
    nested, sizes, b = six_field(bs.Grid(3, 4, 4, 4), seed=2)
    order = list(spec.WORKLOAD_ORDER) + [SOLID]
    pos = {f: p for p, f in enumerate(order)}
    sub = [0, 0, 0, 0, 0, 2]
    o = oracle.BGS(nested, sizes, order, oracle.default_options(max_coarse=10_000, subsolver=sub))
    assert o.setup() == 0
    M = dense([[B if (B is not None and pos[c] <= pos[r]) else None for c, B in enumerate(row)]
               for r, row in enumerate(nested)], sizes)
    v = np.random.default_rng(3).standard_normal(sum(sizes))
    ref = np.linalg.solve(M, v)
    assert np.abs(o.apply(v) - ref).max() <= 1e-10 * np.abs(ref).max()
    o2 = oracle.BGS(nested, sizes, order, oracle.default_options(max_coarse=20, subsolver=sub))
    assert o2.setup() == 0
    x, info = o2.solve(b)
    A = dense(nested, sizes)
    assert info.converged and np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
