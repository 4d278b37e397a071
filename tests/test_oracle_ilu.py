"""Pins of the oracle's DD(0)-ILU(0) subblock solver (one-level restricted additive Schwarz without
overlap, one ILU(0) sweep per subdomain; Sec. 2.1 Eq. one-level-schwarz, Sec. 3.1.1), all against
dense linear algebra:
  * ILU(0) reproduces A on its pattern: (L U)_ij = a_ij wherever a_ij is stored;
  * without fill-in (a tridiagonal matrix) ILU(0) is the exact LU, so the sweep solves exactly;
  * the preconditioner is block diagonal over the subdomains and each block is (L_s U_s)^-1 of the
    subdomain matrix;
  * the transposed sweep is the adjoint: <M^-T a, b> = <a, M^-1 b>;
  * inside the block sweep, species blocks on DD(0)-ILU(0) still give a converged solve."""
import numpy as np
import pytest

import battery_system as bs
import oracle
from battery_system import spec


def _csr(B):
    return oracle.CSR(B.rowptr, B.col, B.val, B.nrows, B.ncols)


def _lu_dense(F):
    D = F.to_dense()
    L = np.tril(D, -1) + np.eye(F.nrows)
    U = np.triu(D)
    return L, U


@pytest.mark.parametrize("rows", [10_000, 97])
def test_ilu0_reproduces_a_on_its_pattern(rows):
    s = bs.assemble(grid=bs.Grid(3, 8, 7, 6), seed=3)
    A = _csr(s.blocks[(spec.C1, spec.C1)])             # nonsymmetric: diffusion + upwind advection
    m = oracle.ILU(A, rows)
    assert m.status == 0
    F = m.factors()
    L, U = _lu_dense(F)
    LU = L @ U
    Ad = A.to_dense()
    rows_ = np.repeat(np.arange(F.nrows), np.diff(F.rowptr))
    assert np.abs(LU[rows_, F.col] - Ad[rows_, F.col]).max() <= 1e-13 * np.abs(Ad).max()
    # the kept pattern is A's pattern restricted to the subdomains
    sub = lambda i: i // rows
    keep = np.array([sub(i) == sub(j) for i, j in zip(np.repeat(np.arange(A.nrows), np.diff(A.rowptr)), A.col)])
    assert F.nnz == int(keep.sum())


def test_ilu0_without_fill_is_exact():
    n = 200
    rng = np.random.default_rng(5)
    lo, di, up = rng.uniform(-1, -0.1, n - 1), rng.uniform(3, 4, n), rng.uniform(-1, -0.1, n - 1)
    D = np.diag(di) + np.diag(lo, -1) + np.diag(up, 1)
    rp = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                cols.append(j)
                vals.append(D[i, j])
        rp[i + 1] = len(cols)
    A = oracle.CSR(rp, np.array(cols), np.array(vals), n, n)
    m = oracle.ILU(A, n)
    b = rng.standard_normal(n)
    x = m.apply(b)
    assert np.abs(x - np.linalg.solve(D, b)).max() <= 1e-12 * np.abs(x).max()


def test_dd_sweep_is_block_diagonal_over_subdomains():
    s = bs.assemble(grid=bs.Grid(3, 9, 8, 7), seed=2)
    A = _csr(s.blocks[(spec.C2, spec.C2)])
    R = 64
    m = oracle.ILU(A, R)
    F = m.factors()
    L, U = _lu_dense(F)
    r = np.random.default_rng(1).standard_normal(A.nrows)
    z = m.apply(r)
    n = A.nrows
    for s0 in range(0, n, R):
        s1 = min(n, s0 + R)
        zs = np.linalg.solve(U[s0:s1, s0:s1], np.linalg.solve(L[s0:s1, s0:s1], r[s0:s1]))
        assert np.abs(z[s0:s1] - zs).max() <= 1e-12 * max(1.0, np.abs(zs).max())
    # no coupling between subdomains: L and U are block diagonal
    blockmask = np.equal.outer(np.arange(n) // R, np.arange(n) // R)
    assert not np.any((L - np.eye(n))[~blockmask]) and not np.any(U[~blockmask])


def test_transposed_sweep_is_the_adjoint():
    s = bs.assemble(grid=bs.Grid(3, 9, 8, 7), seed=2)
    m = oracle.ILU(_csr(s.blocks[(spec.C1, spec.C1)]), 100)
    rng = np.random.default_rng(8)
    a, b = rng.standard_normal(s.ncells), rng.standard_normal(s.ncells)
    lhs = m.apply_transposed(a) @ b
    rhs = a @ m.apply(b)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_block_sweep_with_dd_ilu_species_solves():
    s = bs.assemble(grid=bs.Grid(3, 10, 9, 8), seed=4)
    sub = [0, 0, 0, 1, 1]                                # c1, c2 on DD(0)-ILU(0)
    o = oracle.bgs_for_system(s, order=list(spec.WORKLOAD_ORDER),
                              opts=oracle.default_options(subsolver=sub, ilu_rows=128, max_coarse=40))
    for k in (spec.C1, spec.C2):
        assert not o.p.contents.amg[k] and o.ilu(k).status == 0
    x, info = o.solve(s.b)
    assert info.converged
    assert np.linalg.norm(s.b - s.matvec(x)) <= 1e-8 * np.linalg.norm(s.b)
    lam, ia = o.solve_adjoint(s.b)
    assert ia.converged
    # x = A^-1 b and lam = A^-T b, so b.x = lam.b up to the solve tolerance
    assert abs(s.b @ x - lam @ s.b) <= 1e-6 * abs(s.b @ x)
