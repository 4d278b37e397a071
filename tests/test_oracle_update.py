"""Pins of the oracle's numeric re-set-up (the aggregation of the full set-up is kept, every numeric
quantity is recomputed from the new values; Sec. 3.2 on reusing the symbolic phase across
nonlinear iterations):
  * with the old values it reproduces the full set-up bit for bit;
  * when the new values leave every strength decision and aggregate unchanged, it equals a fresh
    full set-up on the new values bit for bit (the defining property of the reading);
  * when they do not, the aggregates stay the old ones and the level-0 prolongator and coarse
    operator equal the smoothing formula and a dense R A P built from the new values;
  * the updated solver still solves the new system."""
import numpy as np

import battery_system as bs
import oracle
from battery_system import spec


def _system():
    return bs.assemble(grid=bs.Grid(3, 10, 9, 8), seed=3)


def _perturb_diag(system, rel, seed, rel_phi_s=None):
    """New values: every diagonal block's diagonal entries grow by a random factor in [0, rel]
    (phi_s: [0, rel_phi_s] when given); off-diagonal entries unchanged; couplings scaled by 0.75."""
    u = bs.rng_uniform(seed, 9, np.arange(sum(B.nnz for B in system.blocks.values()), dtype=np.uint64))
    new, q = {}, 0
    for key in sorted(system.blocks):
        B = system.blocks[key]
        v = B.val.copy()
        if key[0] == key[1]:
            rows = np.repeat(np.arange(B.nrows), np.diff(B.rowptr))
            d = B.col == rows
            g = rel_phi_s if (rel_phi_s is not None and key[0] == spec.PHI_S) else rel
            v[d] = v[d] * (1.0 + g * u[q:q + B.nnz][d])
        else:
            v = v * 0.75
        q += B.nnz
        new[key] = v
    return new


def _blocks(system, vals=None):
    F = 5
    out = [[None] * F for _ in range(F)]
    for (r, c), B in system.blocks.items():
        out[r][c] = oracle.CSR(B.rowptr, B.col, B.val if vals is None else vals[(r, c)], B.nrows, B.ncols)
    return out


def _nested(vals):
    out = [[None] * 5 for _ in range(5)]
    for (r, c), v in vals.items():
        out[r][c] = v
    return out


def _hier_equal(a, b):
    assert a.nlevels == b.nlevels
    for l in range(a.nlevels):
        A1, A2 = a.level_matrix(l), b.level_matrix(l)
        assert np.array_equal(A1.rowptr, A2.rowptr) and np.array_equal(A1.col, A2.col)
        assert np.array_equal(A1.val, A2.val)
        if l + 1 < a.nlevels:
            for f in ("prolongator", "restriction"):
                M1, M2 = getattr(a, f)(l), getattr(b, f)(l)
                assert np.array_equal(M1.rowptr, M2.rowptr) and np.array_equal(M1.col, M2.col)
                assert np.array_equal(M1.val, M2.val)
            assert np.array_equal(a.aggregates(l), b.aggregates(l))
            assert a.omega(l) == b.omega(l)
            assert np.array_equal(a.dinv(l), b.dinv(l))
            assert a.cheb_bounds(l) == b.cheb_bounds(l)


ORDER = list(spec.WORKLOAD_ORDER)


def test_update_with_same_values_is_identity():
    system = _system()
    o = oracle.BGS(_blocks(system), system.field_sizes, ORDER)
    ref = oracle.BGS(_blocks(system), system.field_sizes, ORDER)
    assert o.setup() == 0 and ref.setup() == 0
    assert o.update_values(_nested({k: B.val for k, B in system.blocks.items()})) == 0
    for k in range(5):
        _hier_equal(o.amg(k), ref.amg(k))


def test_update_equals_fresh_setup_when_decisions_unchanged():
    system = _system()
    opts = oracle.default_options(max_coarse=60)
    vals = _perturb_diag(system, 1e-3, seed=17)     # small enough that no decision flips
    o = oracle.BGS(_blocks(system), system.field_sizes, ORDER, opts)
    fresh = oracle.BGS(_blocks(system, vals), system.field_sizes, ORDER, opts)
    assert o.setup() == 0 and fresh.setup() == 0
    old = [[o.amg(k).aggregates(l) for l in range(o.amg(k).nlevels - 1)] for k in range(5)]
    old_strong = [[o.amg(k).strong(l) for l in range(o.amg(k).nlevels - 1)] for k in range(5)]
    # hypothesis of the property: the fresh set-up makes the same decisions on every level
    for k in range(5):
        h = fresh.amg(k)
        assert h.nlevels == o.amg(k).nlevels
        for l in range(h.nlevels - 1):
            assert np.array_equal(h.strong(l), old_strong[k][l])
            assert np.array_equal(h.aggregates(l), old[k][l])
    assert any(o.amg(k).nlevels > 2 for k in range(5))
    assert o.update_values(_nested(vals)) == 0
    for k in range(5):
        _hier_equal(o.amg(k), fresh.amg(k))
    b = system.b
    x1, i1 = o.solve(b)
    x2, i2 = fresh.solve(b)
    assert i1.converged and np.array_equal(x1, x2)


def test_update_keeps_aggregates_and_recomputes_numerics():
    system = _system()
    # a large change on phi_s: strong connections weaken relative to the diagonal
    vals = _perturb_diag(system, 0.8, seed=23, rel_phi_s=100.0)
    o = oracle.BGS(_blocks(system), system.field_sizes, ORDER)
    assert o.setup() == 0
    k = spec.PHI_S
    h = o.amg(k)
    agg0, nagg0, strong0 = h.aggregates(0), h.nagg(0), h.strong(0)
    P_old = h.prolongator(0)
    assert o.update_values(_nested(vals)) == 0
    h = o.amg(k)
    assert np.array_equal(h.aggregates(0), agg0)
    fresh_flags = oracle.strength_flags(oracle.CSR(system.blocks[(k, k)].rowptr, system.blocks[(k, k)].col,
                                                   vals[(k, k)], system.ncells, system.ncells),
                                        oracle.default_options().theta[k])
    assert not np.array_equal(fresh_flags, strong0)      # a fresh set-up would decide differently
    # level-0 prolongator from the smoothing formula with the kept flags and the new values
    B = system.blocks[(k, k)]
    A = oracle.CSR(B.rowptr, B.col, vals[(k, k)], B.nrows, B.ncols)
    vF, dF = oracle.filter_matrix(A, strong0, 1)
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    mask = (A.col == rows) | (strong0 == 1)
    rp = np.zeros(A.nrows + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows[mask], minlength=A.nrows), out=rp[1:])
    AF = oracle.CSR(rp, A.col[mask], vF[mask], A.nrows, A.ncols)
    AFd = AF.to_dense()
    lam = oracle.power_lambda(AF, 1.0 / dF, 10)
    omega = (4.0 / 3.0) / lam
    assert h.omega(0) == omega
    Pt = np.zeros((A.nrows, nagg0))
    Pt[np.arange(A.nrows), agg0] = 1.0
    Pd = Pt - omega * (AFd / dF[:, None]) @ Pt
    P = h.prolongator(0)
    assert np.array_equal(P.rowptr, P_old.rowptr) and np.array_equal(P.col, P_old.col)
    assert np.abs(P.to_dense() - Pd).max() <= 1e-14
    assert np.abs(P.val - P_old.val).max() > 1e-3        # the values did change
    # coarse operator: dense Galerkin product with the new level-0 values
    Ac = Pd.T @ A.to_dense() @ Pd
    assert np.abs(h.level_matrix(1).to_dense() - Ac).max() <= 1e-13 * np.abs(Ac).max()
    # the updated solver solves the new system; the full operator carries the new values
    new_sys = {key: vals[key] for key in vals}
    x, info = o.solve(system.b)
    assert info.converged

    def matvec(xv):
        y = np.zeros(system.ndof)
        n = system.ncells
        for (r, c), Bk in system.blocks.items():
            M = oracle.CSR(Bk.rowptr, Bk.col, new_sys[(r, c)], Bk.nrows, Bk.ncols)
            y[r * n:(r + 1) * n] += oracle.spmv(M, xv[c * n:(c + 1) * n])
        return y

    r = system.b - matvec(x)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(system.b)
    assert np.abs(o.full_matvec(x) - matvec(x)).max() <= 1e-12 * np.abs(matvec(x)).max()
