"""Pins of the oracle's building blocks against closed forms, dense linear algebra,
published test values and brute force (no GPU)."""
import itertools
import math
import os

import numpy as np
import pytest

import battery_system as bs
import oracle
from battery_system import spec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hash_vectors.txt")


def rand_csr(n, m, density, rng, diag=False):
    d = (rng.random((n, m)) < density) * rng.standard_normal((n, m))
    if diag:
        np.fill_diagonal(d, np.abs(d).sum(axis=1) + 1.0)
    return dense_to_csr(d), d


def dense_to_csr(d, keep=None):
    mask = d != 0 if keep is None else keep
    rows, cols = np.nonzero(mask)
    rp = np.zeros(d.shape[0] + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows, minlength=d.shape[0]), out=rp[1:])
    return oracle.CSR(rp, cols.astype(np.int32), d[rows, cols], d.shape[0], d.shape[1])


def laplacian_2d(n, neumann=True, shift=0.0):
    g = bs.Grid(2, n, n, 1)
    c = np.ones(g.ncells)
    blk = bs._stencil_block(g, [c, c, c], [np.full(g.ncells, shift)] if shift else None).to_csr()
    return oracle.CSR(blk.rowptr, blk.col, blk.val, blk.nrows, blk.ncols)


def test_fmix32_published_values():
    for line in open(GOLDEN):
        if line.startswith("fmix32"):
            _, a, b = line.split()
            assert oracle.fmix32(int(a, 0)) == int(b, 0)


def test_fmix32_is_a_bijection_on_a_sample():
    xs = list(range(0, 1 << 16)) + [0xFFFFFFFF - i for i in range(1000)]
    hs = {oracle.fmix32(x) for x in xs}
    assert len(hs) == len(set(xs))


def test_spmv_transpose_spgemm_against_dense():
    rng = np.random.default_rng(0)
    A, Ad = rand_csr(37, 23, 0.2, rng)
    B, Bd = rand_csr(23, 41, 0.15, rng)
    x = rng.standard_normal(23)
    assert np.allclose(oracle.spmv(A, x), Ad @ x, rtol=0, atol=1e-13)
    T = oracle.transpose(A)
    assert np.array_equal(T.to_dense(), Ad.T)
    assert all(np.all(np.diff(T.col[T.rowptr[i]:T.rowptr[i + 1]]) > 0) for i in range(T.nrows))
    Cm = oracle.spgemm(A, B)
    ref = Ad @ Bd
    assert np.abs(Cm.to_dense() - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
    # pattern = structural product pattern (numerical zeros kept)
    struct = ((Ad != 0).astype(int) @ (Bd != 0).astype(int)) > 0
    assert Cm.nnz == struct.sum()
    for i in range(Cm.nrows):
        cols = Cm.col[Cm.rowptr[i]:Cm.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
        assert set(cols) == set(np.nonzero(struct[i])[0])


def test_strength_symmetric_test_and_graph():
    rng = np.random.default_rng(1)
    n = 30
    d = np.zeros((n, n))
    for i in range(n):
        d[i, i] = 4.0 + rng.random()
        for j in rng.choice(n, 4, replace=False):
            if j != i:
                d[i, j] = rng.standard_normal() * (10.0 ** rng.integers(-3, 1))
    A = dense_to_csr(d)
    theta = 0.1
    s = oracle.strength_flags(A, theta)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    for e in range(A.nnz):
        i, j = rows[e], A.col[e]
        if i == j:
            assert s[e] == 0
            continue
        thr = theta * theta * abs(d[i, i] * d[j, j])
        assert s[e] == int(d[i, j] ** 2 > thr or d[j, i] ** 2 > thr)
    S = oracle.strength_graph(A, s)
    Sd = S.to_dense() != 0
    # the graph is the symmetrised strong pattern, without the diagonal
    strong = np.zeros((n, n), dtype=bool)
    strong[rows[s == 1], A.col[s == 1]] = True
    want = strong | strong.T
    pat = np.zeros((n, n), dtype=bool)
    pat[np.repeat(np.arange(n), np.diff(S.rowptr)), S.col] = True
    assert np.array_equal(pat, want)
    # values carry a_ij, or 0 where only a_ji is stored
    srows = np.repeat(np.arange(n), np.diff(S.rowptr))
    assert np.array_equal(S.val, d[srows, S.col])
    del Sd


def _graph(edges, n):
    d = np.zeros((n, n))
    for a, b in edges:
        d[a, b] = d[b, a] = 1.0
    keep = d != 0
    return dense_to_csr(d, keep)


def _dist2(S):
    n = S.nrows
    adj = np.zeros((n, n), dtype=bool)
    adj[np.repeat(np.arange(n), np.diff(S.rowptr)), S.col] = True
    a1 = adj | np.eye(n, dtype=bool)
    a2 = (a1.astype(int) @ a1.astype(int)) > 0
    return a2


def _replay_rounds(S, salt):
    """The round rule applied naively over the dense distance-2 relation."""
    n = S.nrows
    a2 = _dist2(S)
    key = [(oracle.fmix32(i ^ salt), i) for i in range(n)]
    st = [0] * n
    while 0 in st:
        new = [v for v in range(n) if st[v] == 0 and all(key[v] > key[u] for u in range(n)
                                                        if u != v and st[u] == 0 and a2[v, u])]
        for v in new:
            st[v] = 1
        for v in range(n):
            if st[v] == 0 and any(st[u] == 1 and a2[v, u] for u in range(n)):
                st[v] = 2
    return st


def _graphs():
    out = []
    out.append(("path7", _graph([(i, i + 1) for i in range(6)], 7)))
    grid = [(i * 5 + j, i * 5 + j + 1) for i in range(5) for j in range(4)] + \
           [(i * 5 + j, (i + 1) * 5 + j) for i in range(4) for j in range(5)]
    out.append(("grid5x5", _graph(grid, 25)))
    rng = np.random.default_rng(5)
    for t in range(6):
        n = int(rng.integers(2, 13))
        edges = [(a, b) for a, b in itertools.combinations(range(n), 2) if rng.random() < 0.3]
        out.append((f"rand{t}", _graph(edges, n)))
    out.append(("isolated", _graph([(0, 1)], 4)))
    return out


@pytest.mark.parametrize("salt", [0, oracle.mis_salt(1), oracle.mis_salt(3)])
def test_mis2_by_definition_and_replay(salt):
    for name, S in _graphs():
        st, rounds = oracle.mis2(S, salt)
        assert rounds >= 1
        a2 = _dist2(S)
        roots = np.nonzero(st == 1)[0]
        assert set(np.unique(st)) <= {1, 2}
        # independent at distance 2
        for a, b in itertools.combinations(roots, 2):
            assert not a2[a, b], name
        # maximal: every other node within distance 2 of a root
        for v in np.nonzero(st == 2)[0]:
            assert a2[v, roots].any(), name
        assert list(st) == _replay_rounds(S, salt), name


def test_aggregation_rules():
    for name, S in _graphs():
        st, _ = oracle.mis2(S, 0)
        agg, nagg = oracle.aggregate(S, st)
        assert nagg == int((st == 1).sum())
        roots = np.nonzero(st == 1)[0]
        # ids = roots ranked by node index
        assert list(agg[roots]) == list(range(nagg))
        assert agg.min() >= 0 and agg.max() < nagg
        n = S.nrows
        adj = np.zeros((n, n), dtype=bool)
        adj[np.repeat(np.arange(n), np.diff(S.rowptr)), S.col] = True
        phase1 = set(roots)
        for r in roots:
            for u in np.nonzero(adj[r])[0]:
                assert agg[u] == agg[r]
                phase1.add(u)
        for v in range(n):
            if v not in phase1:
                # phase 2: joins an aggregate of a phase-1 neighbour (all weights equal: smallest id)
                cand = [agg[u] for u in np.nonzero(adj[v])[0] if u in phase1]
                assert cand and agg[v] == min(cand), name


def test_tentative_prolongator_preserves_constants():
    A = laplacian_2d(9)
    s = oracle.strength_flags(A, 0.0)
    S = oracle.strength_graph(A, s)
    st, _ = oracle.mis2(S, 0)
    agg, nagg = oracle.aggregate(S, st)
    vF, dF = oracle.filter_matrix(A, s, 1)
    Pt = oracle.smooth_prolongator(oracle.CSR(A.rowptr, A.col, vF, A.nrows, A.ncols), 1.0 / dF, agg, nagg, 0.0)
    ones = np.ones(nagg)
    assert np.array_equal(oracle.spmv(Pt, ones), np.ones(A.nrows))
    D = Pt.to_dense()
    assert np.array_equal((D == 1.0).sum(axis=1), np.ones(A.nrows))
    assert np.array_equal(D[np.arange(A.nrows), agg], np.ones(A.nrows))


def test_smoothed_prolongator_interpolates_constants_on_zero_row_sum():
    A = laplacian_2d(12)          # pure Neumann: every row sums to zero
    for theta in (0.0, 0.2):
        s = oracle.strength_flags(A, theta)
        S = oracle.strength_graph(A, s)
        st, _ = oracle.mis2(S, 0)
        agg, nagg = oracle.aggregate(S, st)
        vF, dF = oracle.filter_matrix(A, s, 1)
        AF = oracle.CSR(A.rowptr, A.col, vF, A.nrows, A.ncols)
        # lumping keeps zero row sums
        assert np.abs(oracle.spmv(AF, np.ones(A.nrows))).max() < 1e-14
        lam = oracle.power_lambda(AF, 1.0 / dF, 10)
        assert 0 < lam <= 1.0 + 1e-12        # ||D_F^-1 A_F||_inf <= 1 for the row-sum diagonal
        P = oracle.smooth_prolongator(AF, 1.0 / dF, agg, nagg, (4.0 / 3.0) / lam)
        assert np.abs(oracle.spmv(P, np.ones(nagg)) - 1.0).max() < 1e-14
        # P = P_tent - omega D_F^-1 A_F P_tent, densely
        Pt = np.zeros((A.nrows, nagg))
        Pt[np.arange(A.nrows), agg] = 1.0
        ref = Pt - ((4.0 / 3.0) / lam) * (np.diag(1.0 / dF) @ AF.to_dense() @ Pt)
        assert np.abs(P.to_dense() - ref).max() < 1e-14


def test_filter_lumps_dropped_entries():
    rng = np.random.default_rng(3)
    A, d = rand_csr(25, 25, 0.2, rng, diag=True)
    s = oracle.strength_flags(A, 0.25)
    vF, dF = oracle.filter_matrix(A, s, 1)
    rows = np.repeat(np.arange(25), np.diff(A.rowptr))
    AFd = np.zeros_like(d)
    AFd[rows, A.col] = vF
    assert np.allclose(AFd.sum(axis=1), d.sum(axis=1), rtol=0, atol=1e-12)
    assert np.allclose(dF, np.abs(AFd).sum(axis=1), rtol=0, atol=1e-12)
    _, dF0 = oracle.filter_matrix(A, s, 0)
    assert np.array_equal(dF0, np.diag(AFd))


def test_galerkin_rap_against_dense():
    A = laplacian_2d(10, shift=0.3)
    amg = oracle.AMG(A, theta=0.0, degree=2, opts=oracle.default_options(max_coarse=10))
    assert amg.nlevels >= 3
    for l in range(amg.nlevels - 1):
        Al = amg.level_matrix(l).to_dense()
        P = amg.prolongator(l).to_dense()
        R = amg.restriction(l).to_dense()
        assert np.array_equal(R, P.T)
        Ac = amg.level_matrix(l + 1).to_dense()
        ref = P.T @ Al @ P
        assert np.abs(Ac - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.abs(Ac - Ac.T).max() <= 1e-13 * np.abs(ref).max()   # symmetric A -> symmetric A_c


def _cheb_T(k, t):
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1
    out[inside] = np.cos(k * np.arccos(t[inside]))
    ts = t[~inside]
    out[~inside] = np.sign(ts) ** k * np.cosh(k * np.arccosh(np.abs(ts)))
    return out


@pytest.mark.parametrize("deg", [1, 2, 3, 4, 6])
def test_chebyshev_closed_form_on_diagonal(deg):
    lam = np.linspace(0.05, 2.0, 40)
    A = dense_to_csr(np.diag(lam))
    dinv = np.ones(40)
    lmax, lmin = 2.2, 2.2 / 30
    xt = np.random.default_rng(deg).standard_normal(40)
    b = lam * xt
    x = oracle.chebyshev(A, dinv, lmin, lmax, deg, b)
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    factor = _cheb_T(deg, (theta - lam) / delta) / _cheb_T(deg, np.array([theta / delta]))[0]
    assert np.abs((xt - x) - factor * xt).max() <= 1e-12 * np.abs(xt).max()
    # from a non-zero start the same polynomial acts on the initial error
    x0 = np.random.default_rng(9).standard_normal(40)
    x1 = oracle.chebyshev(A, dinv, lmin, lmax, deg, b, x0)
    assert np.abs((xt - x1) - factor * (xt - x0)).max() <= 1e-12 * np.abs(xt - x0).max()


def test_power_iteration_estimates_lambda_max():
    lam = np.concatenate([np.linspace(0.1, 1.0, 50), [3.0]])
    A = dense_to_csr(np.diag(lam))
    est = oracle.power_lambda(A, np.ones(51), 10)
    assert abs(est - 3.0) < 1e-3
    Lp = laplacian_2d(8, shift=0.5)
    D = Lp.to_dense()
    dinv = 1.0 / np.diag(D)
    M = np.diag(np.sqrt(dinv)) @ D @ np.diag(np.sqrt(dinv))
    ev = np.linalg.eigvalsh(M).max()
    est = oracle.power_lambda(Lp, dinv, 200)
    assert abs(est - ev) < 5e-3 * ev


def test_dense_lu_partial_pivoting():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((30, 30))
    a[0, 0] = 0.0           # forces a pivot
    lu, piv, st = oracle.lu_factor(a)
    assert st == 0
    L = np.tril(lu, -1) + np.eye(30)
    U = np.triu(lu)
    pa = a.copy()
    for k, p in enumerate(piv):
        pa[[k, p]] = pa[[p, k]]
    assert np.abs(L @ U - pa).max() < 1e-12
    b = rng.standard_normal(30)
    x = oracle.lu_solve(lu, piv, b)
    assert np.abs(a @ x - b).max() < 1e-11
    sing = np.ones((4, 4))
    assert oracle.lu_factor(sing)[2] == 6


def test_vcycle_symmetric_for_spd():
    A = laplacian_2d(16, shift=0.01)
    amg = oracle.AMG(A, theta=0.0, degree=2, opts=oracle.default_options(max_coarse=20))
    assert amg.nlevels >= 3
    rng = np.random.default_rng(6)
    y, z = rng.standard_normal(A.nrows), rng.standard_normal(A.nrows)
    lhs, rhs = y @ amg.vcycle(z), z @ amg.vcycle(y)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _vcycle_factor(dim, N, deg, max_coarse=300):
    A0, _, _ = bs.poisson_dirichlet(dim, N)
    A = oracle.CSR(A0.rowptr, A0.col, A0.val, A0.nrows, A0.ncols)
    amg = oracle.AMG(A, theta=0.0, degree=deg, opts=oracle.default_options(max_coarse=max_coarse))
    rng = np.random.default_rng(7)
    xt = rng.standard_normal(A.nrows)
    b = oracle.spmv(A, xt)
    x = np.zeros(A.nrows)
    errs = []
    for _ in range(12):
        x = x + amg.vcycle(b - oracle.spmv(A, x))
        e = x - xt
        errs.append(math.sqrt(e @ oracle.spmv(A, e)))     # energy norm
    return (errs[-1] / errs[4]) ** (1 / 7), amg.nlevels


def test_vcycle_convergence_factor_poisson():
    """Stationary V-cycle on Dirichlet Poisson: bounded, mesh-independent energy-norm factor."""
    r4, _ = _vcycle_factor(2, 64, 4)
    assert r4 < 0.3, r4
    r2a, _ = _vcycle_factor(2, 32, 2)
    r2b, nl = _vcycle_factor(2, 64, 2)
    assert nl >= 3
    assert r2a < 0.65 and r2b < 0.65
    assert abs(r2a - r2b) < 0.05         # independent of h
    r3, _ = _vcycle_factor(3, 16, 4)
    assert r3 < 0.3


def weak_laplacian(n, eps=1e-3):
    """2D 5-point pattern whose off-diagonals are all weak at theta = 0.04 (diagonally dominant)."""
    A = laplacian_2d(n)
    d = A.to_dense()
    off = d - np.diag(np.diag(d))
    d = eps * off + np.diag(np.full(n * n, 4.0))
    return dense_to_csr(d)


def test_stalled_coarsening_is_retried_without_dropping():
    A = weak_laplacian(12)
    # theta = 0.04: every node isolated -> singleton aggregates, coarsening stalls
    s = oracle.strength_flags(A, 0.04)
    assert s.sum() == 0
    amg = oracle.AMG(A, theta=0.04, degree=2, opts=oracle.default_options(max_coarse=10))
    assert amg.nlevels >= 2
    assert amg.nagg(0) < 0.5 * A.nrows                  # aggregated as with theta = 0
    ref = oracle.AMG(A, theta=0.0, degree=2, opts=oracle.default_options(max_coarse=10))
    assert np.array_equal(amg.aggregates(0), ref.aggregates(0))


def test_zero_filtered_rows_keep_the_tentative_prolongator():
    """theta = 0.08 on the 24^3 phi_s block: some level-1 rows have every connection weak and a zero
    row sum, so their lumped filtered row is zero (D_F = 0).  Such a row takes no part in the
    smoothing: its row of P is its P_tent row, omega stays finite, and the solve converges."""
    s = bs.assemble(grid=bs.Grid(3, 24, 24, 24), seed=1)
    B = s.blocks[(0, 0)]
    opts = oracle.default_options(max_coarse=100)
    opts.theta[0] = 0.08
    h = oracle.AMG(oracle.CSR(B.rowptr, B.col, B.val, B.nrows, B.ncols), theta=0.08, degree=4, opts=opts)
    assert h.status == 0 and h.nlevels >= 3
    zero_rows = 0
    for l in range(h.nlevels - 1):
        assert np.isfinite(h.omega(l))
        A = h.level_matrix(l)
        strong = h.strong(l)
        vF, dF = oracle.filter_matrix(A, strong, 1)
        P = h.prolongator(l)
        agg = h.aggregates(l)
        for i in np.flatnonzero(dF == 0.0):
            zero_rows += 1
            row = slice(P.rowptr[i], P.rowptr[i + 1])
            assert list(P.col[row]) == [agg[i]] and list(P.val[row]) == [1.0]
    assert zero_rows > 0
    x = h.vcycle(s.b[:s.ncells])
    assert np.isfinite(x).all()
    o = oracle.BGS([[oracle.CSR(B.rowptr, B.col, B.val, B.nrows, B.ncols)]], [s.ncells], [0], opts)
    assert o.setup() == 0
    xs, info = o.solve(s.b[:s.ncells])
    assert info.converged


def test_theta_grid_phi_s_always_solves():
    """The drop-tolerance grid of Sec. 3.1.4 (theta = 0 ... 0.64, doubling) on a phi_s block: every
    set-up succeeds with finite smoothing weights and FGMRES(30) with one V-cycle converges.  Large
    theta drops every coupling on some levels; the stall retry and the zero-row rule keep the
    hierarchy usable."""
    s = bs.assemble(grid=bs.Grid(3, 14, 13, 12), seed=1)
    B = s.blocks[(0, 0)]
    A = oracle.CSR(B.rowptr, B.col, B.val, B.nrows, B.ncols)
    iters = {}
    for th in (0.0, 0.01, 0.02, 0.04, 0.08, 0.16, 0.32, 0.64):
        opts = oracle.default_options(restart=30, max_coarse=60)
        opts.theta[0] = th
        o = oracle.BGS([[A]], [s.ncells], [0], opts)
        assert o.setup() == 0, th
        h = o.amg(0)
        assert all(np.isfinite(h.omega(l)) for l in range(h.nlevels - 1)), th
        x, info = o.solve(s.b[:s.ncells])
        assert info.converged, th
        iters[th] = info.iters
    assert max(iters.values()) <= 3 * min(iters.values())


def _cheb_T(k, w):
    t0, t1 = np.ones_like(w), w
    if k == 0:
        return t0
    for _ in range(k - 1):
        t0, t1 = t1, 2 * w * t1 - t0
    return t1


def test_skew_radius_and_ellipse_chebyshev_closed_form():
    """Nonsymmetric Chebyshev on an ellipse (Sec. 2.2.1, Manteuffel): on a normal matrix made of
    2x2 rotation-scaling blocks [[a, -g], [g, a]] (eigenvalues of D^-1 A: 1 +- i g/a) the Bendixson
    radius is max g/a exactly, and one smoother application from x = 0 multiplies each block's error
    by |T_k((theta - z)/c) / T_k(theta/c)|, z = 1 + i g/a, for theta and c^2 = A^2 - B^2 of either
    sign (an ellipse wider or taller than its real extent)."""
    rng = np.random.default_rng(9)
    m = 40
    a = rng.uniform(1.0, 3.0, m)
    t = np.sort(rng.uniform(0.05, 0.6, m))
    t[-1] = 0.8                               # a separated largest rate: the power iteration converges
    g = a * t
    rp, ci, vals = [0], [], []
    for j in range(m):
        for r, row in ((0, [(0, a[j]), (1, -g[j])]), (1, [(0, g[j]), (1, a[j])])):
            for c, v in row:
                ci.append(2 * j + c)
                vals.append(v)
            rp.append(len(ci))
    n = 2 * m
    A = oracle.CSR(np.array(rp), np.array(ci), np.array(vals), n, n)
    rad = oracle.skew_radius(A, 60)
    assert abs(rad - t.max()) <= 1e-12 * t.max()
    dinv = np.repeat(1.0 / a, 2)
    xs = rng.standard_normal(n)
    b = oracle.spmv(A, xs)
    for theta, c2, deg in ((1.0, 0.3 ** 2 - 0.5 ** 2, 4), (1.1, 0.6 ** 2 - 0.2 ** 2, 3), (0.9, -0.04, 2)):
        x = oracle.chebyshev_ellipse(A, dinv, theta, c2, deg, b)
        e = (xs - x).reshape(m, 2)
        c = np.sqrt(complex(c2))
        z = 1.0 + 1j * t
        fac = np.abs(_cheb_T(deg, (theta - z) / c) / _cheb_T(deg, theta / c + 0j))
        assert np.allclose(np.linalg.norm(e, axis=1), fac * np.linalg.norm(xs.reshape(m, 2), axis=1),
                           rtol=1e-10, atol=1e-14)
    # a symmetric block: no imaginary extent, and the ellipse option leaves the hierarchy as it was
    s = bs.assemble(grid=bs.Grid(3, 8, 7, 6), seed=2)
    B = s.blocks[(spec.PRESS, spec.PRESS)]
    Ap = oracle.CSR(B.rowptr, B.col, B.val, B.nrows, B.ncols)
    assert np.array_equal(Ap.to_dense(), Ap.to_dense().T)
    assert oracle.skew_radius(Ap) == 0.0


def test_ellipse_smoother_on_advective_species_blocks():
    """With the ellipse option the species blocks (upwind advection) get an imaginary extent on their
    levels, the symmetric blocks keep theirs at 0, and the block sweep still solves."""
    s = bs.assemble(grid=bs.Grid(3, 10, 9, 8), seed=4)
    base = oracle.bgs_for_system(s, order=list(spec.WORKLOAD_ORDER), opts=oracle.default_options(max_coarse=40))
    ell = oracle.bgs_for_system(s, order=list(spec.WORKLOAD_ORDER),
                                opts=oracle.default_options(max_coarse=40, cheb_ellipse=1))
    for k in (spec.C1, spec.C2):
        h = ell.amg(k)
        assert all(h.cheb_imag(l) > 0.0 for l in range(h.nlevels - 1))
    h = ell.amg(spec.PRESS)
    assert all(h.cheb_imag(l) == 0.0 for l in range(h.nlevels - 1))
    v = np.random.default_rng(1).standard_normal(s.ncells)
    assert np.array_equal(ell.amg(spec.PRESS).vcycle(v), base.amg(spec.PRESS).vcycle(v))
    x, info = ell.solve(s.b)
    assert info.converged and np.linalg.norm(s.b - s.matvec(x)) <= 1e-8 * np.linalg.norm(s.b)
    lam, ia = ell.solve_adjoint(s.b)
    assert ia.converged


def _scaled_chebyshev(A, dinv, inv_theta, alpha, scale, b, x0):
    """The Chebyshev smoothing pass in the scaled form the CUDA kernels carry (e = d / c2 of the
    step: first step e = D^-1 r, x += e / theta; step k: e = alpha_k e + D^-1 r, x += scale_k e)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    e = dinv * (b - A @ x)
    x = x + inv_theta * e
    for a, c in zip(alpha, scale):
        e = a * e + dinv * (b - A @ x)
        x = x + c * e
    return x


def _scaled_coefs(theta, delta, c2e, deg, ellipse):
    """alpha_k = c1 c2_prev / c2 and scale_k = c2 from the recurrence coefficients of the interval
    (Saad's rho form) or of the ellipse (tau form)."""
    inv_theta = 1.0 / theta
    st, sc = (inv_theta if ellipse else delta / theta), inv_theta
    alpha, scale = [], []
    for _ in range(1, deg):
        if ellipse:
            tn = 1.0 / (2.0 * theta - c2e * st)
            c1, c2, st = c2e * tn * st, 2.0 * tn, tn
        else:
            rn = 1.0 / (2.0 * theta / delta - st)
            c1, c2, st = rn * st, 2.0 * rn / delta, rn
        alpha.append(c1 * sc / c2)
        scale.append(c2)
        sc = c2
    return inv_theta, alpha, scale


@pytest.mark.parametrize("deg", [1, 2, 4, 7])
@pytest.mark.parametrize("start", ["zero", "given"])
def test_scaled_chebyshev_recurrence_equals_the_oracle(deg, start):
    """Carrying e = d / c2 instead of d (two fewer FP64 operations per row in the kernels) gives the
    oracle's iterates on the interval and on the ellipse, from x = 0 and from a given x."""
    rng = np.random.default_rng(deg)
    n = 40
    D = np.diag(4.0 + rng.uniform(0, 1, n))
    for i in range(n - 1):
        D[i, i + 1] = -rng.uniform(0.2, 1.2)
        D[i + 1, i] = -rng.uniform(0.2, 1.2)
    D[0, 5], D[7, 2] = 0.3, -0.4                     # nonsymmetric
    rp, ci, v = [0], [], []
    for i in range(n):
        nz = np.nonzero(D[i])[0]
        ci += nz.tolist()
        v += D[i, nz].tolist()
        rp.append(len(ci))
    A = oracle.CSR(np.array(rp), np.array(ci), np.array(v), n, n)
    dinv = 1.0 / np.diag(D)
    b = rng.standard_normal(n)
    x0 = None if start == "zero" else rng.standard_normal(n)
    lmax, lmin = 1.9, 1.9 / 30.0
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    ref = oracle.chebyshev(A, dinv, lmin, lmax, deg, b, x0)
    got = _scaled_chebyshev(D, dinv, *_scaled_coefs(theta, delta, 0.0, deg, False), b, x0)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    for c2e in (0.5 * delta ** 2, -0.3 * delta ** 2):   # real and imaginary focal parameter
        ref = oracle.chebyshev_ellipse(A, dinv, theta, c2e, deg, b, x0)
        got = _scaled_chebyshev(D, dinv, *_scaled_coefs(theta, delta, c2e, deg, True), b, x0)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _fmix32_np(h):
    h = np.uint32(h)
    h ^= h >> np.uint32(16)
    h = np.uint32((int(h) * 0x85EBCA6B) & 0xFFFFFFFF)
    h ^= h >> np.uint32(13)
    h = np.uint32((int(h) * 0xC2B2AE35) & 0xFFFFFFFF)
    h ^= h >> np.uint32(16)
    return int(h)


def _power_unnormalised(D, dinv, iters):
    """The CUDA form of the power iteration: unnormalised iterates u_k = D^-1 A u_k-1 from the
    hashed start, rescaled to unit norm before every 8th step except the last, estimate
    ||u_k|| / ||u_k-1||."""
    n = D.shape[0]
    u = np.array([((_fmix32_np(i ^ 0x7F4A7C15) >> 8) + 0.5) / 16777216.0 for i in range(n)])
    prev = u
    for it in range(iters):
        if it > 0 and it % 8 == 0 and it < iters - 1:
            nu = np.linalg.norm(u)
            u = u / nu if nu > 0 else 0.0 * u   # a zero norm scales by 0, as the kernel's rsqrt does
        prev, u = u, dinv * (D @ u)
    b = prev @ prev
    return float(np.sqrt((u @ u) / b)) if b > 0 else 0.0


@pytest.mark.parametrize("iters", [1, 2, 8, 9, 10, 17, 40])
def test_unnormalised_power_iteration_equals_the_oracle(iters):
    """||u_k|| / ||u_k-1|| on the unnormalised iterates (what the kernels compute, with a rescale
    every 8 steps) equals the oracle's normalised estimate ||D^-1 A v||, v = u_k-1 / ||u_k-1||."""
    assert _fmix32_np(0) == oracle.fmix32(0) and _fmix32_np(12345) == oracle.fmix32(12345)
    Lp = laplacian_2d(7, shift=0.3)
    D = Lp.to_dense()
    D[3, 10] -= 0.2                                   # nonsymmetric
    A = dense_to_csr(D)
    dinv = 1.0 / np.diag(D)
    ref = oracle.power_lambda(A, dinv, iters)
    got = _power_unnormalised(D, dinv, iters)
    assert abs(got - ref) <= 1e-13 * ref
    zero = dense_to_csr(np.zeros((6, 6)) + np.diag(np.zeros(6)))
    assert oracle.power_lambda(zero, np.ones(6), iters) == 0.0
    assert _power_unnormalised(np.zeros((6, 6)), np.ones(6), iters) == 0.0
