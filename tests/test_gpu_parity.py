"""GPU parity tests: the CUDA path through the C ABI against the FP64 CPU oracle.

Integer results (strength decisions, MIS-2, aggregates) must match bit for bit; floating-point
results within tolerances derived from the arithmetic (documented per test)."""
import numpy as np
import pytest

import battery_system as bs
import oracle
from battery_system import spec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bgs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_13079_gb300 import _build
    _build.build()
    import paper_2602_13079_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def opts_kw(**kw):
    return kw


def make_pair(bgs, system, order=None, **kw):
    order = list(order if order is not None else spec.WORKLOAD_ORDER)
    s = bgs.solver_for_system(system, order=order, **kw)
    s.setup()
    o = oracle.bgs_for_system(system, order=order, opts=oracle.default_options(
        **{k: v for k, v in kw.items() if k not in ("precision", "graph", "autotune")}))
    return s, o


# ------------------------------------------------------------------------------------- SpMV
@pytest.mark.parametrize("lanes", [0, 1, 2, 4, 8, 16, 32])
def test_csr_spmv_matches_oracle(bgs, lanes):
    rng = np.random.default_rng(lanes)
    n = 20_011                                  # several blocks and a ragged tail
    lens = rng.integers(0, 40, n)
    lens[::97] = 0                               # empty rows
    lens[5] = 700                                # one long row
    rp = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(lens, out=rp[1:])
    col = np.concatenate([np.sort(rng.choice(n, l, replace=False)) for l in lens]).astype(np.int32)
    val = rng.standard_normal(rp[-1])
    x = rng.standard_normal(n)
    A = oracle.CSR(rp, col, val, n, n)
    ref = oracle.spmv(A, x)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = bgs.bgs_csr_spmv(n, rp[-1], dev(rp), dev(col), dev(val), dev(x), y, lanes)
    torch.cuda.synchronize()
    assert st == 0
    rows = np.repeat(np.arange(n), lens)
    scale = np.bincount(rows, weights=np.abs(val * x[col]), minlength=n)
    # FP64 sums of the same products in another order: |diff| <= len * eps * sum |a x|
    tol = 64 * np.finfo(float).eps * (lens + 1) * scale + 1e-300
    assert np.all(np.abs(y.cpu().numpy() - ref) <= tol)


@pytest.mark.parametrize("cnt", [1, 7, 16, 17, 50, 64])
def test_arnoldi_dots_match_fp64_dot_products(bgs, cnt):
    rng = np.random.default_rng(cnt)
    n = 100_003                                  # odd: exercises the tail row
    ld = n + 1
    V = rng.standard_normal((cnt, ld))
    w = rng.standard_normal(n)
    h = torch.zeros(cnt + 1, dtype=torch.float64, device="cuda")
    assert bgs.bgs_arnoldi_dots(dev(V), ld, cnt, dev(w), n, h) == 0
    torch.cuda.synchronize()
    ref = np.concatenate([V[:, :n] @ w, [w @ w]])
    # FP64 sums of n products in another order: |diff| <= n eps sum |v w|
    scale = np.concatenate([np.abs(V[:, :n]) @ np.abs(w), [w @ w]])
    assert np.all(np.abs(h.cpu().numpy() - ref) <= 4 * n * np.finfo(float).eps * scale)
    bad = torch.zeros(66, dtype=torch.float64, device="cuda")
    assert bgs.bgs_arnoldi_dots(dev(V), ld, 65, dev(w), n, bad) == bgs.INVALID_ARG
    assert bgs.bgs_arnoldi_dots(dev(V), n, cnt, dev(w), n, h) == bgs.INVALID_ARG   # odd leading dimension


def test_full_operator_spmv(bgs):
    s = bs.assemble("C1")
    g, o = bgs.solver_for_system(s), oracle.bgs_for_system(s, setup=False)
    x = np.random.default_rng(1).standard_normal(s.ndof)
    y = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    g.bgs_full_spmv(dev(x), y)
    ref = o.full_matvec(x)
    assert np.allclose(y.cpu().numpy(), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


# ------------------------------------------------------------------------------------- setup
SETUP_CASES = [
    ("C1-mc100", lambda: bs.assemble("C1"), dict(max_coarse=100)),
    ("3D-17x13x11", lambda: bs.assemble(grid=bs.Grid(3, 17, 13, 11), seed=2), dict(max_coarse=60)),
    ("3D-24", lambda: bs.assemble(grid=bs.Grid(3, 24, 24, 24), seed=1), dict()),
    ("stack-8x8x40", lambda: bs.assemble(grid=bs.Grid(3, 8, 8, 40), stack=True, seed=3), dict(max_coarse=80)),
    # theta = 0.08 on phi_s: level-1 rows whose filtered entries lump to zero (D_F = 0)
    ("3D-24-theta0.08", lambda: bs.assemble(grid=bs.Grid(3, 24, 24, 24), seed=1),
     dict(max_coarse=100, theta=[0.08, 0, 0, 0, 0])),
]


@pytest.mark.parametrize("name,mk,kw", SETUP_CASES, ids=[c[0] for c in SETUP_CASES])
def test_hierarchy_parity(bgs, name, mk, kw):
    system = mk()
    g, o = make_pair(bgs, system, **kw)
    for k in range(5):
        oa = o.amg(k)
        nl = g.bgs_num_levels(k)
        assert nl == oa.nlevels, (k, nl, oa.sizes())
        for l in range(nl):
            info = g.bgs_level_info(k, l)
            assert info["rows"] == oa.sizes()[l]
            if l + 1 < nl:
                # integer decisions: bit-exact
                assert info["nagg"] == oa.nagg(l)
                assert info["mis_rounds"] == oa.mis_rounds(l)
                assert np.array_equal(g.bgs_level_aggregates(k, l), oa.aggregates(l)), (k, l)
                assert abs(info["omega"] - oa.omega(l)) <= 1e-12 * abs(oa.omega(l))
                lo, hi = oa.cheb_bounds(l)
                assert abs(info["lmax"] - hi) <= 1e-10 * hi and abs(info["lmin"] - lo) <= 1e-10 * lo
                for which, ref in ((1, oa.prolongator(l)), (2, oa.restriction(l))):
                    rp, ci, v = g.bgs_level_copy(k, l, which)
                    assert np.array_equal(rp, ref.rowptr) and np.array_equal(ci, ref.col)
                    assert np.abs(v - ref.val).max() <= 1e-12 * max(1.0, np.abs(ref.val).max())
            rp, ci, v = g.bgs_level_copy(k, l, 0)
            ref = oa.level_matrix(l)
            assert np.array_equal(rp, ref.rowptr) and np.array_equal(ci, ref.col), (k, l)
            assert np.abs(v - ref.val).max() <= 1e-11 * np.abs(ref.val).max(), (k, l)


def test_stalled_coarsening_retry_parity(bgs):
    """A block whose couplings are all weak at theta = 0.04: both sides retry the aggregation without
    dropping and must agree bit for bit."""
    n = 16
    g = bs.Grid(2, n, n, 1)
    c = np.ones(g.ncells)
    lap = bs._stencil_block(g, [c, c, c]).to_csr()
    val = np.where(np.repeat(np.arange(lap.nrows), np.diff(lap.rowptr)) == lap.col, 4.0, 1e-3 * lap.val)
    blk = bs.CSR(lap.rowptr, lap.col, val, lap.nrows, lap.ncols)

    class _O:
        pass
    o = _O()
    o.rowptr, o.col, o.val = blk.rowptr, blk.col, blk.val
    solver = bgs.Solver([[o]], [blk.nrows], [0], max_coarse=10, theta=[0.04])
    solver.setup()
    ref = oracle.AMG(oracle.CSR(blk.rowptr, blk.col, blk.val, blk.nrows, blk.ncols), theta=0.04, degree=4,
                     opts=oracle.default_options(max_coarse=10))
    assert solver.bgs_num_levels(0) == ref.nlevels >= 2
    for l in range(ref.nlevels - 1):
        assert np.array_equal(solver.bgs_level_aggregates(0, l), ref.aggregates(l))


@pytest.mark.parametrize("precision", [0, 1])
def test_vcycle_and_sweep_parity(bgs, precision):
    system = bs.assemble(grid=bs.Grid(3, 17, 13, 11), seed=2)
    g, o = make_pair(bgs, system, max_coarse=60, precision=precision)
    rng = np.random.default_rng(3)
    # FP64: the same arithmetic up to summation order; FP32 hierarchy: single-precision error
    tol = 1e-10 if precision == 0 else 2e-4
    for k in range(5):
        n = system.ncells
        b = rng.standard_normal(n)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        g.bgs_apply_vcycle(k, dev(b), x)
        ref = o.amg(k).vcycle(b)
        err = np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= tol, (k, err)
    v = rng.standard_normal(system.ndof)
    z = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    g.bgs_apply_preconditioner(dev(v), z)
    ref = o.apply(v)
    err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= (1e-10 if precision == 0 else 5e-3), err


@pytest.mark.parametrize("precision", [0, 1])
def test_sweep_ignores_unwritten_output_entries(bgs, precision):
    """The coupling SpMVs of the sweep read the output z only in fields already computed in the same
    sweep; the entries of later fields may hold anything (here NaN) without changing the result.
    In the paper's order phi_s (column block 0) comes last, so no padded SELL slot may read a column
    it does not store (SELL kept: autotuning off)."""
    system = bs.assemble(grid=bs.Grid(3, 17, 13, 11), seed=2)
    g = bgs.solver_for_system(system, order=list(spec.PAPER_ORDER), max_coarse=60, precision=precision,
                              autotune=0)
    g.setup()
    v = dev(np.random.default_rng(11).standard_normal(system.ndof))
    z0 = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    g.bgs_apply_preconditioner(v, z0)
    zn = torch.full((system.ndof,), float("nan"), dtype=torch.float64, device="cuda")
    g.bgs_apply_preconditioner(v, zn)
    assert bool(torch.isfinite(zn).all()) and torch.equal(z0, zn)


def test_ellipse_smoother_parity(bgs):
    """Chebyshev on an ellipse (cheb_ellipse = 1): the imaginary semi-axis of every level against the
    oracle's Bendixson estimate, the V-cycles of all blocks, and the solve."""
    system = bs.assemble(grid=bs.Grid(3, 17, 13, 11), seed=2)
    g, o = make_pair(bgs, system, max_coarse=60, cheb_ellipse=1)
    rng = np.random.default_rng(12)
    for k in range(5):
        oa = o.amg(k)
        for l in range(oa.nlevels - 1):
            ref = oa.cheb_imag(l)
            got = g.bgs_level_ellipse(k, l)
            assert (ref == 0.0) == (got == 0.0), (k, l, ref, got)
            assert abs(got - ref) <= 1e-10 * max(ref, 1e-300), (k, l, ref, got)
        b = rng.standard_normal(system.ncells)
        x = torch.zeros(system.ncells, dtype=torch.float64, device="cuda")
        g.bgs_apply_vcycle(k, dev(b), x)
        ref = oa.vcycle(b)
        assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref), k
    assert any(o.amg(k).cheb_imag(0) > 0 for k in (spec.C1, spec.C2))
    xr, ir = o.solve(system.b)
    x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    info = g.bgs_solve(dev(system.b), x)
    assert info.converged and ir.converged
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-6 * np.linalg.norm(xr)


# ------------------------------------------------------------------------------------- solve
@pytest.mark.parametrize("order", [spec.WORKLOAD_ORDER, spec.PAPER_ORDER], ids=["workload", "paper"])
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_parity(bgs, order, precision):
    system = bs.assemble("C1")
    g, o = make_pair(bgs, system, order=order, max_coarse=100, precision=precision)
    xr, ir = o.solve(system.b)
    assert ir.converged
    x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    info = g.bgs_solve(dev(system.b), x)
    xh = x.cpu().numpy()
    assert info.converged and info.status == 0
    true_rel = np.linalg.norm(system.b - o.full_matvec(xh)) / np.linalg.norm(system.b)
    assert true_rel <= 1e-8 and abs(true_rel - info.rel_true_resid) <= 1e-3 * true_rel + 1e-15
    assert np.linalg.norm(xh - xr) <= 1e-6 * np.linalg.norm(xr)
    if precision == 0:
        assert abs(info.iters - ir.iters) <= 2


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_is_bit_identical(bgs, precision):
    """The captured preconditioner graph runs the same kernels in the same order as direct
    launches, so the whole solve (forward and adjoint) must agree bit for bit."""
    system = bs.assemble(grid=bs.Grid(3, 17, 13, 11), seed=2)
    out = []
    for graph in (0, 1):
        g = bgs.solver_for_system(system, max_coarse=60, precision=precision, graph=graph)
        g.setup()
        x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
        info = g.bgs_solve(dev(system.b), x)
        lam = torch.zeros_like(x)
        info_a = g.bgs_solve_adjoint(dev(system.b), lam)
        out.append((x.cpu().numpy(), info.iters, lam.cpu().numpy(), info_a.iters))
        g.close()
    assert out[0][1] == out[1][1] and out[0][3] == out[1][3]
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("precision", [0, 1])
def test_block_jacobi_parity(bgs, precision):
    """Block Jacobi (couplings left out; the V-cycles run as concurrent branches): the
    preconditioner against the oracle's, the solve and adjoint against the oracle, and the
    concurrent graph replay bit-identical to the direct launches."""
    system = bs.assemble(grid=bs.Grid(3, 17, 13, 11), seed=2)
    o = oracle.bgs_for_system(system, order=list(spec.WORKLOAD_ORDER),
                              opts=oracle.default_options(max_coarse=60, jacobi=1))
    v = np.random.default_rng(7).standard_normal(system.ndof)
    ref = o.apply(v)
    xr, ir = o.solve(system.b)
    lr, il = o.solve_adjoint(system.b)
    out = []
    for graph in (0, 1):
        g = bgs.solver_for_system(system, order=list(spec.WORKLOAD_ORDER), max_coarse=60, precision=precision,
                                  graph=graph, jacobi=1)
        g.setup()
        z = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
        g.bgs_apply_preconditioner(dev(v), z)
        err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= (1e-10 if precision == 0 else 5e-3), err
        x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
        info = g.bgs_solve(dev(system.b), x)
        lam = torch.zeros_like(x)
        info_a = g.bgs_solve_adjoint(dev(system.b), lam)
        assert info.converged and info_a.converged
        xh, lh = x.cpu().numpy(), lam.cpu().numpy()
        assert np.linalg.norm(xh - xr) <= 1e-6 * np.linalg.norm(xr)
        assert np.linalg.norm(lh - lr) <= 1e-6 * np.linalg.norm(lr)
        if precision == 0:
            assert abs(info.iters - ir.iters) <= 2
        out.append((xh, lh, info.iters))
        g.close()
    assert out[0][2] == out[1][2]
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_solve_3d_default_options_and_host_buffers(bgs):
    system = bs.assemble(grid=bs.Grid(3, 24, 24, 24), seed=1)
    g, o = make_pair(bgs, system)
    xr, ir = o.solve(system.b)
    x = np.zeros(system.ndof)                     # host in, host out through the C ABI
    info = g.bgs_solve(system.b, x)
    assert info.converged
    assert np.linalg.norm(system.b - o.full_matvec(x)) <= 1e-8 * np.linalg.norm(system.b)
    assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)


def test_adjoint_parity_and_gradient(bgs):
    system = bs.assemble(grid=bs.Grid(3, 10, 9, 8), seed=4)
    g, o = make_pair(bgs, system, max_coarse=40, rtol=1e-12)
    rng = np.random.default_rng(5)
    gvec = rng.standard_normal(system.ndof)
    lam_ref, ir = o.solve_adjoint(gvec)
    lam = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    info = g.bgs_solve_adjoint(dev(gvec), lam)
    assert info.converged and ir.converged
    lh = lam.cpu().numpy()
    assert np.linalg.norm(lh - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    g.bgs_solve(dev(system.b), x)
    assert abs(gvec @ x.cpu().numpy() - lh @ system.b) <= 1e-9 * abs(gvec @ x.cpu().numpy())
    # dL/dA on the pattern of every stored block
    for (r, c), blk in system.blocks.items():
        d = torch.zeros(blk.nnz, dtype=torch.float64, device="cuda")
        g.bgs_grad_values(r, c, lam, x, d)
        n = system.ncells
        rows = np.repeat(np.arange(blk.nrows), np.diff(blk.rowptr))
        ref = -(lh[r * n + rows] * x.cpu().numpy()[c * n + blk.col])
        assert np.array_equal(d.cpu().numpy(), ref)


# ------------------------------------------------------------------------------------- errors
def test_error_statuses(bgs):
    system = bs.assemble(grid=bs.Grid(3, 6, 6, 6), seed=1)
    # unsorted columns in a diagonal block -> INVALID_ARG
    bad = bs.assemble(grid=bs.Grid(3, 6, 6, 6), seed=1)
    B = bad.blocks[(0, 0)]
    B.col[1], B.col[2] = B.col[2], B.col[1]
    with pytest.raises(bgs.BGSError) as e:
        bgs.solver_for_system(bad)
    assert e.value.status == bgs.INVALID_ARG
    # a missing diagonal entry -> INVALID_ARG
    bad2 = bs.assemble(grid=bs.Grid(3, 6, 6, 6), seed=1)
    B = bad2.blocks[(2, 2)]
    keep = np.ones(B.nnz, dtype=bool)
    keep[np.nonzero(B.col == 0)[0][0]] = False   # row 0's diagonal
    rows = np.repeat(np.arange(B.nrows), np.diff(B.rowptr))
    B.col, B.val = B.col[keep], B.val[keep]
    B.rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=B.nrows))]).astype(np.int32)
    with pytest.raises(bgs.BGSError) as e:
        bgs.solver_for_system(bad2)
    assert e.value.status == bgs.INVALID_ARG
    g = bgs.solver_for_system(system, max_coarse=20)
    x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(bgs.BGSError) as e:
        g.bgs_solve(dev(system.b), x)
    assert e.value.status == bgs.NOT_SETUP
    g.setup()
    bn = system.b.copy()
    bn[7] = np.nan
    with pytest.raises(bgs.BGSError) as e:
        g.bgs_solve(dev(bn), x)
    assert e.value.status == bgs.NAN_INF
    g2 = bgs.solver_for_system(system, max_coarse=20, maxit=1)
    g2.setup()
    info = g2.bgs_solve(dev(system.b), x)
    assert info.status == bgs.NO_CONVERGENCE and info.iters == 1 and not info.converged
    # zero right-hand side: x = 0, converged, no iterations
    info = g.bgs_solve(torch.zeros(system.ndof, dtype=torch.float64, device="cuda"), x)
    assert info.converged and info.iters == 0 and float(x.abs().max()) == 0.0


@pytest.mark.parametrize("precision", [0, 1])
def test_six_field_system_with_diagonal_field(bgs, precision):
    """Six fields, the sixth a diagonal solid-species block on the diagonal solve (subsolver 2, the
    direct inverse of A_s in Sec. 2.2): that block's solve is 1/diag bit for bit, and the solve and
    adjoint agree with the oracle."""
    from six_field import six_field, dense, SOLID
    nested, sizes, b = six_field(bs.Grid(3, 10, 9, 8), seed=3)
    order = list(spec.WORKLOAD_ORDER) + [SOLID]
    sub = [0, 0, 0, 0, 0, 2]
    o = oracle.BGS(nested, sizes, order, oracle.default_options(max_coarse=40, subsolver=sub))
    assert o.setup() == 0
    xr, ir = o.solve(b)
    lr, il = o.solve_adjoint(b)
    g = bgs.Solver(nested, sizes, order, max_coarse=40, subsolver=sub, precision=precision)
    g.setup()
    assert g.bgs_num_levels(SOLID) == 1
    r = np.random.default_rng(2).standard_normal(sizes[SOLID])
    z = torch.zeros(sizes[SOLID], dtype=torch.float64, device="cuda")
    g.bgs_apply_vcycle(SOLID, dev(r), z)
    d = nested[SOLID][SOLID].val
    if precision == 0:
        assert np.array_equal(z.cpu().numpy(), (1.0 / d) * r)
    else:
        assert np.abs(z.cpu().numpy() - r / d).max() <= 1e-6 * np.abs(r / d).max()
    x = torch.zeros(sum(sizes), dtype=torch.float64, device="cuda")
    info = g.bgs_solve(dev(b), x)
    A = dense(nested, sizes)
    xh = x.cpu().numpy()
    assert info.converged and ir.converged
    assert np.linalg.norm(b - A @ xh) <= 1e-8 * np.linalg.norm(b)
    assert np.linalg.norm(xh - xr) <= 1e-6 * np.linalg.norm(xr)
    lam = torch.zeros_like(x)
    assert g.bgs_solve_adjoint(dev(b), lam).converged
    assert np.linalg.norm(lam.cpu().numpy() - lr) <= 1e-6 * np.linalg.norm(lr)
