"""Parity at the benchmark's full size (3D 128^3, 10.5M DOFs) in the configuration bench.py times,
on outputs the oracle can recompute there: the level-0 strength decisions and aggregates of two
blocks (bit-exact), the level-0 smoothed prolongator, and the true residual of the solve; plus
degenerate block structures at small size."""
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


@pytest.fixture(scope="module")
def c4():
    return bs.assemble("C4", seed=1)


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_solve_and_level0_parity(bgs, c4, precision):
    system = c4
    g = bgs.solver_for_system(system, precision=precision)   # library defaults, as in bench.py
    g.setup()
    x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    info = g.bgs_solve(torch.from_numpy(system.b).cuda(), x)
    assert info.converged
    full = oracle.CSR(*(lambda A: (A.rowptr, A.col, A.val, A.nrows, A.ncols))(system.full_csr()))
    r = system.b - oracle.spmv(full, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(system.b)
    if precision == 1:
        return
    opts = oracle.default_options()
    for field in (spec.PHI_S, spec.C1):
        blk = system.blocks[(field, field)]
        A = oracle.CSR(blk.rowptr, blk.col, blk.val, blk.nrows, blk.ncols)
        strong = oracle.strength_flags(A, opts.theta[field])
        S = oracle.strength_graph(A, strong)
        state, rounds = oracle.mis2(S, oracle.mis_salt(0))
        agg, nagg = oracle.aggregate(S, state)
        info0 = g.bgs_level_info(field, 0)
        assert info0["nagg"] == nagg and info0["mis_rounds"] == rounds
        assert np.array_equal(g.bgs_level_aggregates(field, 0), agg)
        # smoothed prolongator from the oracle's filter and power iteration
        vF, dF = oracle.filter_matrix(A, strong, opts.filter_diag)
        rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
        mask = (A.col == rows) | (strong == 1)
        rp = np.zeros(A.nrows + 1, dtype=np.int32)
        np.cumsum(np.bincount(rows[mask], minlength=A.nrows), out=rp[1:])
        AF = oracle.CSR(rp, A.col[mask], vF[mask], A.nrows, A.ncols)
        lam = oracle.power_lambda(AF, 1.0 / dF, opts.power_iters)
        P = oracle.smooth_prolongator(AF, 1.0 / dF, agg, nagg, (4.0 / 3.0) / lam)
        prp, pci, pv = g.bgs_level_copy(field, 0, 1)
        assert np.array_equal(prp, P.rowptr) and np.array_equal(pci, P.col)
        assert np.abs(pv - P.val).max() <= 1e-12
        assert abs(info0["omega"] - (4.0 / 3.0) / lam) <= 1e-12 * abs(info0["omega"])


def _subsystem(system, fields):
    n = system.ncells
    blocks = [[system.blocks.get((r, c)) for c in fields] for r in fields]
    b = np.concatenate([system.b[f * n:(f + 1) * n] for f in fields])
    return blocks, [n] * len(fields), b


class _Obj:
    pass


def _solver(bgs, blocks, sizes, order, **kw):
    bl = []
    for row in blocks:
        r2 = []
        for B in row:
            if B is None:
                r2.append(None)
                continue
            o = _Obj()
            o.rowptr, o.col, o.val = B.rowptr, B.col, B.val
            r2.append(o)
        bl.append(r2)
    return bgs.Solver(bl, sizes, order, **kw)


@pytest.mark.parametrize("fields", [[spec.PHI_S], [spec.PHI_S, spec.PHI_E], [spec.PRESS, spec.C1, spec.C2]])
def test_degenerate_block_structures(bgs, fields):
    system = bs.assemble(grid=bs.Grid(3, 12, 11, 10), seed=5)
    blocks, sizes, b = _subsystem(system, fields)
    order = list(range(len(fields)))[::-1]
    for mc in (20, 5000):                    # multi-level, and a single direct (dense LU) level
        g = _solver(bgs, blocks, sizes, order, max_coarse=mc)
        g.setup()
        x = np.zeros(sum(sizes))
        info = g.bgs_solve(b, x, check=False)
        o = oracle.BGS(blocks, sizes, order, oracle.default_options(max_coarse=mc))
        assert o.setup() == 0
        xr, ir = o.solve(b)
        assert info.converged and ir.converged, (mc, info.status, info.iters, ir.iters)
        assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)
        if mc == 5000:
            assert all(g.bgs_num_levels(k) == 1 for k in range(len(fields)))
            assert info.iters <= 10           # exact block solves: only the ignored upper blocks remain
