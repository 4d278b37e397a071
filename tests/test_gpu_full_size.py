"""Parity at the benchmark's full size (3D 128^3, 10.5M DOFs) in the configuration bench.py times,
and on the largest workload (the 160x160x400 pellet stack, 51.2M DOFs).

128^3: the GPU hierarchy against the oracle's on every block and level (strength decisions, MIS-2
round counts, aggregates and patterns bit-exact; omega, Chebyshev bounds, P, R and A_l values within
the tolerances of the small cases), and both solves against the oracle's solution.  160x160x400:
the FP64 and mixed solves reach a true relative residual of 1e-8 (checked on the host with the
oracle's SpMV).  Plus degenerate block structures at small size."""
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


@pytest.fixture(scope="module")
def c4_ref(c4):
    o = oracle.bgs_for_system(c4)           # oracle defaults = library defaults
    x, info = o.solve(c4.b)
    assert info.converged
    return o, x, info


def test_full_size_hierarchy_parity(bgs, c4, c4_ref):
    o = c4_ref[0]
    g = bgs.solver_for_system(c4)            # library defaults, as in bench.py
    g.setup()
    for k in range(5):
        oa = o.amg(k)
        nl = g.bgs_num_levels(k)
        assert nl == oa.nlevels, (k, nl, oa.sizes())
        for l in range(nl):
            info = g.bgs_level_info(k, l)
            assert info["rows"] == oa.sizes()[l], (k, l)
            rp, ci, v = g.bgs_level_copy(k, l, 0)
            A = oa.level_matrix(l)
            assert np.array_equal(rp, A.rowptr) and np.array_equal(ci, A.col), (k, l)
            assert np.abs(v - A.val).max() <= 1e-11 * np.abs(A.val).max(), (k, l)
            if l + 1 == nl:
                continue
            assert np.array_equal(g.bgs_level_strength(k, l), oa.strong(l)), (k, l)
            assert info["mis_rounds"] == oa.mis_rounds(l) and info["nagg"] == oa.nagg(l), (k, l)
            assert np.array_equal(g.bgs_level_aggregates(k, l), oa.aggregates(l)), (k, l)
            assert abs(info["omega"] - oa.omega(l)) <= 1e-12 * abs(oa.omega(l)), (k, l)
            lo, hi = oa.cheb_bounds(l)
            assert abs(info["lmax"] - hi) <= 1e-10 * hi and abs(info["lmin"] - lo) <= 1e-10 * lo, (k, l)
            for which, M in ((1, oa.prolongator(l)), (2, oa.restriction(l))):
                prp, pci, pv = g.bgs_level_copy(k, l, which)
                assert np.array_equal(prp, M.rowptr) and np.array_equal(pci, M.col), (k, l, which)
                assert np.abs(pv - M.val).max() <= 1e-12 * max(1.0, np.abs(M.val).max()), (k, l, which)
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_solve_matches_the_oracle(bgs, c4, c4_ref, precision):
    o, xr, ir = c4_ref
    g = bgs.solver_for_system(c4, precision=precision)
    g.setup()
    x = torch.zeros(c4.ndof, dtype=torch.float64, device="cuda")
    info = g.bgs_solve(torch.from_numpy(c4.b).cuda(), x)
    assert info.converged
    xh = x.cpu().numpy()
    rel = np.linalg.norm(c4.b - o.full_matvec(xh)) / np.linalg.norm(c4.b)
    err = np.linalg.norm(xh - xr) / np.linalg.norm(xr)
    print(f"128^3 precision={precision}: iters {info.iters} (oracle {ir.iters}), true rel. residual {rel:.3e}, "
          f"||x - x_oracle|| / ||x_oracle|| = {err:.3e}")
    assert rel <= 1e-8 and err <= 1e-6
    if precision == 0:
        assert abs(info.iters - ir.iters) <= 2
    g.close()


@pytest.fixture(scope="module")
def c5():
    return bs.assemble("C5", seed=1)


@pytest.mark.parametrize("precision", [0, 1])
def test_largest_workload_true_residual(bgs, c5, precision):
    g = bgs.solver_for_system(c5, precision=precision)
    g.setup()
    x = torch.zeros(c5.ndof, dtype=torch.float64, device="cuda")
    info = g.bgs_solve(torch.from_numpy(c5.b).cuda(), x)
    assert info.converged
    xh, n = x.cpu().numpy(), c5.ncells
    Ax = np.zeros(c5.ndof)
    for (r, c), blk in c5.blocks.items():       # block by block: the full operator is 7 GB on the host
        Ax[r * n:(r + 1) * n] += oracle.spmv(oracle.CSR(blk.rowptr, blk.col, blk.val, blk.nrows, blk.ncols),
                                             xh[c * n:(c + 1) * n])
    rel = np.linalg.norm(c5.b - Ax) / np.linalg.norm(c5.b)
    print(f"160x160x400 precision={precision}: iters {info.iters}, true rel. residual {rel:.3e} "
          f"(library's {info.rel_true_resid:.3e})")
    assert rel <= 1e-8
    g.close()
    del g
    torch.cuda.empty_cache()


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
