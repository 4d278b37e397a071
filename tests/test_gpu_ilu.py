"""DD(0)-ILU(0) species solver on the GPU against the oracle: the factors and one sweep bit for bit
(same operations in the same order, products and differences rounded separately), the solve and
adjoint with the species blocks on DD(0)-ILU(0) in both precisions, and the numeric re-set-up."""
import numpy as np
import pytest

import battery_system as bs
import oracle
from battery_system import spec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDER = list(spec.WORKLOAD_ORDER)
SUB = [0, 0, 0, 1, 1]          # c1, c2 on DD(0)-ILU(0)


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


def _csr(B):
    return oracle.CSR(B.rowptr, B.col, B.val, B.nrows, B.ncols)


@pytest.mark.parametrize("rows", [128, 1000, 8192])
def test_factors_and_sweep_bit_exact(bgs, rows):
    system = bs.assemble(grid=bs.Grid(3, 17, 13, 11), seed=2)      # 2431 rows: several subdomains + a ragged tail
    g = bgs.solver_for_system(system, order=ORDER, subsolver=SUB, ilu_rows=rows, max_coarse=60)
    g.setup()
    rng = np.random.default_rng(rows)
    for k in (spec.C1, spec.C2):
        ref = oracle.ILU(_csr(system.blocks[(k, k)]), rows)
        assert ref.status == 0
        F = ref.factors()
        rp, ci, v = g.bgs_ilu_factors(k)
        assert np.array_equal(rp, F.rowptr) and np.array_equal(ci, F.col)
        assert np.array_equal(v, F.val)
        assert g.bgs_num_levels(k) == 1
        b = rng.standard_normal(system.ncells)
        x = torch.zeros(system.ncells, dtype=torch.float64, device="cuda")
        g.bgs_apply_vcycle(k, dev(b), x)
        assert np.array_equal(x.cpu().numpy(), ref.apply(b))


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_and_adjoint_with_dd_ilu(bgs, precision):
    system = bs.assemble(grid=bs.Grid(3, 16, 14, 12), seed=3)
    o = oracle.bgs_for_system(system, order=ORDER,
                              opts=oracle.default_options(subsolver=SUB, ilu_rows=256, max_coarse=60))
    xr, ir = o.solve(system.b)
    lr, il = o.solve_adjoint(system.b)
    assert ir.converged and il.converged
    g = bgs.solver_for_system(system, order=ORDER, subsolver=SUB, ilu_rows=256, max_coarse=60,
                              precision=precision)
    g.setup()
    v = np.random.default_rng(2).standard_normal(system.ndof)
    z = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    g.bgs_apply_preconditioner(dev(v), z)
    ref = o.apply(v)
    err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= (1e-10 if precision == 0 else 5e-3), err
    x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    info = g.bgs_solve(dev(system.b), x)
    assert info.converged
    xh = x.cpu().numpy()
    assert np.linalg.norm(system.b - system.matvec(xh)) <= 1e-8 * np.linalg.norm(system.b)
    assert np.linalg.norm(xh - xr) <= 1e-6 * np.linalg.norm(xr)
    if precision == 0:
        assert abs(info.iters - ir.iters) <= 2
    lam = torch.zeros_like(x)
    assert g.bgs_solve_adjoint(dev(system.b), lam).converged
    assert np.linalg.norm(lam.cpu().numpy() - lr) <= 1e-6 * np.linalg.norm(lr)


def test_update_refactors_dd_ilu(bgs):
    system = bs.assemble(grid=bs.Grid(3, 12, 11, 10), seed=7)
    g = bgs.solver_for_system(system, order=ORDER, subsolver=SUB, ilu_rows=200, max_coarse=40)
    g.setup()
    rng = np.random.default_rng(4)
    vals = [[None] * 5 for _ in range(5)]
    new = {}
    for k in (spec.C1, spec.C2):
        B = system.blocks[(k, k)]
        new[k] = B.val * (1.0 + 0.3 * rng.uniform(0, 1, B.nnz))
        vals[k][k] = new[k]
    g.bgs_update_values(vals)
    for k in (spec.C1, spec.C2):
        B = system.blocks[(k, k)]
        ref = oracle.ILU(oracle.CSR(B.rowptr, B.col, new[k], B.nrows, B.ncols), 200)
        rp, ci, v = g.bgs_ilu_factors(k)
        assert np.array_equal(v, ref.factors().val)


def test_ilu_option_errors(bgs):
    system = bs.assemble(grid=bs.Grid(3, 6, 5, 4), seed=1)
    with pytest.raises(bgs.BGSError):
        bgs.solver_for_system(system, subsolver=[0, 0, 0, 3, 0])
    with pytest.raises(bgs.BGSError):
        bgs.solver_for_system(system, subsolver=SUB, ilu_rows=9000)
    g = bgs.solver_for_system(system, order=ORDER)
    g.setup()
    with pytest.raises(bgs.BGSError):
        g.bgs_ilu_factors(spec.C1)                 # that field is on the V-cycle
