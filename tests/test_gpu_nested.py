"""Nested variant on the GPU (Sec. 2.2: the block preconditioner over the groups [phi_s, phi_e] and
[p, c1, c2], each group's block solved by an inner FGMRES preconditioned by the group's sweep;
Sec. 3.2: outer FGMRES(5)) against the oracle's nested variant."""
import numpy as np
import pytest

import battery_system as bs
import oracle
from battery_system import spec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDER = list(spec.WORKLOAD_ORDER)
NEST = dict(ngroups=2, group_end=[2, 5])


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


def test_nested_preconditioner_with_tight_inner_solves(bgs):
    """Inner solves to 1e-12: the preconditioner is the group-triangular inverse up to that
    tolerance on both sides, so GPU and oracle agree far below the outer tolerance."""
    system = bs.assemble(grid=bs.Grid(3, 12, 11, 10), seed=5)
    kw = dict(max_coarse=40, inner_rtol=1e-12, inner_maxit=300, inner_restart=60, **NEST)
    o = oracle.bgs_for_system(system, order=ORDER, opts=oracle.default_options(**kw))
    g = bgs.solver_for_system(system, order=ORDER, **kw)
    g.setup()
    v = np.random.default_rng(3).standard_normal(system.ndof)
    z = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    g.bgs_apply_preconditioner(dev(v), z)
    ref = o.apply(v)
    assert np.linalg.norm(z.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_nested_solve_and_adjoint(bgs, precision):
    """The paper's nested configuration: outer FGMRES(5), inner FGMRES(30) to 1e-6."""
    system = bs.assemble(grid=bs.Grid(3, 16, 14, 12), seed=3)
    kw = dict(max_coarse=60, restart=5, **NEST)
    o = oracle.bgs_for_system(system, order=ORDER, opts=oracle.default_options(**kw))
    xr, ir = o.solve(system.b)
    lr, il = o.solve_adjoint(system.b)
    assert ir.converged and il.converged
    g = bgs.solver_for_system(system, order=ORDER, precision=precision, **kw)
    g.setup()
    x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    info = g.bgs_solve(dev(system.b), x)
    assert info.converged
    xh = x.cpu().numpy()
    assert np.linalg.norm(system.b - system.matvec(xh)) <= 1e-8 * np.linalg.norm(system.b)
    assert np.linalg.norm(xh - xr) <= 1e-6 * np.linalg.norm(xr)
    if precision == 0:
        assert abs(info.iters - ir.iters) <= 1
    lam = torch.zeros_like(x)
    assert g.bgs_solve_adjoint(dev(system.b), lam).converged
    assert np.linalg.norm(lam.cpu().numpy() - lr) <= 1e-6 * np.linalg.norm(lr)


def test_nested_paper_order_and_errors(bgs):
    system = bs.assemble(grid=bs.Grid(3, 10, 9, 8), seed=2)
    order = list(spec.PAPER_ORDER)                       # [p, c1, c2] then [phi_e, phi_s]
    kw = dict(max_coarse=40, restart=5, ngroups=2, group_end=[3, 5])
    o = oracle.bgs_for_system(system, order=order, opts=oracle.default_options(**kw))
    xr, _ = o.solve(system.b)
    g = bgs.solver_for_system(system, order=order, **kw)
    g.setup()
    x = np.zeros(system.ndof)
    assert g.bgs_solve(system.b, x).converged
    assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)
    for bad in (dict(ngroups=2, group_end=[2, 4]),          # does not end at the last position
                dict(ngroups=2, group_end=[3, 3]),          # empty group
                dict(ngroups=2, group_end=[1, 5])):         # {c1, c2, phi_e, phi_s}: ids not consecutive
        with pytest.raises(bgs.BGSError):
            bgs.solver_for_system(system, order=order, **bad)
    with pytest.raises(bgs.BGSError):                        # fields {phi_s, p} are not consecutive ids
        bgs.solver_for_system(system, order=[0, 2, 1, 3, 4], ngroups=2, group_end=[2, 5])
