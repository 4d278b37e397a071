"""Gradients through the solve on the 3D 48^3 five-field system (553k DOFs): the autograd path
(adjoint solve + -lambda x^T on the pattern) against central finite differences of full solves
and against the oracle's adjoint."""
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


def loss_weights(system):
    """L = mean of phi_s over the current-collector face."""
    c = np.zeros(system.ndof)
    c[system.collector] = 1.0 / len(system.collector)
    return c


def solve_loss(bgs, system, rtol):
    g = bgs.solver_for_system(system, rtol=rtol)
    g.setup()
    x = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    info = g.bgs_solve(torch.from_numpy(system.b).cuda(), x)
    assert info.converged
    return float(loss_weights(system) @ x.cpu().numpy())


def test_adjoint_gradients_c3(bgs):
    system = bs.assemble("C3", seed=1)
    keys = sorted(system.blocks.keys())
    pats = {k: (torch.from_numpy(system.blocks[k].rowptr).cuda(), torch.from_numpy(system.blocks[k].col).cuda())
            for k in keys}
    vals = {k: torch.from_numpy(system.blocks[k].val).cuda().requires_grad_(True) for k in keys}
    b = torch.from_numpy(system.b).cuda().requires_grad_(True)
    # FP64 solves of this system stagnate near a true residual of 1.4e-12, so 1e-11 is the tightest
    # tolerance used; the oracle comparison uses 1e-10 on both sides
    x = bgs.bgs_solve_autograd(pats, vals, b, system.field_sizes, list(spec.WORKLOAD_ORDER), rtol=1e-11)
    w = torch.from_numpy(loss_weights(system)).cuda()
    L = (w * x).sum()
    L.backward()
    lam = b.grad.cpu().numpy()

    # dL/db against the oracle's adjoint solve (transposed block sweep, MGS FGMRES)
    o = oracle.bgs_for_system(system, opts=oracle.default_options(rtol=1e-10))
    lam_or, info = o.solve_adjoint(loss_weights(system))
    assert info.converged
    assert np.linalg.norm(lam - lam_or) <= 1e-6 * np.linalg.norm(lam_or)

    # per-layer conductivity means and the exchange-current scale: chain rule through the
    # assembled values (d values / d parameter by central differences of the assembly, which is
    # exact arithmetic on smooth functions) against central differences of full solves
    def grad_param(make):
        # central differences: truncation O(h^2) and the noise of the solves to 1e-11 over 2h; h = 1e-4
        # keeps both near 1e-8-1e-7 relative, well inside the 1e-5 check (h = 1e-6 put the noise at it)
        h = 1e-4
        sp, sm = make(+h), make(-h)
        g = 0.0
        for k in keys:
            dv = (sp.blocks[k].val - sm.blocks[k].val) / (2 * h) if k in sp.blocks else 0.0
            g += float(vals[k].grad.cpu().numpy() @ dv) if np.ndim(dv) else 0.0
        fd = (solve_loss(bgs, sp, 1e-11) - solve_loss(bgs, sm, 1e-11)) / (2 * h)
        return g, fd

    means = np.array(spec.SIGMA_S_MEANS)
    for layer in range(3):
        def make(eps, layer=layer):
            m = means.copy()
            m[layer] *= (1.0 + eps)
            return bs.assemble("C3", seed=1, sigma_means=m)
        g, fd = grad_param(make)
        assert abs(g - fd) <= 1e-5 * abs(fd) + 1e-12, (layer, g, fd)
    g, fd = grad_param(lambda eps: bs.assemble("C3", seed=1, i0_scale=1.0 + eps))
    assert abs(g - fd) <= 1e-5 * abs(fd) + 1e-12, ("i0", g, fd)
