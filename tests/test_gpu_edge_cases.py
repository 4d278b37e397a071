"""Degenerate shapes through the C ABI against dense solves: a 1 x 1 system, a two-row field, fields
of different sizes with rectangular couplings, an explicitly empty coupling block, a zero
right-hand side, and every block solver on the smallest sizes."""
import numpy as np
import pytest

import battery_system as bs

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


def csr(D):
    D = np.asarray(D, dtype=np.float64)
    r, c = np.nonzero(D)                        # row-major order
    rp = np.searchsorted(r, np.arange(D.shape[0] + 1)).astype(np.int32)
    return bs.CSR(rp, c.astype(np.int32), D[r, c].copy(), D.shape[0], D.shape[1])


def dd_matrix(n, rng):
    """A nonsymmetric, diagonally dominant tridiagonal matrix."""
    D = np.diag(4.0 + rng.uniform(0, 1, n))
    for i in range(n - 1):
        D[i, i + 1] = -rng.uniform(0.2, 1.0)
        D[i + 1, i] = -rng.uniform(0.2, 1.0)
    return D


def solve(bgs, nested, sizes, order, b, **kw):
    g = bgs.Solver(nested, sizes, order, **kw)
    g.setup()
    x = np.zeros(sum(sizes))
    info = g.bgs_solve(np.asarray(b, dtype=np.float64), x)
    g.close()
    return x, info


@pytest.mark.parametrize("subsolver", [0, 1, 2])
def test_one_by_one_system(bgs, subsolver):
    x, info = solve(bgs, [[csr([[4.0]])]], [1], [0], [2.0], subsolver=[subsolver], ilu_rows=1)
    assert info.converged and info.iters <= 1 and x[0] == 0.5


@pytest.mark.parametrize("subsolver", [0, 1])
def test_two_fields_of_different_sizes(bgs, subsolver):
    rng = np.random.default_rng(4)
    n0, n1 = 7, 2
    A00, A11 = dd_matrix(n0, rng), dd_matrix(n1, rng)
    A10 = np.zeros((n1, n0))
    A10[0, 3], A10[1, 6] = -0.5, 0.25
    A01 = np.zeros((n0, n1))
    A01[2, 1] = 0.3
    nested = [[csr(A00), csr(A01)], [csr(A10), csr(A11)]]
    A = np.block([[A00, A01], [A10, A11]])
    b = rng.standard_normal(n0 + n1)
    for order in ([0, 1], [1, 0]):
        x, info = solve(bgs, nested, [n0, n1], order, b, max_coarse=1, subsolver=[subsolver, subsolver],
                        ilu_rows=3)
        assert info.converged
        assert np.linalg.norm(A @ x - b) <= 1e-8 * np.linalg.norm(b)
        assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-7 * np.linalg.norm(x)


def test_explicit_empty_coupling_and_zero_rhs(bgs):
    rng = np.random.default_rng(5)
    n = 40
    A00, A11 = dd_matrix(n, rng), dd_matrix(n, rng)
    empty = bs.CSR(np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0), n, n)
    nested = [[csr(A00), empty], [csr(np.eye(n) * 0.1), csr(A11)]]
    A = np.block([[A00, np.zeros((n, n))], [np.eye(n) * 0.1, A11]])
    b = rng.standard_normal(2 * n)
    x, info = solve(bgs, nested, [n, n], [0, 1], b, max_coarse=8)
    assert info.converged and np.linalg.norm(A @ x - b) <= 1e-8 * np.linalg.norm(b)
    x0, info0 = solve(bgs, nested, [n, n], [0, 1], np.zeros(2 * n), max_coarse=8)
    assert info0.converged and info0.iters == 0 and not np.any(x0)


@pytest.mark.parametrize("n", [1, 7, 9, 17, 483, 1000, 1281, 2560, 2561])
def test_coarsest_direct_solve_sizes(bgs, n):
    """A single-level hierarchy (max_coarse >= n): the V-cycle is the coarsest direct solve alone.
    Sizes below and above the blocked Gauss-Jordan panel width (16) and its shared-memory limit
    (2560 rows, beyond which the one-launch-per-pivot form runs), against a dense FP64 solve of a
    nonsymmetric matrix whose pivots need row interchanges."""
    rng = np.random.default_rng(n)
    D = dd_matrix(n, rng)
    # strong couplings to a few far rows, and a small diagonal on every third row: partial
    # pivoting must interchange rows
    for i in range(n):
        for j in rng.choice(n, size=min(n, 3), replace=False):
            D[i, j] += rng.uniform(-3.0, 3.0)
    D[np.arange(0, n, 3), np.arange(0, n, 3)] = 1e-3
    b = rng.standard_normal(n)
    g = bgs.Solver([[csr(D)]], [n], [0], max_coarse=max(n, 1))
    g.setup()
    assert g.bgs_num_levels(0) == 1
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    g.bgs_apply_vcycle(0, torch.from_numpy(b).cuda(), x)
    ref = np.linalg.solve(D, b)
    cond = np.linalg.cond(D)
    # backward-stable elimination: relative error within a small multiple of n eps cond
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 4 * n * np.finfo(float).eps * cond * np.linalg.norm(ref)
    g.close()
