"""Pins of the seeded input generator (the synthetic coupled battery system).

The generator is the problem definition both sides consume; these tests tie it to
closed forms and to an independent loop-by-loop assembly.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import battery_system as bs
from battery_system import spec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hash_vectors.txt")


def _golden(kind):
    out = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, a, b = line.split()
        if k == kind:
            out.append((int(a, 0), int(b, 0)))
    return out


def test_splitmix64_published_values():
    # the generator's mixer, run as the plain SplitMix64 sequence from state 0
    for idx, want in _golden("splitmix64"):
        state = np.uint64(((idx + 1) * 0x9E3779B97F4A7C15) & ((1 << 64) - 1))
        assert int(bs._mix64_np(np.array([state]))[0]) == want


def test_uniform_and_normal_moments():
    c = np.arange(200000, dtype=np.uint64)
    u = bs.rng_uniform(7, 3, c)
    assert u.min() > 0.0 and u.max() <= 1.0
    assert abs(u.mean() - 0.5) < 4e-3 and abs(u.var() - 1 / 12) < 2e-3
    z = bs.rng_normal(7, 3, c)
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 1.5e-2
    # streams and seeds are independent sequences
    assert not np.array_equal(bs.rng_u64(7, 3, c[:10]), bs.rng_u64(7, 4, c[:10]))
    assert not np.array_equal(bs.rng_u64(7, 3, c[:10]), bs.rng_u64(8, 3, c[:10]))


def _brute_force(system):
    """Loop-by-loop dense assembly of the same equations, written independently of the
    vectorised slots (same summation order so that the result is bit-identical)."""
    g = system.grid
    n = g.ncells
    d = g.dim
    h = g.h
    V = h ** d
    hfac = h ** (d - 2)
    hface = h ** (d - 1)
    co = system.params
    F = 5
    A = np.zeros((F * n, F * n))
    kx = co["kx"]
    kz = kx * (spec.PERM_Z_RATIO if d == 3 else 1.0)
    perm = (kx, kx, kz)
    kbv = spec.bv_rate_constant() * co["i0"]
    U = spec.DUDC

    def cell(i, j, k):
        return i + g.nx * (j + g.ny * k)

    # face order of the diagonal sum: z-, y-, x-, x+, y+, z+
    faces = ([(2, -1)] if d == 3 else []) + [(1, -1), (0, -1), (0, 1), (1, 1)] + ([(2, 1)] if d == 3 else [])
    dims = (g.nx, g.ny, g.nz)

    def neighbours(i, j, k):
        out = []
        for ax, sd in faces:
            ijk = [i, j, k]
            ijk[ax] += sd
            if 0 <= ijk[ax] < dims[ax]:
                out.append((ax, sd, cell(*ijk)))
        return out

    def hm(a, b):
        return 2.0 * a * b / (a + b)

    for k in range(g.nz):
        for j in range(g.ny):
            for i in range(g.nx):
                c = cell(i, j, k)
                nb = neighbours(i, j, k)
                Vk = V * kbv[c]
                elec = kbv[c] > 0
                on_dir = (k == 0) if co["stack"] else (i == 0)
                # phi_s
                dg = 0.0
                for ax, sd, m in nb:
                    t = hfac * hm(co["sigma"][c], co["sigma"][m])
                    A[c, m] = -t
                    dg = dg + t
                dg = dg + (2.0 * hfac * co["sigma"][c] if on_dir else 0.0)
                dg = dg + Vk
                A[c, c] = dg
                # phi_e
                r = n + c
                dg = 0.0
                for ax, sd, m in nb:
                    t = hfac * hm(co["kappa"][c], co["kappa"][m])
                    A[r, n + m] = -t
                    dg = dg + t
                A[r, r] = dg + V * spec.TAU_OVER_DT + Vk
                # p
                r = 2 * n + c
                dg = 0.0
                for ax, sd, m in nb:
                    t = hfac * hm(perm[ax][c], perm[ax][m])
                    A[r, 2 * n + m] = -t
                    dg = dg + t
                A[r, r] = dg + V * spec.STORAGE_OVER_DT
                # species
                fout = hface * (hm(kx[c], kx[c + 1]) if i < g.nx - 1 else kx[c])
                fin = hface * hm(kx[c], kx[c - 1]) if i > 0 else 0.0
                for mm, dm in enumerate((co["d1"], co["d2"])):
                    r = (3 + mm) * n + c
                    dg = 0.0
                    lk = 0.0
                    for ax, sd, m in nb:
                        t = hfac * hm(dm[c], dm[m])
                        val = -t
                        if ax == 0 and sd < 0:
                            val = val - fin
                        A[r, (3 + mm) * n + m] = val
                        dg = dg + t
                        tk = hfac * hm(perm[ax][c], perm[ax][m])
                        A[r, 2 * n + m] = spec.C0[mm] * (-tk)
                        lk = lk + tk
                    A[r, 2 * n + c] = spec.C0[mm] * lk
                    A[r, r] = dg + fout + V / spec.DT + V * spec.EPS_CROSS + spec.GAMMA_C[mm] * Vk * U
                    other = (4 - mm) * n + c
                    A[r, other] = -V * spec.EPS_CROSS
                    if elec and spec.GAMMA_C[mm] != 0.0:
                        A[r, c] = -spec.GAMMA_C[mm] * Vk
                        A[r, n + c] = spec.GAMMA_C[mm] * Vk
                if elec:
                    A[c, n + c] = -Vk
                    A[c, 3 * n + c] = -Vk * U
                    A[n + c, c] = -Vk
                    A[n + c, 3 * n + c] = Vk * U
                    A[2 * n + c, c] = -spec.GAMMA_P * Vk
                    A[2 * n + c, n + c] = spec.GAMMA_P * Vk
                    A[2 * n + c, 3 * n + c] = spec.GAMMA_P * Vk * U
    return A


@pytest.mark.parametrize("grid,stack", [(bs.Grid(3, 4, 4, 4), False), (bs.Grid(2, 5, 4, 1), False),
                                        (bs.Grid(3, 3, 3, 20), True)])
def test_assembly_bit_identical_to_brute_force(grid, stack):
    s = bs.assemble(grid=grid, stack=stack, seed=3)
    A = s.full_dense()
    B = _brute_force(s)
    assert np.array_equal(A, B)
    # structural entries are exactly the non-zeros of the brute force
    nnz_bf = int(np.count_nonzero(B))
    assert s.nnz == nnz_bf


def test_diffusion_blocks_symmetric_and_conservative():
    s = bs.assemble(grid=bs.Grid(3, 6, 5, 4), seed=2)
    n = s.ncells
    V = s.params["V"]
    for f in (spec.PHI_S, spec.PHI_E, spec.PRESS):
        D = s.blocks[(f, f)].to_dense()
        assert np.array_equal(D, D.T)
    # p block: every row sums to the storage term (no boundary condition on p)
    P = s.blocks[(spec.PRESS, spec.PRESS)].to_dense()
    rs = P.sum(axis=1)
    assert np.allclose(rs, V * spec.STORAGE_OVER_DT, rtol=0, atol=1e-14 * np.abs(np.diag(P)).max())
    # A_{c,p} is c0 times a zero-row-sum Laplacian
    for m, f in enumerate((spec.C1, spec.C2)):
        L = s.blocks[(f, spec.PRESS)].to_dense()
        assert np.abs(L.sum(axis=1)).max() <= 1e-14 * np.abs(np.diag(L)).max()
    # separator cells carry no Butler-Volmer coupling
    sep = np.nonzero(s.layer == 1)[0]
    bv = s.blocks[(spec.PHI_S, spec.PHI_E)]
    rows = np.repeat(np.arange(n), np.diff(bv.rowptr))
    assert not np.isin(rows, sep).any()


def _manufactured_error(dim, N):
    A, centres, grid = bs.poisson_dirichlet(dim, N, coef=1.0)
    u = np.ones(grid.ncells)
    for x in centres:
        u = u * np.sin(math.pi * x)
    f = dim * math.pi ** 2 * u
    V = grid.h ** dim
    M = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.nrows, A.ncols))
    uh = spla.spsolve(M.tocsc(), V * f)
    return np.abs(uh - u).max()


@pytest.mark.parametrize("dim,N", [(2, 32), (3, 12)])
def test_manufactured_solution_second_order(dim, N):
    e1 = _manufactured_error(dim, N)
    e2 = _manufactured_error(dim, 2 * N)
    rate = math.log2(e1 / e2)
    assert rate >= 1.8, rate


def test_named_configs_sizes():
    s = bs.assemble("C1")
    assert s.ndof == 20480
    per_row = s.nnz / s.ndof
    assert 7 < per_row < 12
    g = bs.Grid(3, 64, 64, 64)
    assert 5 * g.ncells == 1310720
    g5 = spec.CONFIGS["C5"]
    assert 5 * g5["nx"] * g5["ny"] * g5["nz"] == 51_200_000
