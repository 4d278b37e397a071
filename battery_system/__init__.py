"""Seeded synthetic coupled systems for the block Gauss-Seidel solve.

This module is the input generator that the CPU oracle, the tests and the
benchmark all draw from.  It holds no part of the solver: it assembles the
five-field layered battery system (phi_s, phi_e, p, c1, c2) as a 5 x 5 grid of
CSR blocks plus a right-hand side, from per-cell random coefficients drawn by a
counter-based generator (SplitMix64, Steele/Lea/Flood 2014).  The structure
follows the paper's description of the coupled electrochemical physics
(Sec. 1.1, Eqs. solid-phase-voltage ... stefan-maxwell) and its block splitting
(Sec. 2.2, Eq. block-splitting); the numbers are the readings in ``spec``.

Discretisation: cell-centred finite volumes on a uniform grid of spacing
h = 1/nx, cell volume V = h^d, face transmissibility T = h^(d-2) * 2ab/(a+b)
(harmonic mean of the two cell coefficients).  Cell index = i + nx*(j + ny*k);
every CSR row lists its columns in increasing order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import spec

_MASK64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


# --------------------------------------------------------------------------------------------
# Counter-based random numbers: element c of the SplitMix64 sequence started at key(seed, stream)
# --------------------------------------------------------------------------------------------
def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _mix64_int(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def rng_u64(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output number ``counter`` (0-based) of the sequence whose state starts at
    key = mix64(seed * 256 + stream): out = mix64(key + (counter + 1) * gamma)."""
    key = np.uint64(_mix64_int(seed * 256 + stream))
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = key + (c + np.uint64(1)) * np.uint64(_GAMMA)
        return _mix64_np(state)


def rng_uniform(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """U(0, 1]: ((x >> 11) + 1) * 2^-53."""
    x = rng_u64(seed, stream, counter)
    return ((x >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * (2.0 ** -53)


def rng_normal(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """Standard normal by Box-Muller from the uniforms 2c and 2c+1."""
    c = np.asarray(counter, dtype=np.uint64)
    u1 = rng_uniform(seed, stream, c * np.uint64(2))
    u2 = rng_uniform(seed, stream, c * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------------------------
# Grid and stencil slots
# --------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Grid:
    dim: int
    nx: int
    ny: int
    nz: int

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def h(self) -> float:
        return 1.0 / self.nx

    def ijk(self):
        c = np.arange(self.ncells, dtype=np.int64)
        i = c % self.nx
        j = (c // self.nx) % self.ny
        k = c // (self.nx * self.ny)
        return i, j, k

    def slots(self):
        """Off-diagonal stencil slots in increasing column order, with the diagonal slot index.

        Returns (offsets, axes, sides, diag_slot): slot s couples cell c with c + offsets[s]
        across the face on axis axes[s] (0 x, 1 y, 2 z), side -1 or +1."""
        if self.dim == 2:
            offs = [-self.nx, -1, 0, 1, self.nx]
            axes = [1, 0, -1, 0, 1]
            sides = [-1, -1, 0, 1, 1]
            return offs, axes, sides, 2
        nxy = self.nx * self.ny
        offs = [-nxy, -self.nx, -1, 0, 1, self.nx, nxy]
        axes = [2, 1, 0, -1, 0, 1, 2]
        sides = [-1, -1, -1, 0, 1, 1, 1]
        return offs, axes, sides, 3

    def neighbour_valid(self, axis: int, side: int) -> np.ndarray:
        i, j, k = self.ijk()
        coord, n = [(i, self.nx), (j, self.ny), (k, self.nz)][axis]
        return (coord > 0) if side < 0 else (coord < n - 1)


def harmonic_face(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """2ab/(a+b), evaluated as ((2a) b) / (a + b)."""
    return 2.0 * a * b / (a + b)


@dataclasses.dataclass
class SlotBlock:
    """A block stored as per-row slots (ncells x S) in increasing column order."""
    cols: np.ndarray     # int64 (n, S)
    vals: np.ndarray     # float64 (n, S)
    valid: np.ndarray    # bool (n, S)

    def to_csr(self):
        counts = self.valid.sum(axis=1)
        rowptr = np.zeros(self.valid.shape[0] + 1, dtype=np.int64)
        np.cumsum(counts, out=rowptr[1:])
        col = self.cols[self.valid]
        val = self.vals[self.valid]
        return CSR(rowptr.astype(np.int32), col.astype(np.int32), np.ascontiguousarray(val, dtype=np.float64),
                   self.valid.shape[0], self.valid.shape[0])


@dataclasses.dataclass
class CSR:
    rowptr: np.ndarray   # int32 (nrows + 1)
    col: np.ndarray      # int32 (nnz)
    val: np.ndarray      # float64 (nnz)
    nrows: int
    ncols: int

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols))
        rows = np.repeat(np.arange(self.nrows), np.diff(self.rowptr))
        d[rows, self.col] = self.val
        return d

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.nrows), np.diff(self.rowptr))
        return np.bincount(rows, weights=self.val * x[self.col], minlength=self.nrows)


def _stencil_block(grid: Grid, coef_axes, extra_diag=None) -> SlotBlock:
    """Diffusion stencil -div(coef grad u): off-diagonal -T, diagonal sum of T over the interior
    faces in slot order, then ``extra_diag`` (a list of per-cell arrays added in order)."""
    n = grid.ncells
    offs, axes, sides, dslot = grid.slots()
    S = len(offs)
    c = np.arange(n, dtype=np.int64)
    cols = np.empty((n, S), dtype=np.int64)
    vals = np.zeros((n, S))
    valid = np.zeros((n, S), dtype=bool)
    hfac = grid.h ** (grid.dim - 2)
    diag = np.zeros(n)
    for s in range(S):
        if s == dslot:
            cols[:, s] = c
            valid[:, s] = True
            continue
        ok = grid.neighbour_valid(axes[s], sides[s])
        nb = np.where(ok, c + offs[s], c)
        a = coef_axes[axes[s]]
        t = hfac * harmonic_face(a, a[nb])
        t = np.where(ok, t, 0.0)
        cols[:, s] = nb
        vals[:, s] = -t
        valid[:, s] = ok
        diag = diag + t
    for e in (extra_diag or []):
        diag = diag + e
    vals[:, dslot] = diag
    return SlotBlock(cols, vals, valid)


def _point_block(n: int, values: np.ndarray, mask: np.ndarray) -> CSR:
    counts = mask.astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    rows = np.nonzero(mask)[0]
    return CSR(rowptr.astype(np.int32), rows.astype(np.int32), np.ascontiguousarray(values[mask]), n, n)


@dataclasses.dataclass
class CoupledSystem:
    name: str
    grid: Grid
    seed: int
    blocks: dict          # (row field, col field) -> CSR; absent = zero block
    b: np.ndarray         # field-blocked right-hand side, length 5 * ncells
    layer: np.ndarray     # per-cell layer id (0 anode, 1 separator, 2 cathode)
    collector: np.ndarray  # cells on the unit-current (collector) face
    dirichlet: np.ndarray  # cells on the Dirichlet face
    params: dict

    @property
    def ncells(self) -> int:
        return self.grid.ncells

    @property
    def field_sizes(self):
        return [self.grid.ncells] * spec.NFIELDS

    @property
    def ndof(self) -> int:
        return spec.NFIELDS * self.grid.ncells

    @property
    def nnz(self) -> int:
        return sum(b.nnz for b in self.blocks.values())

    def block_list(self):
        """Row-major F x F list of CSR or None."""
        F = spec.NFIELDS
        return [[self.blocks.get((r, c)) for c in range(F)] for r in range(F)]

    def full_dense(self) -> np.ndarray:
        n = self.ncells
        A = np.zeros((self.ndof, self.ndof))
        for (r, c), blk in self.blocks.items():
            A[r * n:(r + 1) * n, c * n:(c + 1) * n] = blk.to_dense()
        return A

    def full_csr(self) -> CSR:
        """The field-blocked full operator as one CSR (rows of field r list blocks (r, 0..4) in order)."""
        n = self.ncells
        F = spec.NFIELDS
        counts = np.zeros(self.ndof, dtype=np.int64)
        for (r, c), blk in self.blocks.items():
            counts[r * n:(r + 1) * n] += np.diff(blk.rowptr)
        rowptr = np.zeros(self.ndof + 1, dtype=np.int64)
        np.cumsum(counts, out=rowptr[1:])
        col = np.empty(int(rowptr[-1]), dtype=np.int32)
        val = np.empty(int(rowptr[-1]))
        cursor = rowptr[:-1].copy()
        for r in range(F):
            for c in range(F):
                blk = self.blocks.get((r, c))
                if blk is None:
                    continue
                lens = np.diff(blk.rowptr).astype(np.int64)
                start = np.repeat(cursor[r * n:(r + 1) * n], lens)
                within = np.arange(blk.nnz) - np.repeat(blk.rowptr[:-1].astype(np.int64), lens)
                col[start + within] = blk.col + c * n
                val[start + within] = blk.val
                cursor[r * n:(r + 1) * n] += lens
        return CSR(rowptr.astype(np.int32), col, val, self.ndof, self.ndof)

    def matvec(self, x: np.ndarray) -> np.ndarray:
        n = self.ncells
        y = np.zeros(self.ndof)
        for (r, c), blk in self.blocks.items():
            y[r * n:(r + 1) * n] += blk.matvec(x[c * n:(c + 1) * n])
        return y


def _layers(grid: Grid, stack: bool) -> np.ndarray:
    i, j, k = grid.ijk()
    if stack:
        return (3 * (k % spec.STACK_PERIOD)) // spec.STACK_PERIOD
    return np.minimum(2, (3 * i) // grid.nx)


def coefficient_fields(grid: Grid, seed: int, stack: bool, sigma_means=None, i0_scale=1.0):
    """Per-cell coefficients: lognormal (sigma_log 0.5) around the layer means, i0 ~ U[0.5, 2]."""
    n = grid.ncells
    c = np.arange(n, dtype=np.uint64)
    layer = _layers(grid, stack)
    sm = np.asarray(sigma_means if sigma_means is not None else spec.SIGMA_S_MEANS, dtype=np.float64)
    gs = np.exp(spec.LOG_SIGMA * rng_normal(seed, spec.STREAM_SIGMA, c))
    sigma = sm[layer] * gs
    kappa = spec.KAPPA_E_MEAN * np.exp(spec.LOG_SIGMA * rng_normal(seed, spec.STREAM_KAPPA, c))
    kx = spec.PERM_MEAN * np.exp(spec.LOG_SIGMA * rng_normal(seed, spec.STREAM_PERM, c))
    d1 = spec.DIFF_MEANS[0] * np.exp(spec.LOG_SIGMA * rng_normal(seed, spec.STREAM_D1, c))
    d2 = spec.DIFF_MEANS[1] * np.exp(spec.LOG_SIGMA * rng_normal(seed, spec.STREAM_D2, c))
    lo, hi = spec.I0_RANGE
    i0 = lo + (hi - lo) * rng_uniform(seed, spec.STREAM_I0, c)
    i0 = np.where(layer == 1, 0.0, i0) * i0_scale
    return dict(layer=layer, sigma=sigma, sigma_shape=gs, kappa=kappa, kx=kx, d1=d1, d2=d2, i0=i0)


def assemble(name: str = "C1", seed: int = 1, grid: Grid | None = None, stack: bool | None = None,
             sigma_means=None, i0_scale: float = 1.0) -> CoupledSystem:
    """Assemble the coupled five-field system of a named workload (or an explicit grid).

    Row equations (all integrated over the cell, j_i = V k_i (phi_s - phi_e - U' c1) in the
    electrodes, k_i = a i0_i alpha F / (R T)):
      phi_s: sum_f T_sigma (phi_s_i - phi_s_n) + j = V f_s; Dirichlet phi_s = 0 on the first
             collector face adds 2 h^(d-2) sigma_i; the unit current on the far face adds h^(d-1) to b.
      phi_e: sum_f T_kappa (.) + V (tau/dt) phi_e - j = V f_e
      p:     sum_f T_K (.) + V (s/dt) p - gamma_p j = V f_p
      c_m:   V c_m / dt + sum_f T_Dm (.) + upwind advection by the Darcy flux of p0 = 1 - x
             + c0_m sum_f T_K (p_i - p_n) + V eps (c_m - c_other) - gamma_m j = V f_c
    """
    if grid is None:
        cfg = spec.CONFIGS[name]
        grid = Grid(cfg["dim"], cfg["nx"], cfg["ny"], cfg["nz"])
        stack = cfg["stack"] if stack is None else stack
    stack = bool(stack)
    n = grid.ncells
    d = grid.dim
    h = grid.h
    V = h ** d
    hfac = h ** (d - 2)
    hface = h ** (d - 1)
    co = coefficient_fields(grid, seed, stack, sigma_means, i0_scale)
    layer = co["layer"]
    i, j, k = grid.ijk()
    if stack:
        dir_mask = k == 0
        col_mask = k == grid.nz - 1
    else:
        dir_mask = i == 0
        col_mask = i == grid.nx - 1

    kbv = spec.bv_rate_constant() * co["i0"]       # k_i (0 in the separator)
    elec = kbv > 0.0
    Vk = V * kbv
    U = spec.DUDC

    def iso(a):
        return [a, a, a]

    kz = co["kx"] * (spec.PERM_Z_RATIO if d == 3 else 1.0)
    perm = [co["kx"], co["kx"], kz]
    blocks = {}

    # phi_s
    dir_term = np.where(dir_mask, 2.0 * hfac * co["sigma"], 0.0)
    blocks[(0, 0)] = _stencil_block(grid, iso(co["sigma"]), [dir_term, Vk]).to_csr()
    # phi_e
    blocks[(1, 1)] = _stencil_block(grid, iso(co["kappa"]), [np.full(n, V * spec.TAU_OVER_DT), Vk]).to_csr()
    # p
    blocks[(2, 2)] = _stencil_block(grid, perm, [np.full(n, V * spec.STORAGE_OVER_DT)]).to_csr()

    # species: diffusion + upwind advection along +x + mass + cross coupling + BV diagonal term
    offs, axes, sides, dslot = grid.slots()
    xm_slot = [s for s in range(len(offs)) if axes[s] == 0 and sides[s] < 0][0]
    ok_xm = grid.neighbour_valid(0, -1)
    ok_xp = grid.neighbour_valid(0, +1)
    cidx = np.arange(n, dtype=np.int64)
    kx = co["kx"]
    # outflow through the +x face: interior faces use the harmonic K, the boundary face K_x,i
    f_out = np.where(ok_xp, hface * harmonic_face(kx, kx[np.where(ok_xp, cidx + 1, cidx)]), hface * kx)
    f_in = np.where(ok_xm, hface * harmonic_face(kx, kx[np.where(ok_xm, cidx - 1, cidx)]), 0.0)
    for m, (dm, field) in enumerate(((co["d1"], spec.C1), (co["d2"], spec.C2))):
        bv_diag = spec.GAMMA_C[m] * Vk * U
        sb = _stencil_block(grid, iso(dm), [f_out, np.full(n, V / spec.DT), np.full(n, V * spec.EPS_CROSS), bv_diag])
        sb.vals[:, xm_slot] = sb.vals[:, xm_slot] - f_in
        blocks[(field, field)] = sb.to_csr()
        # Newton term c0_m * (K-Laplacian) in block (c_m, p)
        lk = _stencil_block(grid, perm)
        lk.vals = spec.C0[m] * lk.vals
        blocks[(field, spec.PRESS)] = lk.to_csr()
    cross = np.full(n, -V * spec.EPS_CROSS)
    allm = np.ones(n, dtype=bool)
    blocks[(spec.C1, spec.C2)] = _point_block(n, cross, allm)
    blocks[(spec.C2, spec.C1)] = _point_block(n, cross, allm)

    # Butler-Volmer point couplings (electrode cells only)
    blocks[(0, 1)] = _point_block(n, -Vk, elec)
    blocks[(0, 3)] = _point_block(n, -Vk * U, elec)
    blocks[(1, 0)] = _point_block(n, -Vk, elec)
    blocks[(1, 3)] = _point_block(n, Vk * U, elec)
    blocks[(2, 0)] = _point_block(n, -spec.GAMMA_P * Vk, elec)
    blocks[(2, 1)] = _point_block(n, spec.GAMMA_P * Vk, elec)
    blocks[(2, 3)] = _point_block(n, spec.GAMMA_P * Vk * U, elec)
    if spec.GAMMA_C[0] != 0.0:
        blocks[(3, 0)] = _point_block(n, -spec.GAMMA_C[0] * Vk, elec)
        blocks[(3, 1)] = _point_block(n, spec.GAMMA_C[0] * Vk, elec)
    if spec.GAMMA_C[1] != 0.0:
        blocks[(4, 0)] = _point_block(n, -spec.GAMMA_C[1] * Vk, elec)
        blocks[(4, 1)] = _point_block(n, spec.GAMMA_C[1] * Vk, elec)

    # right-hand side: V f with f ~ U[-1, 1] per DOF (counter = global DOF index)
    dof = np.arange(spec.NFIELDS * n, dtype=np.uint64)
    b = V * (2.0 * rng_uniform(seed, spec.STREAM_RHS, dof) - 1.0)
    b[:n] = b[:n] + np.where(col_mask, hface, 0.0)

    return CoupledSystem(name=name, grid=grid, seed=seed, blocks=blocks, b=b, layer=layer,
                         collector=np.nonzero(col_mask)[0], dirichlet=np.nonzero(dir_mask)[0],
                         params=dict(co, stack=stack, h=h, V=V))


def poisson_dirichlet(dim: int, n: int, coef: float = 1.0):
    """Single-field -div(coef grad u) on the unit square/cube with homogeneous Dirichlet on every
    face (half-cell distance: 2 h^(d-2) coef per boundary face).  Returns (CSR, cell centres)."""
    grid = Grid(dim, n, n, n if dim == 3 else 1)
    c = np.full(grid.ncells, float(coef))
    i, j, k = grid.ijk()
    hfac = grid.h ** (dim - 2)
    extra = []
    for coord, m in ((i, n), (j, n)) + (((k, n),) if dim == 3 else ()):
        extra.append(np.where(coord == 0, 2.0 * hfac * c, 0.0))
        extra.append(np.where(coord == m - 1, 2.0 * hfac * c, 0.0))
    A = _stencil_block(grid, [c, c, c], extra).to_csr()
    centres = [(i + 0.5) * grid.h, (j + 0.5) * grid.h] + ([(k + 0.5) * grid.h] if dim == 3 else [])
    return A, centres, grid


def transpose_csr(A: CSR) -> CSR:
    """Plain transpose (rows sorted), used by the tests to build adjoint inputs."""
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    order = np.lexsort((rows, A.col))
    counts = np.bincount(A.col, minlength=A.ncols)
    rowptr = np.zeros(A.ncols + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(rowptr.astype(np.int32), rows[order].astype(np.int32), A.val[order].copy(), A.ncols, A.nrows)
