"""A six-field test system: the five-field battery system plus a solid-phase species field whose
diagonal block is diagonal (uncoupled ODEs, the A_s of Sec. 2.2), coupled to c1 by diagonal blocks
in both directions.  Values are seeded; the extra field's right-hand side is uniform in [-1, 1]."""
import numpy as np

import battery_system as bs
from battery_system import spec

SOLID = 5


def _diag_csr(vals):
    n = len(vals)
    return bs.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.asarray(vals, dtype=np.float64),
                  n, n)


def six_field(grid, seed):
    s = bs.assemble(grid=grid, seed=seed)
    n = s.ncells
    u = bs.rng_uniform(seed, 11, np.arange(3 * n, dtype=np.uint64))
    V = grid.h ** grid.dim
    blocks = dict(s.blocks)
    blocks[(SOLID, SOLID)] = _diag_csr(V * (1.0 / spec.DT) * (1.0 + u[:n]))
    blocks[(SOLID, spec.C1)] = _diag_csr(-0.5 * V * (1.0 + u[n:2 * n]))
    blocks[(spec.C1, SOLID)] = _diag_csr(-0.5 * V * (1.0 + u[2 * n:]))
    b = np.concatenate([s.b, 2.0 * bs.rng_uniform(seed, 12, np.arange(n, dtype=np.uint64)) - 1.0])
    nested = [[blocks.get((r, c)) for c in range(6)] for r in range(6)]
    return nested, [n] * 6, b


def dense(nested, sizes):
    offs = np.concatenate([[0], np.cumsum(sizes)])
    M = np.zeros((offs[-1], offs[-1]))
    for r, row in enumerate(nested):
        for c, B in enumerate(row):
            if B is not None:
                M[offs[r]:offs[r + 1], offs[c]:offs[c + 1]] = B.to_dense()
    return M
