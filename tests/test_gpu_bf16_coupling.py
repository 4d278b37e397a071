"""The BF16 coupling values of the mixed form, against their error bound.

Two fields whose diagonal blocks take the diagonal solve (subsolver 2, exact up to FP32 rounding)
isolate the coupling product of the mixed sweep: z_0 = D_0^-1 v_0 and z_1 = D_1^-1 (v_1 - L z_0),
with L stored in BF16 and the products summed in FP32.  BF16 rounding to nearest (8 significant
bits) moves each value by at most 2^-8 of itself, so against the exact FP64 result

    |dz_1,i| <= (2^-8 sum_j |L_ij z_0,j| + c u (|v_1,i| + sum_j |L_ij z_0,j|)) / d_1,i + c u |z_1,i|

with u = 2^-24 and c covering the FP32 roundings of the sum (k <= 8 terms), of z_0 and of the
diagonal solves.  The bound holds row by row; the measured worst ratio to it is printed, and the
largest error shows the BF16 rounding (it is far above FP32 rounding)."""
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


def _diag(d):
    n = len(d)
    return bs.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.asarray(d, dtype=np.float64),
                  n, n)


def test_bf16_coupling_error_bound(bgs):
    rng = np.random.default_rng(21)
    n, per_row = 4000, 6
    d0 = rng.uniform(1.0, 2.0, n)
    d1 = rng.uniform(1.0, 2.0, n)
    cols = np.sort(np.stack([rng.choice(n, size=per_row, replace=False) for _ in range(n)]), axis=1)
    vals = rng.uniform(-1.0, 1.0, (n, per_row))
    L = bs.CSR(np.arange(0, n * per_row + 1, per_row, dtype=np.int32), cols.ravel().astype(np.int32),
               vals.ravel(), n, n)
    nested = [[_diag(d0), None], [L, _diag(d1)]]
    g = bgs.Solver(nested, [n, n], [0, 1], subsolver=[2, 2], precision=1)
    g.setup()
    v = rng.standard_normal(2 * n)
    z = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    g.bgs_apply_preconditioner(torch.from_numpy(v).cuda(), z)
    zg = z.cpu().numpy()
    g.close()
    # exact FP64 sweep
    z0 = v[:n] / d0
    Lz = (vals * z0[cols]).sum(axis=1)
    z1 = (v[n:] - Lz) / d1
    u, c = 2.0 ** -24, 16.0
    absLz = (np.abs(vals) * np.abs(z0[cols])).sum(axis=1)
    bound = (2.0 ** -8 * absLz + c * u * (np.abs(v[n:]) + absLz)) / d1 + c * u * np.abs(z1)
    err1 = np.abs(zg[n:] - z1)
    assert np.all(np.abs(zg[:n] - z0) <= c * u * np.abs(z0))      # no coupling into field 0
    assert np.all(err1 <= bound)
    rel = np.linalg.norm(err1) / np.linalg.norm(z1)
    print(f"BF16 coupling: max error / bound {np.max(err1 / bound):.3f}, "
          f"||dz_1|| / ||z_1|| = {rel:.2e}, max |dz_1| / (2^-8 |L| |z_0| / d_1) = "
          f"{np.max(err1 / (2.0 ** -8 * absLz / d1)):.3f}")
    # the values really are BF16: the error is far above what FP32 values would leave
    assert np.max(err1 / (c * u * (absLz / d1 + np.abs(z1)))) > 10.0
