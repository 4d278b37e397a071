"""One Gram-Schmidt pass of the FGMRES orthogonalisation (bgs_gram_schmidt_pass: the solver's own
kernels, with the products split between the FP64 pipe and exact fixed-point integer arithmetic)
against exact rational arithmetic.

Reference values are exact (fractions.Fraction over the doubles).  Bounds, u = 2^-53:
  * dots on the fixed-point side (vectors 3..7 of every 8): each thread's sum is exact up to the
    truncations of the scheme, 2^-62 ||w||_1 + 2^-55 max|w| ||v||_1 + n 2^-84 max|w|, then rounded
    and added in a fixed tree of at most 40 levels: T + 40 u sum_i |v_i w_i|;
  * dots on the FP64 side (vectors 0..2 of every 8) and ||w||^2: each thread adds its terms one by one
    before the same tree: (m + 40) u sum_i |v_i w_i|, m the terms per thread;
  * the update's odd rows (fixed point): 2^-62 sum_k |h_k| + 2^-55 max|h| sum_k |V_ik| + cnt 2^-84
    max|h|, then the sum's rounding and the subtraction's: + 2u (|s_i| + |w'_i|);
  * its even rows (FP64): (cnt + 1) u (|w_i| + sum_k |h_k V_ik|).
A systematic slip in the integer arithmetic (a dropped partial product, a wrong scale) moves the
fixed-point results by far more than these bounds.  A second case runs enough rows that every thread
rounds its fixed-point sums more than once (batches of 60 row pairs) and compares with the FP64-only
dots of bgs_arnoldi_dots."""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def bgs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_13079_gb300 import _build
    _build.build()
    import paper_2602_13079_gb300 as m
    return m


def _basis(rng, n, cnt):
    V = rng.standard_normal((cnt, n))
    V[:, ::97] = 0.0                      # exact zeros
    V[:, 5::211] *= 2.0 ** -40            # tiny entries (truncated at 2^-62)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    return V


def _w(rng, n):
    w = rng.choice([-1.0, 1.0], n) * np.exp2(rng.uniform(-30.0, 10.0, n))
    w[::89] = 0.0
    w[7] = 5e-324                         # a subnormal
    return w


def _run(bgs, V, w, ld):
    cnt, n = V.shape
    Vd = torch.zeros(cnt * ld, dtype=torch.float64, device="cuda")
    for k in range(cnt):
        Vd[k * ld:k * ld + n] = torch.from_numpy(V[k])
    wd = torch.from_numpy(w.copy()).cuda()
    h = torch.zeros(cnt + 1, dtype=torch.float64, device="cuda")
    nw = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert bgs.bgs_gram_schmidt_pass(Vd, ld, cnt, wd, n, h, nw) == 0
    torch.cuda.synchronize()
    return h.cpu().numpy(), wd.cpu().numpy(), float(nw.item())


@pytest.mark.parametrize("n,cnt", [(4099, 19), (1030, 64), (513, 1)])
def test_gram_schmidt_pass_against_exact_arithmetic(bgs, n, cnt):
    # odd n: the last row goes through the FP64 tail; 64 vectors: eight full chunks; one vector:
    # no fixed-point dot at all (vector 0 of a chunk is on the FP64 side)
    rng = np.random.default_rng(13 + cnt)
    ld = n + (n & 1)
    V, w = _basis(rng, n, cnt), _w(rng, n)
    h, wout, nw = _run(bgs, V, w, ld)
    wf = [Fraction(float(x)) for x in w]
    absw = np.abs(w)
    threads = 256 * min(-(-(n // 2 + 1) // 256), 2 * torch.cuda.get_device_properties(0).multi_processor_count)
    m = 2 * -(-(n // 2) // threads) + 1
    for k in range(cnt):
        exact = sum(Fraction(float(V[k, i])) * wf[i] for i in range(n))
        s_abs = float(np.sum(np.abs(V[k]) * absw))
        err = abs(Fraction(float(h[k])) - exact)
        if k % 8 >= 3:
            bound = (2.0 ** -62 * absw.sum() + 2.0 ** -55 * absw.max() * np.abs(V[k]).sum()
                     + n * 2.0 ** -84 * absw.max() + 40 * U * s_abs)
        else:
            bound = (m + 40) * U * s_abs
        assert float(err) <= bound, (k, float(err), bound)
    exact_nw = sum(x * x for x in wf)
    assert abs(float(Fraction(float(h[cnt])) - exact_nw)) <= (m + 40) * U * float(exact_nw)
    # the update with the returned h
    hf = [Fraction(float(x)) for x in h[:cnt]]
    habs = np.abs(h[:cnt])
    for i in range(n):
        s = sum(hf[k] * Fraction(float(V[k, i])) for k in range(cnt))
        exact = wf[i] - s
        err = float(abs(Fraction(float(wout[i])) - exact))
        t = float(np.sum(habs * np.abs(V[:, i])))
        if i % 2 == 1 and i < n - 1:
            bound = (2.0 ** -62 * habs.sum() + 2.0 ** -55 * habs.max() * np.abs(V[:, i]).sum()
                     + cnt * 2.0 ** -84 * habs.max() + 2 * U * (abs(float(s)) + abs(float(exact))))
        else:
            bound = (cnt + 1) * U * (absw[i] + t)
        assert err <= bound, (i, err, bound)
    ref_nw = float(np.sum(wout * wout))
    assert abs(nw - ref_nw) <= (m + 40) * U * ref_nw


def test_gram_schmidt_pass_out_of_range_basis_gives_nan(bgs):
    rng = np.random.default_rng(14)
    n, cnt = 1024, 8
    V, w = _basis(rng, n, cnt), rng.standard_normal(n)
    V[3, 5] = 2.5                          # vector 3 is on the fixed-point side; row 5 is odd
    h, wout, _ = _run(bgs, V, w, n)
    assert np.isnan(h[3]) and np.all(np.isfinite(h[[0, 1, 2, 4, 5, 6, 7]]))
    assert np.all(np.isnan(wout))          # every row subtracts h[3] V_3
    w2 = w.copy()
    w2[10] = np.inf
    h2, _, _ = _run(bgs, _basis(rng, n, cnt), w2, n)
    assert not np.any(np.isfinite(h2))


def test_gram_schmidt_pass_many_batches_matches_fp64_dots(bgs):
    # the dots run 2 * SMs blocks of 256 threads: 180 row pairs per thread, so every thread rounds
    # its fixed-point sums three times (batches of 60 pairs)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 2 * 60 * 4 * sms * 256 * 3 // 2 + 2
    cnt = 9
    g = torch.Generator(device="cuda").manual_seed(5)
    V = torch.randn(cnt, n, dtype=torch.float64, device="cuda", generator=g)
    V /= V.norm(dim=1, keepdim=True)
    w = torch.randn(n, dtype=torch.float64, device="cuda", generator=g) * torch.exp2(
        torch.randint(-20, 20, (n,), device="cuda", generator=g).double())
    h_fp = torch.zeros(cnt + 1, dtype=torch.float64, device="cuda")
    assert bgs.bgs_arnoldi_dots(V, n, cnt, w, n, h_fp) == 0
    w2 = w.clone()
    h = torch.zeros(cnt + 1, dtype=torch.float64, device="cuda")
    nw = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert bgs.bgs_gram_schmidt_pass(V, n, cnt, w2, n, h, nw) == 0
    s_abs = (V.abs() * w.abs()).sum(dim=1)
    m = 2 * -(-(n // 2) // (2 * sms * 256)) + 80
    bound = 2 * (m + 40) * U * s_abs + 2.0 ** -62 * w.abs().sum() + 2.0 ** -55 * w.abs().max() * V.abs().sum(dim=1)
    assert torch.all((h[:cnt] - h_fp[:cnt]).abs() <= bound)
    assert abs(float(h[cnt] - h_fp[cnt])) <= 2 * (m + 40) * U * float(h_fp[cnt])
    # the update against w - V^T h in FP64 (torch), row by row
    hk = h[:cnt]
    ref = w - hk @ V
    t = w.abs() + hk.abs() @ V.abs()
    bound = (2 * (cnt + 2) * U * t + 2.0 ** -62 * float(hk.abs().sum())
             + 2.0 ** -55 * float(hk.abs().max()) * V.abs().sum(dim=0) + 4 * U * ref.abs())
    assert torch.all((w2 - ref).abs() <= bound)
    assert abs(float(nw) - float(w2 @ w2)) <= 2 * (m + 40) * U * float(w2 @ w2)
