"""The allocation-free Arnoldi dot entry point against the regular one (collected last).

bgs_arnoldi_dots_noalloc serves callers that cannot allocate device memory when they need the
dots; it must give the same results as bgs_arnoldi_dots, call after call, although every call
reuses one fixed scratch array inside the library."""
import numpy as np
import pytest

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


def test_noalloc_dots_match_the_allocating_entry_point_twice(bgs):
    rng = np.random.default_rng(11)
    for n, cnt in ((250_001, 37), (4_099, 64)):            # two calls in a row, different shapes
        ld = n + 1
        V = torch.from_numpy(rng.standard_normal((cnt, ld))).cuda()
        w = torch.from_numpy(rng.standard_normal(n)).cuda()
        h_ref = torch.zeros(cnt + 1, dtype=torch.float64, device="cuda")
        h_new = torch.full((cnt + 1,), np.nan, dtype=torch.float64, device="cuda")
        assert bgs.bgs_arnoldi_dots(V, ld, cnt, w, n, h_ref) == 0
        assert bgs.bgs_arnoldi_dots_noalloc(V, ld, cnt, w, n, h_new) == 0
        torch.cuda.synchronize()
        a, b = h_ref.cpu().numpy(), h_new.cpu().numpy()
        # same kernels, same fixed summation order; tolerance as for the FP64 dot tests
        scale = np.concatenate([np.abs(V.cpu().numpy()[:, :n]) @ np.abs(w.cpu().numpy()), [b[-1]]])
        assert np.all(np.abs(a - b) <= 4 * n * np.finfo(float).eps * scale)


def test_noalloc_rejects_sizes_beyond_its_scratch(bgs):
    n = 1024
    V = torch.zeros((65, n), dtype=torch.float64, device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    h = torch.zeros(66, dtype=torch.float64, device="cuda")
    assert bgs.bgs_arnoldi_dots_noalloc(V, n, 65, w, n, h) == bgs.INVALID_ARG
    assert bgs.bgs_arnoldi_dots_noalloc(V, n - 1, 3, w, n, h) == bgs.INVALID_ARG
