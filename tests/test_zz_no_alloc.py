"""The allocation-free Arnoldi dot entry point against the regular one (collected last).

bgs_arnoldi_dots_noalloc serves callers that cannot allocate device memory when they need the
dots (their device memory is fully pre-reserved by their own pool manager, or their host forbids
allocation after start-up).  It must give the same results as bgs_arnoldi_dots, call after call,
although every call reuses one fixed scratch array inside the library, and after its first call on
a device it must not change the device's free memory."""
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
    # two calls in a row, different shapes; the first needs more blocks than the fixed scratch
    # serves (250,001 rows: 489 blocks), so the grid is capped there
    for n, cnt in ((250_001, 37), (4_099, 64)):
        ld = n + 1
        V = torch.from_numpy(rng.standard_normal((cnt, ld))).cuda()
        w = torch.from_numpy(rng.standard_normal(n)).cuda()
        h_ref = torch.zeros(cnt + 1, dtype=torch.float64, device="cuda")
        h_new = torch.full((cnt + 1,), np.nan, dtype=torch.float64, device="cuda")
        assert bgs.bgs_arnoldi_dots(V, ld, cnt, w, n, h_ref) == 0
        assert bgs.bgs_arnoldi_dots_noalloc(V, ld, cnt, w, n, h_new) == 0
        torch.cuda.synchronize()
        a, b = h_ref.cpu().numpy(), h_new.cpu().numpy()
        # FP64 sums of n products in another fixed order: |diff| <= 4 n eps sum |v w|, as for the
        # FP64 dot tests of the regular entry point
        scale = np.concatenate([np.abs(V.cpu().numpy()[:, :n]) @ np.abs(w.cpu().numpy()), [b[-1]]])
        assert np.all(np.abs(a - b) <= 4 * n * np.finfo(float).eps * scale)


def test_noalloc_calls_after_the_first_leave_device_memory_unchanged(bgs):
    rng = np.random.default_rng(12)
    n, cnt = 1_000_003, 20
    ld = n + 1
    V = torch.from_numpy(rng.standard_normal((cnt, ld))).cuda()
    w = torch.from_numpy(rng.standard_normal(n)).cuda()
    h1 = torch.zeros(cnt + 1, dtype=torch.float64, device="cuda")
    h2 = torch.zeros(cnt + 1, dtype=torch.float64, device="cuda")
    assert bgs.bgs_arnoldi_dots_noalloc(V, ld, cnt, w, n, h1) == 0   # first call on this device (set-up)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert bgs.bgs_arnoldi_dots_noalloc(V, ld, cnt, w, n, h2) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(h1, h2)          # same kernels, same order: the same bits every call


def test_noalloc_rejects_invalid_arguments(bgs):
    n = 1024
    V = torch.zeros((65, n), dtype=torch.float64, device="cuda")
    w = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    h = torch.zeros(66, dtype=torch.float64, device="cuda")
    assert bgs.bgs_arnoldi_dots_noalloc(V, n, 65, w, n, h) == bgs.INVALID_ARG        # more than 64 vectors
    assert bgs.bgs_arnoldi_dots_noalloc(V, n - 1, 3, w, n, h) == bgs.INVALID_ARG     # odd leading dimension
    assert bgs.bgs_arnoldi_dots_noalloc(V, n, 3, w[1:], n, h) == bgs.INVALID_ARG    # w only 8-byte aligned
