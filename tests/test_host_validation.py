"""bgs_create checks its arguments on the host before any CUDA call, so these run without a GPU:
every malformed shape, order or option returns BGS_INVALID_ARG and leaves the handle NULL, while
the same call with valid arguments passes the checks (and then needs a device)."""
import ctypes as C
import os
import shutil

import numpy as np
import pytest

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def bgs():
    from paper_2602_13079_gb300 import _build
    _build.build()
    import paper_2602_13079_gb300 as m
    return m


def _identity(n):
    return (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))


class System:
    """Two fields of 3 and 2 rows, identity diagonal blocks, zero couplings (host arrays)."""

    def __init__(self, bgs):
        self.bgs = bgs
        self.F = 2
        self.sizes = [3, 2]
        self.order = [0, 1]
        self.arrays = {(0, 0): _identity(3), (1, 1): _identity(2)}
        self.shape = {}
        self.raw = {}   # (r, c) -> (nrows, ncols, nnz, rowptr, col, val) passed as given

    def call(self, options=None, F=None, out=True):
        b = self.bgs
        F = self.F if F is None else F
        blocks = (b.bgs_csr * max(F * F, 1))()
        for (r, c), (rp, ci, v) in self.arrays.items():
            if r >= F or c >= F:
                continue
            nr, nc = self.shape.get((r, c), (self.sizes[r], self.sizes[c]))
            blocks[r * F + c] = b.bgs_csr(nr, nc, len(ci), rp.ctypes.data, ci.ctypes.data if len(ci) else None,
                                          v.ctypes.data if len(v) else None)
        for (r, c), f in self.raw.items():
            blocks[r * F + c] = b.bgs_csr(*f)
        sizes = (C.c_int64 * max(F, 1))(*self.sizes[:F])
        order = (C.c_int * max(F, 1))(*self.order[:F])
        h = C.c_void_p()
        opts = options if options is not None else b.bgs_default_options()
        st = b.lib().bgs_create(C.byref(h) if out else None, F, sizes, blocks, order, C.byref(opts), None)
        return st, h


def test_valid_arguments_pass_the_host_checks(bgs):
    st, h = System(bgs).call()
    assert st != bgs.INVALID_ARG
    if st == bgs.OK:                     # a GPU is present
        assert h.value
        bgs.lib().bgs_destroy(h)
    else:
        assert st in (bgs.CUDA_ERROR, bgs.OOM) and not h.value


@pytest.mark.parametrize("defect", ["F0", "F9", "no_out", "dup_order", "order_range", "size0", "zero_diag",
                                    "rows_mismatch", "cols_mismatch", "null_col"])
def test_malformed_shapes(bgs, defect):
    s = System(bgs)
    kw = {}
    if defect == "F0":
        kw["F"] = 0
    elif defect == "F9":
        kw["F"] = 9
    elif defect == "no_out":
        kw["out"] = False
    elif defect == "dup_order":
        s.order = [0, 0]
    elif defect == "order_range":
        s.order = [0, 2]
    elif defect == "size0":
        s.sizes = [3, 0]
    elif defect == "zero_diag":
        del s.arrays[(1, 1)]
    elif defect == "rows_mismatch":
        s.shape[(0, 0)] = (2, 3)
    elif defect == "cols_mismatch":
        s.shape[(1, 1)] = (2, 3)
    elif defect == "null_col":
        # a coupling block that claims one stored entry but passes no column or value array
        rp = np.array([0, 1, 1, 1], dtype=np.int32)
        s.keep = rp
        s.raw[(0, 1)] = (3, 2, 1, rp.ctypes.data, None, None)
    st, h = s.call(**kw)
    assert st == bgs.INVALID_ARG and not h.value


OPTION_DEFECTS = [
    dict(restart=0), dict(restart=64), dict(maxit=0), dict(rtol=0.0), dict(max_levels=0), dict(max_levels=17),
    dict(precision=2), dict(power_iters=0), dict(cheb_ratio=1.0), dict(cheb_boost=0.0), dict(reorth_eta=-1.0),
    dict(jacobi=2), dict(ilu_rows=0), dict(ilu_rows=9000), dict(cheb_ellipse=2), dict(max_coarse=0),
    dict(cheb_degree=[0, 2]), dict(theta=[-1.0, 0.0]), dict(subsolver=[3, 0]),
    dict(ngroups=3), dict(ngroups=1, group_end=[1]), dict(ngroups=2, group_end=[1, 1]),
    dict(ngroups=1, group_end=[2], inner_restart=0), dict(ngroups=1, group_end=[2], inner_rtol=0.0),
]


@pytest.mark.parametrize("bad", OPTION_DEFECTS, ids=[",".join(f"{k}={v}" for k, v in d.items()) for d in OPTION_DEFECTS])
def test_malformed_options(bgs, bad):
    st, h = System(bgs).call(options=bgs.bgs_default_options(**bad))
    assert st == bgs.INVALID_ARG and not h.value


@pytest.mark.parametrize("entry", ["bgs_arnoldi_dots", "bgs_arnoldi_dots_noalloc"])
def test_arnoldi_dots_reject_misaligned_vectors_on_the_host(bgs, entry):
    """The dot kernel reads V and w as 16-byte pairs: a pointer that is only 8-byte aligned (a view
    such as x[1:]) is refused on the host with BGS_INVALID_ARG, before any CUDA call, so these
    addresses (never dereferenced) are safe to pass without a GPU."""
    f = getattr(bgs.lib(), entry)
    base = 1 << 20                      # 16-byte aligned stand-in addresses, never dereferenced
    n, cnt, ld = 1000, 3, 1000
    for V, w in ((base + 8, base), (base, base + 8), (base + 8, base + 24)):
        assert f(V, ld, cnt, w, n, base, None) == bgs.INVALID_ARG
    # the other host checks, for completeness: odd leading dimension, basis size out of range
    assert f(base, ld + 1, cnt, base, n, base, None) == bgs.INVALID_ARG
    assert f(base, ld, 65, base, n, base, None) == bgs.INVALID_ARG
    assert f(base, n - 2, cnt, base, n, base, None) == bgs.INVALID_ARG


def test_gram_schmidt_pass_rejects_bad_arguments_on_the_host(bgs):
    """bgs_gram_schmidt_pass reads V and w as 16-byte pairs and takes 1..64 basis vectors: every
    malformed call returns BGS_INVALID_ARG on the host, before any CUDA call (these stand-in
    addresses are never dereferenced)."""
    f = bgs.lib().bgs_gram_schmidt_pass
    base = 1 << 20
    n, cnt, ld = 1000, 3, 1000
    ok = dict(V=base, ld=ld, cnt=cnt, w=base, n=n, h=base, nw=base)

    def call(**kw):
        a = dict(ok, **kw)
        return f(a["V"], a["ld"], a["cnt"], a["w"], a["n"], a["h"], a["nw"], None)

    for kw in ({"V": base + 8}, {"w": base + 8}, {"V": None}, {"w": None}, {"h": None}, {"nw": None},
               {"cnt": 0}, {"cnt": 65}, {"ld": ld + 1}, {"ld": n - 2}, {"n": 0}):
        assert call(**kw) == bgs.INVALID_ARG, kw
