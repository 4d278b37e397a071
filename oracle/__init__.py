"""ctypes wrapper of the FP64 CPU oracle (bgs_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg use it; the library never does.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bgs_oracle.c")
_HDR = os.path.join(_HERE, "bgs_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Options(C.Structure):
    _fields_ = [("restart", C.c_int), ("maxit", C.c_int), ("rtol", C.c_double),
                ("cheb_degree", C.c_int * 8), ("theta", C.c_double * 8),
                ("max_coarse", C.c_int), ("max_levels", C.c_int),
                ("cheb_ratio", C.c_double), ("cheb_boost", C.c_double),
                ("power_iters", C.c_int), ("filter_diag", C.c_int), ("jacobi", C.c_int),
                ("subsolver", C.c_int * 8), ("ilu_rows", C.c_int), ("ngroups", C.c_int),
                ("group_end", C.c_int * 8), ("inner_restart", C.c_int), ("inner_maxit", C.c_int),
                ("inner_rtol", C.c_double), ("cheb_ellipse", C.c_int)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("status", C.c_int),
                ("rel_true_resid", C.c_double), ("rel_est_resid", C.c_double)]


class _CSR(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("nnz", C.c_int),
                ("rp", C.POINTER(C.c_int)), ("ci", C.POINTER(C.c_int)), ("v", C.POINTER(C.c_double))]


MAXL = 16


class _AMG(C.Structure):
    _fields_ = [("nlevels", C.c_int), ("A", C.POINTER(_CSR) * MAXL), ("P", C.POINTER(_CSR) * MAXL),
                ("R", C.POINTER(_CSR) * MAXL), ("agg", C.POINTER(C.c_int) * MAXL),
                ("strong", C.POINTER(C.c_uint8) * MAXL), ("nagg", C.c_int * MAXL),
                ("mis_rounds", C.c_int * MAXL), ("omega", C.c_double * MAXL),
                ("dinv", C.POINTER(C.c_double) * MAXL), ("lmax", C.c_double * MAXL),
                ("lmin", C.c_double * MAXL), ("lim", C.c_double * MAXL), ("degree", C.c_int), ("nc", C.c_int),
                ("lu", C.POINTER(C.c_double)), ("piv", C.POINTER(C.c_int)), ("status", C.c_int)]


class _ILU(C.Structure):
    _fields_ = [("rows", C.c_int), ("F", C.POINTER(_CSR)), ("status", C.c_int)]


class _BGS(C.Structure):
    _fields_ = [("F", C.c_int), ("sizes", C.c_int * 8), ("offs", C.c_int * 9), ("order", C.c_int * 8),
                ("pos", C.c_int * 8), ("blk", C.POINTER(_CSR) * 64), ("full", C.POINTER(_CSR)),
                ("amg", C.POINTER(_AMG) * 8), ("ilu", C.POINTER(_ILU) * 8),
                ("dgs", C.POINTER(C.c_double) * 8), ("opt", Options),
                ("status", C.c_int)]


APPLY_FN = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            P = C.POINTER(_CSR)
            L.or_csr_from.restype = P
            L.or_csr_from.argtypes = [C.c_int, C.c_int, i32p, i32p, f64p]
            L.or_csr_free.argtypes = [P]
            L.or_spmv.argtypes = [P, f64p, f64p]
            L.or_transpose.restype = P
            L.or_transpose.argtypes = [P]
            L.or_spgemm.restype = P
            L.or_spgemm.argtypes = [P, P]
            L.or_set_threads.restype = C.c_int
            L.or_set_threads.argtypes = [C.c_int]
            L.or_sum_prod.restype = C.c_double
            L.or_sum_prod.argtypes = [C.c_int, f64p, f64p]
            L.or_fmix32.restype = C.c_uint32
            L.or_fmix32.argtypes = [C.c_uint32]
            L.or_strength_flags.argtypes = [P, C.c_double, u8p]
            L.or_strength_graph.restype = P
            L.or_strength_graph.argtypes = [P, u8p]
            L.or_mis2.restype = C.c_int
            L.or_mis2.argtypes = [P, C.c_uint32, i32p]
            L.or_aggregate.restype = C.c_int
            L.or_aggregate.argtypes = [P, i32p, i32p]
            L.or_filter.argtypes = [P, u8p, C.c_int, f64p, f64p]
            L.or_power_lambda.restype = C.c_double
            L.or_power_lambda.argtypes = [P, f64p, C.c_int]
            L.or_smooth_prolongator.restype = P
            L.or_smooth_prolongator.argtypes = [P, f64p, i32p, C.c_int, C.c_double]
            L.or_chebyshev.argtypes = [P, f64p, C.c_double, C.c_double, C.c_int, f64p, f64p, C.c_int]
            L.or_skew_radius.restype = C.c_double
            L.or_skew_radius.argtypes = [P, C.c_int]
            L.or_chebyshev_ellipse.argtypes = [P, f64p, C.c_double, C.c_double, C.c_int, f64p, f64p, C.c_int]
            L.or_lu_factor.restype = C.c_int
            L.or_lu_factor.argtypes = [C.c_int, f64p, i32p]
            L.or_lu_solve.argtypes = [C.c_int, f64p, i32p, f64p, f64p]
            L.or_amg_setup.restype = C.POINTER(_AMG)
            L.or_amg_setup.argtypes = [P, C.c_double, C.c_int, C.POINTER(Options)]
            L.or_amg_free.argtypes = [C.POINTER(_AMG)]
            L.or_vcycle.argtypes = [C.POINTER(_AMG), f64p, f64p]
            L.or_amg_update.restype = C.c_int
            L.or_amg_update.argtypes = [C.POINTER(_AMG), f64p, C.POINTER(Options)]
            L.or_default_options.argtypes = [C.POINTER(Options)]
            L.or_ilu_setup.restype = C.POINTER(_ILU)
            L.or_ilu_setup.argtypes = [P, C.c_int]
            L.or_ilu_free.argtypes = [C.POINTER(_ILU)]
            L.or_ilu_apply.argtypes = [C.POINTER(_ILU), f64p, f64p]
            L.or_ilu_apply_transposed.argtypes = [C.POINTER(_ILU), f64p, f64p]
            L.or_bgs_create.restype = C.POINTER(_BGS)
            L.or_bgs_create.argtypes = [C.c_int, i32p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_void_p), i32p, i32p, C.POINTER(Options)]
            L.or_bgs_setup.restype = C.c_int
            L.or_bgs_setup.argtypes = [C.POINTER(_BGS)]
            L.or_bgs_update_values.restype = C.c_int
            L.or_bgs_update_values.argtypes = [C.POINTER(_BGS), C.POINTER(C.c_void_p)]
            L.or_bgs_free.argtypes = [C.POINTER(_BGS)]
            L.or_bgs_apply.argtypes = [C.POINTER(_BGS), f64p, f64p]
            L.or_bgs_apply_adjoint.argtypes = [C.POINTER(_BGS), f64p, f64p]
            L.or_bgs_solve.restype = C.c_int
            L.or_bgs_solve.argtypes = [C.POINTER(_BGS), f64p, f64p, C.POINTER(Info)]
            L.or_bgs_solve_adjoint.restype = C.c_int
            L.or_bgs_solve_adjoint.argtypes = [C.POINTER(_BGS), f64p, f64p, C.POINTER(Info)]
            L.or_full_spmv.argtypes = [C.POINTER(_BGS), f64p, f64p]
            L.or_fgmres.restype = C.c_int
            L.or_fgmres.argtypes = [C.c_int, APPLY_FN, C.c_void_p, APPLY_FN, C.c_void_p, f64p, f64p,
                                    C.c_int, C.c_int, C.c_double, C.POINTER(Info)]
        return _lib


# ---------------------------------------------------------------------------------------------
class CSR:
    """Host CSR (int32 indices, float64 values) returned by the oracle."""

    def __init__(self, rowptr, col, val, nrows, ncols):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.nrows, self.ncols = int(nrows), int(ncols)

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_dense(self):
        d = np.zeros((self.nrows, self.ncols))
        rows = np.repeat(np.arange(self.nrows), np.diff(self.rowptr))
        d[rows, self.col] = self.val
        return d


def _to_c(A):
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    v = np.ascontiguousarray(A.val, dtype=np.float64)
    return lib().or_csr_from(int(A.nrows), int(A.ncols), rp, ci, v)


def _from_c(p, free=True):
    c = p.contents
    n, m, nnz = c.n, c.m, c.nnz
    rp = np.ctypeslib.as_array(c.rp, shape=(n + 1,)).copy()
    ci = np.ctypeslib.as_array(c.ci, shape=(max(nnz, 1),))[:nnz].copy()
    v = np.ctypeslib.as_array(c.v, shape=(max(nnz, 1),))[:nnz].copy()
    if free:
        lib().or_csr_free(p)
    return CSR(rp, ci, v, n, m)


class _Handle:
    def __init__(self, A):
        self.p = _to_c(A)

    def __del__(self):
        try:
            lib().or_csr_free(self.p)
        except Exception:
            pass


def spmv(A, x):
    h = _Handle(A)
    y = np.zeros(A.nrows)
    lib().or_spmv(h.p, np.ascontiguousarray(x, dtype=np.float64), y)
    return y


def transpose(A):
    h = _Handle(A)
    return _from_c(lib().or_transpose(h.p))


def spgemm(A, B):
    ha, hb = _Handle(A), _Handle(B)
    return _from_c(lib().or_spgemm(ha.p, hb.p))


def set_threads(n: int = 0) -> int:
    """Host threads for the oracle's row loops (0 keeps the current count); returns the count in use.
    Results do not depend on it."""
    return int(lib().or_set_threads(int(n)))


def sum_prod(a, b) -> float:
    """sum_i a_i b_i in the oracle's fixed block order (blocks of 4096 terms left to right, then the
    block sums left to right)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return float(lib().or_sum_prod(int(a.size), a, b))


def fmix32(x: int) -> int:
    return int(lib().or_fmix32(x & 0xFFFFFFFF))


def mis_salt(level: int) -> int:
    return (level * 0x9E3779B9) & 0xFFFFFFFF


def strength_flags(A, theta):
    h = _Handle(A)
    s = np.zeros(max(A.nnz, 1), dtype=np.uint8)
    lib().or_strength_flags(h.p, float(theta), s)
    return s[:A.nnz]


def strength_graph(A, strong):
    h = _Handle(A)
    s = np.ascontiguousarray(np.concatenate([strong, [0]]).astype(np.uint8))
    return _from_c(lib().or_strength_graph(h.p, s))


def mis2(S, salt):
    h = _Handle(S)
    st = np.zeros(max(S.nrows, 1), dtype=np.int32)
    rounds = lib().or_mis2(h.p, salt & 0xFFFFFFFF, st)
    return st[:S.nrows], rounds


def aggregate(S, state):
    h = _Handle(S)
    agg = np.zeros(max(S.nrows, 1), dtype=np.int32)
    nagg = lib().or_aggregate(h.p, np.ascontiguousarray(np.concatenate([state, [0]]), dtype=np.int32), agg)
    return agg[:S.nrows], nagg


def filter_matrix(A, strong, filter_diag=1):
    h = _Handle(A)
    vF = np.zeros(max(A.nnz, 1))
    dF = np.zeros(max(A.nrows, 1))
    s = np.ascontiguousarray(np.concatenate([strong, [0]]).astype(np.uint8))
    lib().or_filter(h.p, s, int(filter_diag), vF, dF)
    return vF[:A.nnz], dF[:A.nrows]


def power_lambda(A, dinv, iters=10):
    h = _Handle(A)
    return float(lib().or_power_lambda(h.p, np.ascontiguousarray(dinv, dtype=np.float64), int(iters)))


def smooth_prolongator(AF, dinvF, agg, nagg, omega):
    h = _Handle(AF)
    return _from_c(lib().or_smooth_prolongator(h.p, np.ascontiguousarray(dinvF, dtype=np.float64),
                                               np.ascontiguousarray(agg, dtype=np.int32), int(nagg),
                                               float(omega)))


def chebyshev(A, dinv, lmin, lmax, deg, b, x0=None):
    h = _Handle(A)
    x = np.zeros(A.nrows) if x0 is None else np.array(x0, dtype=np.float64)
    lib().or_chebyshev(h.p, np.ascontiguousarray(dinv, dtype=np.float64), float(lmin), float(lmax), int(deg),
                       np.ascontiguousarray(b, dtype=np.float64), x, 1 if x0 is None else 0)
    return x


def skew_radius(A, iters=10):
    h = _Handle(A)                      # keep the C matrix alive across the call
    return lib().or_skew_radius(h.p, int(iters))


def chebyshev_ellipse(A, dinv, theta, c2, deg, b, x0=None):
    h = _Handle(A)
    x = np.zeros(A.nrows) if x0 is None else np.array(x0, dtype=np.float64)
    lib().or_chebyshev_ellipse(h.p, np.ascontiguousarray(dinv, dtype=np.float64), float(theta), float(c2), int(deg),
                               np.ascontiguousarray(b, dtype=np.float64), x, 1 if x0 is None else 0)
    return x


def lu_factor(a):
    n = a.shape[0]
    lu = np.ascontiguousarray(a, dtype=np.float64).copy()
    piv = np.zeros(max(n, 1), dtype=np.int32)
    st = lib().or_lu_factor(n, lu, piv)
    return lu, piv, st


def lu_solve(lu, piv, b):
    n = lu.shape[0]
    x = np.zeros(n)
    lib().or_lu_solve(n, lu, piv, np.ascontiguousarray(b, dtype=np.float64), x)
    return x


def dense_solve(a, b):
    """Dense LU with partial pivoting (oracle's own), used as the exact-solve pin."""
    lu, piv, st = lu_factor(a)
    if st != 0:
        raise RuntimeError("zero pivot")
    return lu_solve(lu, piv, b)


def default_options(**kw) -> Options:
    o = Options()
    lib().or_default_options(C.byref(o))
    for k, v in kw.items():
        if k in ("cheb_degree", "theta", "subsolver", "group_end"):
            arr = getattr(o, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(o, k, v)
    return o


class ILU:
    """DD(0)-ILU(0) on a square CSR matrix: subdomains of `rows` consecutive rows."""

    def __init__(self, A, rows, _ptr=None):
        if _ptr is not None:
            self.p, self._own = _ptr, False
        else:
            self._A = _Handle(A)
            self.p = lib().or_ilu_setup(self._A.p, int(rows))
            self._own = True

    def __del__(self):
        if getattr(self, "_own", False):
            try:
                lib().or_ilu_free(self.p)
            except Exception:
                pass

    @property
    def status(self):
        return self.p.contents.status

    def factors(self):
        """The subdomain-restricted pattern with L (unit, strictly lower) and U in place."""
        return _from_c(self.p.contents.F, free=False)

    def apply(self, r):
        z = np.zeros(self.p.contents.F.contents.n)
        lib().or_ilu_apply(self.p, np.ascontiguousarray(r, dtype=np.float64), z)
        return z

    def apply_transposed(self, r):
        z = np.zeros(self.p.contents.F.contents.n)
        lib().or_ilu_apply_transposed(self.p, np.ascontiguousarray(r, dtype=np.float64), z)
        return z


class AMG:
    """One SA-AMG hierarchy on a square CSR block."""

    def __init__(self, A, theta=0.04, degree=2, opts: Options | None = None, _ptr=None, _owner=None):
        if _ptr is not None:
            self.p, self._own, self._owner = _ptr, False, _owner
        else:
            self._A = _Handle(A)
            self._opts = opts or default_options()
            self.p = lib().or_amg_setup(self._A.p, float(theta), int(degree), C.byref(self._opts))
            self._own = True

    def update(self, values):
        """Numeric re-set-up with new level-0 values on the same pattern."""
        v = np.ascontiguousarray(values, dtype=np.float64)
        assert v.size == self.s.A[0].contents.nnz
        return lib().or_amg_update(self.p, v, C.byref(getattr(self, "_opts", None) or default_options()))

    def strong(self, l):
        nnz = self.s.A[l].contents.nnz
        return np.ctypeslib.as_array(self.s.strong[l], shape=(nnz,)).copy()

    def __del__(self):
        if getattr(self, "_own", False):
            try:
                lib().or_amg_free(self.p)
            except Exception:
                pass

    @property
    def s(self):
        return self.p.contents

    @property
    def nlevels(self):
        return self.s.nlevels

    @property
    def status(self):
        return self.s.status

    def level_matrix(self, l):
        return _from_c(self.s.A[l], free=False)

    def prolongator(self, l):
        return _from_c(self.s.P[l], free=False)

    def restriction(self, l):
        return _from_c(self.s.R[l], free=False)

    def aggregates(self, l):
        n = self.s.A[l].contents.n
        return np.ctypeslib.as_array(self.s.agg[l], shape=(n,)).copy()

    def nagg(self, l):
        return self.s.nagg[l]

    def omega(self, l):
        return self.s.omega[l]

    def mis_rounds(self, l):
        return self.s.mis_rounds[l]

    def dinv(self, l):
        n = self.s.A[l].contents.n
        return np.ctypeslib.as_array(self.s.dinv[l], shape=(n,)).copy()

    def cheb_bounds(self, l):
        return self.s.lmin[l], self.s.lmax[l]

    def cheb_imag(self, l):
        return self.s.lim[l]

    def sizes(self):
        return [self.s.A[l].contents.n for l in range(self.nlevels)]

    def vcycle(self, b):
        x = np.zeros(self.s.A[0].contents.n)
        lib().or_vcycle(self.p, np.ascontiguousarray(b, dtype=np.float64), x)
        return x


class BGS:
    """Block Gauss-Seidel preconditioned flexible GMRES on an F x F block system."""

    def __init__(self, blocks, sizes, order, opts: Options | None = None):
        F = len(sizes)
        self.F = F
        self.sizes = [int(s) for s in sizes]
        self.opts = opts or default_options()
        rps, cis, vs, nnzs = (C.c_void_p * (F * F))(), (C.c_void_p * (F * F))(), (C.c_void_p * (F * F))(), []
        self._keep = []
        for r in range(F):
            for c in range(F):
                B = blocks[r][c]
                k = r * F + c
                if B is None:
                    nnzs.append(0)
                    continue
                rp = np.ascontiguousarray(B.rowptr, dtype=np.int32)
                ci = np.ascontiguousarray(B.col, dtype=np.int32)
                v = np.ascontiguousarray(B.val, dtype=np.float64)
                self._keep += [rp, ci, v]
                rps[k], cis[k], vs[k] = rp.ctypes.data, ci.ctypes.data, v.ctypes.data
                nnzs.append(B.nnz)
        self.p = lib().or_bgs_create(F, np.array(self.sizes, dtype=np.int32), rps, cis, vs,
                                     np.array(nnzs, dtype=np.int32), np.array(order, dtype=np.int32),
                                     C.byref(self.opts))
        self._keep = None
        self.n = sum(self.sizes)

    def __del__(self):
        try:
            lib().or_bgs_free(self.p)
        except Exception:
            pass

    def setup(self):
        return lib().or_bgs_setup(self.p)

    def update_values(self, values):
        """values: F x F nested list of new value arrays (same patterns); None keeps a block's values."""
        F = self.F
        vs = (C.c_void_p * (F * F))()
        keep = []
        for r in range(F):
            for c in range(F):
                v = values[r][c]
                if v is None:
                    continue
                v = np.ascontiguousarray(v, dtype=np.float64)
                keep.append(v)
                vs[r * F + c] = v.ctypes.data
        return lib().or_bgs_update_values(self.p, vs)

    def amg(self, field):
        return AMG(None, _ptr=self.p.contents.amg[field], _owner=self)

    def ilu(self, field):
        return ILU(None, None, _ptr=self.p.contents.ilu[field])

    def apply(self, v):
        z = np.zeros(self.n)
        lib().or_bgs_apply(self.p, np.ascontiguousarray(v, dtype=np.float64), z)
        return z

    def apply_adjoint(self, v):
        z = np.zeros(self.n)
        lib().or_bgs_apply_adjoint(self.p, np.ascontiguousarray(v, dtype=np.float64), z)
        return z

    def full_matvec(self, x):
        y = np.zeros(self.n)
        lib().or_full_spmv(self.p, np.ascontiguousarray(x, dtype=np.float64), y)
        return y

    def full_matrix(self):
        return _from_c(self.p.contents.full, free=False)

    def solve(self, b):
        x = np.zeros(self.n)
        info = Info()
        lib().or_bgs_solve(self.p, np.ascontiguousarray(b, dtype=np.float64), x, C.byref(info))
        return x, info

    def solve_adjoint(self, g):
        lam = np.zeros(self.n)
        info = Info()
        lib().or_bgs_solve_adjoint(self.p, np.ascontiguousarray(g, dtype=np.float64), lam, C.byref(info))
        return lam, info


def fgmres(n, amul, prec, b, restart=50, maxit=1000, rtol=1e-8):
    """FGMRES with Python callbacks (small systems only)."""

    def wrap(f):
        def cb(_ctx, inp, out):
            xin = np.ctypeslib.as_array(inp, shape=(n,))
            xout = np.ctypeslib.as_array(out, shape=(n,))
            xout[:] = f(xin.copy())
        return APPLY_FN(cb)

    a_cb, p_cb = wrap(amul), wrap(prec)
    x = np.zeros(n)
    info = Info()
    lib().or_fgmres(n, a_cb, None, p_cb, None, np.ascontiguousarray(b, dtype=np.float64), x, restart, maxit,
                    rtol, C.byref(info))
    return x, info


def bgs_for_system(system, order=None, opts: Options | None = None, setup=True):
    """Convenience: oracle BGS over a battery_system.CoupledSystem."""
    o = BGS(system.block_list(), system.field_sizes, order if order is not None else list(range(5)), opts)
    if setup:
        st = o.setup()
        if st != 0:
            raise RuntimeError(f"oracle setup failed with status {st}")
    return o
