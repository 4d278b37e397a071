"""Python binding of libbgs (GB300 block Gauss-Seidel / SA-AMG / FGMRES solver).

Argument marshalling only: every step of the solve runs in the CUDA library.  The names follow
the C ABI in include/bgs.h.  PyTorch supplies device memory and the CUDA stream.  There is no
CPU fallback: importing the binding without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbgs.so")

OK, INVALID_ARG, NOT_SETUP, NO_CONVERGENCE, BREAKDOWN, NAN_INF, ZERO_PIVOT, CUDA_ERROR, OOM, INTERNAL = range(10)
FIELD_MAX = 8


class bgs_csr(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class bgs_options(C.Structure):
    _fields_ = [("restart", C.c_int), ("maxit", C.c_int), ("rtol", C.c_double), ("precision", C.c_int),
                ("graph", C.c_int), ("autotune", C.c_int), ("cheb_degree", C.c_int * 8),
                ("theta", C.c_double * 8), ("max_coarse", C.c_int), ("max_levels", C.c_int),
                ("cheb_ratio", C.c_double), ("cheb_boost", C.c_double), ("power_iters", C.c_int),
                ("filter_diag", C.c_int), ("reorth_eta", C.c_double), ("jacobi", C.c_int),
                ("subsolver", C.c_int * 8), ("ilu_rows", C.c_int), ("ngroups", C.c_int),
                ("group_end", C.c_int * 8), ("inner_restart", C.c_int), ("inner_maxit", C.c_int),
                ("inner_rtol", C.c_double), ("cheb_ellipse", C.c_int)]


class bgs_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("status", C.c_int), ("restarts", C.c_int),
                ("reorth", C.c_int), ("rel_true_resid", C.c_double), ("rel_est_resid", C.c_double),
                ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double), ("nlevels", C.c_int * 8)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["nlevels"] = list(self.nlevels)
        return d


class BGSError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


_lib = None


def lib():
    """The loaded libbgs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libbgs.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sig = {
            "bgs_default_options": (i32, [C.POINTER(bgs_options)]),
            "bgs_create": (i32, [C.POINTER(vp), i32, C.POINTER(C.c_int64), C.POINTER(bgs_csr), C.POINTER(C.c_int),
                                 C.POINTER(bgs_options), vp]),
            "bgs_setup": (i32, [vp]),
            "bgs_update_values": (i32, [vp, C.POINTER(vp)]),
            "bgs_solve": (i32, [vp, vp, vp, C.POINTER(bgs_info)]),
            "bgs_solve_adjoint": (i32, [vp, vp, vp, C.POINTER(bgs_info)]),
            "bgs_grad_values": (i32, [vp, i32, i32, vp, vp, vp]),
            "bgs_grad_values_all": (i32, [vp, vp, vp, C.POINTER(vp)]),
            "bgs_apply_preconditioner": (i32, [vp, vp, vp]),
            "bgs_apply_vcycle": (i32, [vp, i32, vp, vp]),
            "bgs_full_spmv": (i32, [vp, vp, vp]),
            "bgs_num_levels": (i32, [vp, i32, C.POINTER(C.c_int)]),
            "bgs_level_info": (i32, [vp, i32, i32, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64),
                                     C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(dbl), C.POINTER(dbl),
                                     C.POINTER(dbl)]),
            "bgs_level_copy": (i32, [vp, i32, i32, i32, vp, vp, vp]),
            "bgs_level_aggregates": (i32, [vp, i32, i32, vp]),
            "bgs_level_strength": (i32, [vp, i32, i32, vp]),
            "bgs_level_format": (i32, [vp, i32, i32, i32, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "bgs_ilu_factors": (i32, [vp, i32, C.POINTER(C.c_int64), vp, vp, vp]),
            "bgs_level_ellipse": (i32, [vp, i32, i32, C.POINTER(C.c_double)]),
            "bgs_set_profiling": (i32, [vp, i32]),
            "bgs_kernel_stats": (i32, [vp, i32, C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl)]),
            "bgs_csr_spmv": (i32, [i64, i64, vp, vp, vp, vp, vp, i32, vp]),
            "bgs_arnoldi_dots": (i32, [vp, i64, i32, vp, i64, vp, vp]),
            "bgs_arnoldi_dots_noalloc": (i32, [vp, i64, i32, vp, i64, vp, vp]),
            "bgs_gram_schmidt_pass": (i32, [vp, i64, i32, vp, i64, vp, vp, vp]),
            "bgs_launch_count": (C.c_int64, []),
            "bgs_release_cached_memory": (i32, []),
            "bgs_destroy": (None, [vp]),
            "bgs_status_string": (C.c_char_p, [i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(st: int) -> str:
    return lib().bgs_status_string(int(st)).decode()


def _check(st, what):
    if st != OK:
        raise BGSError(st, what)


def _ptr(a):
    """Data pointer of a torch tensor or a numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# ---------------------------------------------------------------------------------------------
# Direct entry points (same names as the C ABI)
# ---------------------------------------------------------------------------------------------
def bgs_default_options(**overrides) -> bgs_options:
    o = bgs_options()
    _check(lib().bgs_default_options(C.byref(o)), "bgs_default_options")
    for k, v in overrides.items():
        if k in ("cheb_degree", "theta", "subsolver", "group_end"):
            arr = getattr(o, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(o, k, v)
    return o


def bgs_csr_spmv(nrows, nnz, rowptr, col, val, x, y, lanes=0, stream=None) -> int:
    return lib().bgs_csr_spmv(int(nrows), int(nnz), _ptr(rowptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y),
                              int(lanes), _stream_ptr(stream))


def bgs_arnoldi_dots(V, ld, cnt, w, n, h, stream=None) -> int:
    """h[k] = V_k . w (k < cnt), h[cnt] = w . w; device tensors, V column-major with leading dim ld."""
    return lib().bgs_arnoldi_dots(_ptr(V), int(ld), int(cnt), _ptr(w), int(n), _ptr(h), _stream_ptr(stream))


def bgs_gram_schmidt_pass(V, ld, cnt, w, n, h, nw, stream=None) -> int:
    """One Gram-Schmidt pass of the FGMRES orthogonalisation with the solver's kernels: h = V^T w
    (h[cnt] = ||w||^2), w -= V h in place, nw[0] = ||w||^2 after (device tensors; basis entries
    below 2 in magnitude)."""
    return lib().bgs_gram_schmidt_pass(_ptr(V), int(ld), int(cnt), _ptr(w), int(n), _ptr(h), _ptr(nw),
                                       _stream_ptr(stream))


def bgs_arnoldi_dots_noalloc(V, ld, cnt, w, n, h, stream=None) -> int:
    """Same as bgs_arnoldi_dots, but allocates no device memory: for callers that cannot allocate
    at that point.  Calls share one fixed scratch array, so do not overlap calls on the GPU."""
    return lib().bgs_arnoldi_dots_noalloc(_ptr(V), int(ld), int(cnt), _ptr(w), int(n), _ptr(h),
                                          _stream_ptr(stream))


def bgs_release_cached_memory() -> int:
    return lib().bgs_release_cached_memory()


def bgs_launch_count() -> int:
    return int(lib().bgs_launch_count())


class Solver:
    """Owns one bgs handle.  blocks: F x F list of CSR-like objects (rowptr/col/val arrays,
    numpy or torch, host or device) or None for zero blocks."""

    def __init__(self, blocks, field_sizes, order, options: bgs_options | None = None, stream=None, **opts):
        F = len(field_sizes)
        self.F = F
        self.field_sizes = [int(s) for s in field_sizes]
        self.n = sum(self.field_sizes)
        self.offsets = np.concatenate([[0], np.cumsum(self.field_sizes)]).astype(np.int64)
        self.options = options if options is not None else bgs_default_options(**opts)
        arr = (bgs_csr * (F * F))()
        keep = []
        for r in range(F):
            for c in range(F):
                B = blocks[r][c]
                if B is None:
                    continue
                rp, ci, v = B.rowptr, B.col, B.val
                keep += [rp, ci, v]
                nnz = int(rp[-1])
                arr[r * F + c] = bgs_csr(self.field_sizes[r], self.field_sizes[c], nnz, _ptr(rp), _ptr(ci), _ptr(v))
        self._stream = _stream_ptr(stream)
        h = C.c_void_p()
        sizes = (C.c_int64 * F)(*self.field_sizes)
        ordr = (C.c_int * F)(*[int(k) for k in order])
        _check(lib().bgs_create(C.byref(h), F, sizes, arr, ordr, C.byref(self.options), self._stream),
               "bgs_create")
        self.h = h
        self.order = list(order)
        del keep

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                lib().bgs_destroy(h)
            except Exception:
                pass
            self.h = None

    def close(self):
        self.__del__()

    def bgs_setup(self):
        _check(lib().bgs_setup(self.h), "bgs_setup")

    setup = bgs_setup

    def bgs_update_values(self, values):
        """values: F x F nested list of new value arrays (numpy or torch, host or device, in the
        order of each block's stored entries); None keeps a block's values."""
        F = self.F
        arr = (C.c_void_p * (F * F))()
        keep = []
        for r in range(F):
            for c in range(F):
                v = values[r][c]
                if v is None:
                    continue
                if isinstance(v, np.ndarray):
                    v = np.ascontiguousarray(v, dtype=np.float64)
                keep.append(v)
                arr[r * F + c] = _ptr(v)
        _check(lib().bgs_update_values(self.h, arr), "bgs_update_values")
        del keep

    def bgs_solve(self, b, x, check=True) -> bgs_info:
        info = bgs_info()
        st = lib().bgs_solve(self.h, _ptr(b), _ptr(x), C.byref(info))
        if check and st not in (OK, NO_CONVERGENCE):
            _check(st, "bgs_solve")
        return info

    def bgs_solve_adjoint(self, g, lam, check=True) -> bgs_info:
        info = bgs_info()
        st = lib().bgs_solve_adjoint(self.h, _ptr(g), _ptr(lam), C.byref(info))
        if check and st not in (OK, NO_CONVERGENCE):
            _check(st, "bgs_solve_adjoint")
        return info

    def bgs_grad_values(self, row_field, col_field, lam, x, dvals):
        _check(lib().bgs_grad_values(self.h, row_field, col_field, _ptr(lam), _ptr(x), _ptr(dvals)),
               "bgs_grad_values")

    def bgs_grad_values_all(self, lam, x, dvals):
        """dvals: F x F nested list of device tensors (nnz of each block) or None to skip a block."""
        F = self.F
        arr = (C.c_void_p * (F * F))()
        for r in range(F):
            for c in range(F):
                if dvals[r][c] is not None:
                    arr[r * F + c] = _ptr(dvals[r][c])
        _check(lib().bgs_grad_values_all(self.h, _ptr(lam), _ptr(x), arr), "bgs_grad_values_all")

    def bgs_apply_preconditioner(self, v, z):
        _check(lib().bgs_apply_preconditioner(self.h, _ptr(v), _ptr(z)), "bgs_apply_preconditioner")

    def bgs_apply_vcycle(self, field, b, x):
        _check(lib().bgs_apply_vcycle(self.h, int(field), _ptr(b), _ptr(x)), "bgs_apply_vcycle")

    def bgs_full_spmv(self, x, y):
        _check(lib().bgs_full_spmv(self.h, _ptr(x), _ptr(y)), "bgs_full_spmv")

    def bgs_num_levels(self, field) -> int:
        n = C.c_int()
        _check(lib().bgs_num_levels(self.h, int(field), C.byref(n)), "bgs_num_levels")
        return n.value

    def bgs_level_info(self, field, level) -> dict:
        rows, nnz, pnnz = C.c_int64(), C.c_int64(), C.c_int64()
        nagg, rounds = C.c_int(), C.c_int()
        om, lo, hi = C.c_double(), C.c_double(), C.c_double()
        _check(lib().bgs_level_info(self.h, int(field), int(level), C.byref(rows), C.byref(nnz), C.byref(pnnz),
                                    C.byref(nagg), C.byref(rounds), C.byref(om), C.byref(lo), C.byref(hi)),
               "bgs_level_info")
        return dict(rows=rows.value, nnz=nnz.value, p_nnz=pnnz.value, nagg=nagg.value, mis_rounds=rounds.value,
                    omega=om.value, lmin=lo.value, lmax=hi.value)

    def bgs_level_copy(self, field, level, which):
        """which: 0 A_l, 1 P_l, 2 R_l -> (rowptr, col, val) numpy arrays."""
        info = self.bgs_level_info(field, level)
        if which == 0:
            n, nnz = info["rows"], info["nnz"]
        elif which == 1:
            n, nnz = info["rows"], info["p_nnz"]
        else:
            n, nnz = info["nagg"], info["p_nnz"]
        rp = np.zeros(n + 1, dtype=np.int32)
        ci = np.zeros(max(nnz, 1), dtype=np.int32)
        v = np.zeros(max(nnz, 1), dtype=np.float64)
        _check(lib().bgs_level_copy(self.h, int(field), int(level), int(which), _ptr(rp), _ptr(ci), _ptr(v)),
               "bgs_level_copy")
        return rp, ci[:nnz], v[:nnz]

    def bgs_level_aggregates(self, field, level):
        info = self.bgs_level_info(field, level)
        agg = np.zeros(info["rows"], dtype=np.int32)
        _check(lib().bgs_level_aggregates(self.h, int(field), int(level), _ptr(agg)), "bgs_level_aggregates")
        return agg

    def bgs_level_strength(self, field, level):
        """Strength flag (uint8) of every stored entry of A_l, CSR order."""
        info = self.bgs_level_info(field, level)
        out = np.zeros(max(info["nnz"], 1), dtype=np.uint8)
        _check(lib().bgs_level_strength(self.h, int(field), int(level), _ptr(out)), "bgs_level_strength")
        return out[:info["nnz"]]

    def bgs_level_ellipse(self, field, level) -> float:
        im = C.c_double()
        _check(lib().bgs_level_ellipse(self.h, int(field), int(level), C.byref(im)), "bgs_level_ellipse")
        return im.value

    def bgs_ilu_factors(self, field):
        """DD(0)-ILU(0) factors of a field on subsolver 1: (rowptr, col, val) host arrays."""
        nnz = C.c_int64()
        _check(lib().bgs_ilu_factors(self.h, int(field), C.byref(nnz), None, None, None), "bgs_ilu_factors")
        rp = np.zeros(self.field_sizes[field] + 1, dtype=np.int32)
        ci = np.zeros(max(nnz.value, 1), dtype=np.int32)
        v = np.zeros(max(nnz.value, 1))
        _check(lib().bgs_ilu_factors(self.h, int(field), C.byref(nnz), _ptr(rp), _ptr(ci), _ptr(v)),
               "bgs_ilu_factors")
        return rp, ci[:nnz.value], v[:nnz.value]

    def bgs_level_format(self, field, level, which=0, with_block=False):
        """Layout of a stored operator (which: 0 A_l, 1 P_l, 2 R_l, 3 the full operator): -2 = node
        blocks, -1 = SELL-32 with diagonal offsets, 0 = SELL-32, k > 0 = CSR with k threads per row;
        with with_block, (format, threads per block)."""
        f, t = C.c_int(), C.c_int()
        _check(lib().bgs_level_format(self.h, int(field), int(level), int(which), C.byref(f), C.byref(t)),
               "bgs_level_format")
        return (f.value, t.value) if with_block else f.value

    def bgs_set_profiling(self, on=True):
        _check(lib().bgs_set_profiling(self.h, 1 if on else 0), "bgs_set_profiling")

    def bgs_kernel_stats(self, kernel_class) -> dict:
        n, ms, by = C.c_int64(), C.c_double(), C.c_double()
        _check(lib().bgs_kernel_stats(self.h, int(kernel_class), C.byref(n), C.byref(ms), C.byref(by)),
               "bgs_kernel_stats")
        return dict(launches=n.value, ms=ms.value, bytes=by.value)


KERNEL_CLASSES = {"full_spmv": 0, "chebyshev_fine": 1, "arnoldi": 2, "coupling": 3, "chebyshev_coarse": 4,
                  "dd_ilu": 5}


def solver_for_system(system, order=None, device=True, **opts):
    """Solver over a battery_system.CoupledSystem; the CSR blocks are passed from host memory
    (the library copies them) unless device=True, in which case they are staged as torch tensors."""
    import torch

    class _B:
        pass

    blocks = []
    keep = []
    for r in range(5):
        row = []
        for c in range(5):
            B = system.blocks.get((r, c))
            if B is None:
                row.append(None)
                continue
            o = _B()
            if device:
                o.rowptr = torch.from_numpy(B.rowptr).cuda()
                o.col = torch.from_numpy(B.col).cuda()
                o.val = torch.from_numpy(B.val).cuda()
                o.rowptr_host = B.rowptr
            else:
                o.rowptr, o.col, o.val = B.rowptr, B.col, B.val
            keep.append(o)
            row.append(o)
        blocks.append(row)

    class _RP:
        def __init__(self, o):
            self.rowptr, self.col, self.val = o.rowptr, o.col, o.val

    # the nnz is read from rowptr[-1]: take it from the host copy for device tensors
    blocks2 = []
    for row in blocks:
        r2 = []
        for o in row:
            if o is None:
                r2.append(None)
                continue
            w = _RP(o)
            if device:
                w.rowptr = _Rowptr(o.rowptr, int(o.rowptr_host[-1]))
            r2.append(w)
        blocks2.append(r2)
    s = Solver(blocks2, system.field_sizes, order if order is not None else list(range(5)), **opts)
    torch.cuda.synchronize()
    return s


class _Rowptr:
    """A device rowptr tensor that reports its last element without a device read."""

    def __init__(self, t, last):
        self.t, self.last = t, last

    def __getitem__(self, i):
        if i == -1:
            return self.last
        raise IndexError

    def data_ptr(self):
        return self.t.data_ptr()


# ---------------------------------------------------------------------------------------------
# Differentiable solve: x = A(vals)^-1 b with gradients for b and the stored block values
# ---------------------------------------------------------------------------------------------
class _Block:
    def __init__(self, rowptr, col, val, last):
        self.rowptr = _Rowptr(rowptr, last) if hasattr(rowptr, "data_ptr") else rowptr
        self.col, self.val = col, val


def _autograd_fn():
    import torch

    class BGSSolve(torch.autograd.Function):
        """forward: bgs_create + bgs_setup + bgs_solve.  backward: bgs_solve_adjoint gives
        lambda = A^-T g (so dL/db = lambda) and bgs_grad_values gives dL/dA = -lambda x^T on the
        stored pattern of every block (the adjoint and the gradient kernel are extensions; the
        paper has no adjoint)."""

        @staticmethod
        def forward(ctx, meta, b, *vals):
            keys, patterns, sizes, order, opts = meta
            F = len(sizes)
            blocks = [[None] * F for _ in range(F)]
            for (r, c), v in zip(keys, vals):
                rp, ci, last = patterns[(r, c)]
                blocks[r][c] = _Block(rp, ci, v.detach().contiguous(), last)
            solver = Solver(blocks, sizes, order, **opts)
            solver.setup()
            x = torch.zeros_like(b)
            info = solver.bgs_solve(b.detach().contiguous(), x)
            ctx.solver, ctx.keys, ctx.nnz = solver, keys, [patterns[k][2] for k in keys]
            ctx.info = info
            ctx.save_for_backward(x)
            return x

        @staticmethod
        def backward(ctx, gx):
            (x,) = ctx.saved_tensors
            solver = ctx.solver
            lam = torch.zeros_like(gx)
            solver.bgs_solve_adjoint(gx.detach().contiguous(), lam)
            grads = []
            for (r, c), nnz in zip(ctx.keys, ctx.nnz):
                d = torch.empty(nnz, dtype=torch.float64, device=gx.device)
                solver.bgs_grad_values(r, c, lam, x, d)
                grads.append(d)
            ctx.solver = None
            return (None, lam, *grads)

    return BGSSolve


_BGSSolve = None


def bgs_solve_autograd(patterns, values, b, field_sizes, order, **opts):
    """Differentiable x = A^-1 b.  patterns: {(r, c): (rowptr, col)} device int32 tensors;
    values: {(r, c): float64 device tensor} (may require grad); b: float64 device tensor."""
    global _BGSSolve
    if _BGSSolve is None:
        _BGSSolve = _autograd_fn()
    keys = sorted(values.keys())
    pats = {}
    for k in keys:
        rp, ci = patterns[k]
        last = int(rp[-1].item()) if hasattr(rp, "item") else int(rp[-1])
        pats[k] = (rp, ci, last)
    meta = (keys, pats, [int(s) for s in field_sizes], list(order), dict(opts))
    return _BGSSolve.apply(meta, b, *[values[k] for k in keys])
