// C ABI of libbgs: block operator (Sec. 2.2, Eq. block-splitting), SA-AMG setup per diagonal
// block (Sec. 2.2.1), the forward block Gauss-Seidel sweep (Eqs. hierarchical-bgs, non-voltage-bgs,
// voltage-bgs) and flexible GMRES (Sec. 2.2) with CGS2 Arnoldi on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <cstdlib>
#include <memory>
#include <thread>
#include <type_traits>

#include "internal.h"

using namespace bgs;

namespace {

struct KStats {
    int64_t launches = 0;
    double ms = 0.0, bytes = 0.0;
};

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    int cls = 0;
    double bytes = 0.0;
};

}  // namespace

// Workspace of one FGMRES instance: the outer solve, or one group's inner solve (nested variant).
struct Krylov {
    int64_t n = 0, ld = 0;   // vector length, basis leading dimension (n rounded up to 64 entries)
    int m = 0;               // restart length
    DBuf<double> V, Z, w, r, x, b;
    DBuf<FgState> st;        // the solver's scalar state on the device
    void alloc(int64_t n_, int m_, cudaStream_t s) {
        n = n_;
        m = m_;
        ld = (n + 63) / 64 * 64;
        V.alloc((size_t)ld * (m + 1), s);
        Z.alloc((size_t)ld * m, s);
        w.alloc((size_t)n, s);
        r.alloc((size_t)n, s);
        x.alloc((size_t)n, s);
        b.alloc((size_t)n, s);
        st.alloc(1, s);
    }
};

// One FGMRES restart cycle captured as a CUDA graph: a WHILE node whose body is one step (the
// preconditioner sweep on the staging vectors, z_j stored, w = A z_j, Gram-Schmidt, the step kernel
// that ends the loop).
struct CycleGraph {
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond{};
    long long body_launches = 0;
};

// One group of the nested variant: order positions [p0, p1), fields with consecutive ids, so the
// group's vector is the slice [base, base + n) of a global vector.
struct Group {
    int p0 = 0, p1 = 0;
    int64_t base = 0, n = 0;
    DCsr A, AT;              // the group's diagonal block and its transpose, local columns
    Krylov K;                // inner FGMRES workspace
};

struct bgs_ctx {
    cudaStream_t s = nullptr;
    int F = 0;
    int64_t sizes[8] = {}, offs[9] = {};
    int order[8] = {}, pos[8] = {};
    bgs_options opt{};
    std::vector<DCsr> blk;          // F*F input copies (n == 0: zero block)
    DCsr full, fullT;
    DCsr lower[8], upperT[8];
    Hier H[8];
    bool setup_done = false, adjoint_ready = false;
    Scratch sc;
    // per-block set-up streams and scratch (the hierarchies are built concurrently); the streams
    // live as long as the handle because the hierarchy memory is released on them
    cudaStream_t bs[8] = {};
    Scratch bsc[8];
    // block Jacobi: the V-cycles fork onto bs[k] from the solve stream and join back
    cudaEvent_t fork_ev = nullptr, join_ev[8] = {};
    Krylov K;                       // outer FGMRES workspace
    // nested variant: groups, and per field the couplings of the outer sweep over groups (rows of
    // field k, global columns of the earlier groups; adjoint: transposed couplings of the later
    // groups) and of the inner sweep inside its group (local columns of the group)
    std::vector<Group> groups;
    DCsr go_lower[8], go_upperT[8], gi_lower[8], gi_upperT[8];
    double t_setup_ms = 0.0;
    int last_reorth = 0;
    // profiling
    // CUDA graph of one FGMRES restart cycle (forward, adjoint), captured once on an internal stream
    // with fixed staging vectors gv -> gz for the sweep, replayed for every cycle of every solve
    cudaStream_t gs = nullptr;
    CycleGraph cyc[2];
    DBuf<double> gv, gz;
    DBuf<float> zf;                 // mixed precision: FP32 copy of the sweep output for the couplings
    bool prof = false;
    std::vector<EventPair> ev;
    size_t ev_used = 0;
    KStats stats[6];
};

namespace {

int64_t total_n(const bgs_ctx *h) { return h->offs[h->F]; }


// ------------------------------------------------------------------ profiling helpers
struct Prof {
    bgs_ctx *h;
    EventPair *p = nullptr;
    Prof(bgs_ctx *hh, int cls, double bytes) : h(hh) {
        if (!h->prof) return;
        if (h->ev_used == h->ev.size()) {
            EventPair e;
            CK(cudaEventCreate(&e.a));
            CK(cudaEventCreate(&e.b));
            h->ev.push_back(e);
        }
        p = &h->ev[h->ev_used++];
        p->cls = cls;
        p->bytes = bytes;
        CK(cudaEventRecord(p->a, h->s));
    }
    ~Prof() {
        if (p) cudaEventRecord(p->b, h->s);
    }
};

void prof_collect(bgs_ctx *h) {
    if (!h->prof) return;
    CK(cudaStreamSynchronize(h->s));
    for (size_t i = 0; i < h->ev_used; i++) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev[i].a, h->ev[i].b));
        KStats &k = h->stats[h->ev[i].cls];
        k.launches++;
        k.ms += ms;
        k.bytes += h->ev[i].bytes;
    }
    h->ev_used = 0;
}

// Algorithmic bytes of one application: the stored values once, the index data of the form in use
// (CSR / SELL-32: a column index per entry and the row pointers; diagonal-offset SELL-32: one offset
// per slot of 32 rows and the slice pointers), x read and y written once, plus extra vectors.
double spmv_bytes(const DCsr &A, int vbytes, int xbytes, int extra_vectors) {
    const double idx = A.bsr_active() ? 4.0 * (double)A.bsr_slots + 4.0 * ((A.bsr_nc + 31) / 32 + 1)
                       : A.dia ? 4.0 * (double)(A.dia_nnz / 32) + 4.0 * ((A.n + 31) / 32 + 1)
                               : 4.0 * (double)A.nnz + 4.0 * (A.n + 1);
    return (double)A.nnz * vbytes + idx + (double)xbytes * A.n * (2 + extra_vectors);
}

// ------------------------------------------------------------------ typed buffer access
template <class XT>
struct Buf;
template <>
struct Buf<double> {
    static double *b(Level &L) { return L.b.p; }
    static double *x0(Level &L) { return L.x0.p; }
    static double *x1(Level &L) { return L.x1.p; }
    static double *d(Level &L) { return L.d.p; }
    static double *r(Level &L) { return L.r.p; }
    static const double *dinv(Level &L) { return L.dinv.p; }
    static void alloc(Level &L, int n, cudaStream_t s) {
        L.b.alloc(n, s); L.x0.alloc(n, s); L.x1.alloc(n, s); L.d.alloc(n, s); L.r.alloc(n, s);
    }
};
template <>
struct Buf<float> {
    static float *b(Level &L) { return L.fb.p; }
    static float *x0(Level &L) { return L.fx0.p; }
    static float *x1(Level &L) { return L.fx1.p; }
    static float *d(Level &L) { return L.fd.p; }
    static float *r(Level &L) { return L.fr.p; }
    static const float *dinv(Level &L) { return L.dinvf.p; }
    static void alloc(Level &L, int n, cudaStream_t s) {
        L.fb.alloc(n, s); L.fx0.alloc(n, s); L.fx1.alloc(n, s); L.fd.alloc(n, s); L.fr.alloc(n, s);
    }
};

// ------------------------------------------------------------------ V-cycle (Sec. 2.2.1)
// Chebyshev coefficients of one smoothing pass on a level (deg steps), in the scaled form of the
// step kernels (e = d / c2): step 0 is cheb_first (from x = 0) or a step with alpha = 0 and scale
// 1/theta; step k = 1..deg-1 has alpha[k-1] = c1 c2_prev / c2 and scale[k-1] = c2.  The real
// interval (Saad's form) or the ellipse with imaginary semi-axis lim through its focal parameter
// c2 = delta^2 - lim^2 (tau_k = rho_k / delta form).
void cheb_coefs(const Level &Lv, int deg, double &inv_theta, double *alpha, double *scale) {
    const double theta = (Lv.lmax + Lv.lmin) / 2.0, delta = (Lv.lmax - Lv.lmin) / 2.0;
    const double sigma = theta / delta;
    inv_theta = 1.0 / theta;
    const bool ell = Lv.lim > 0.0;
    const double c2e = delta * delta - Lv.lim * Lv.lim;
    double st = ell ? inv_theta : 1.0 / sigma, sc = inv_theta;
    for (int k = 1; k < deg; k++) {
        double c1, c2;
        if (ell) {
            const double tn = 1.0 / (2.0 * theta - c2e * st);
            c1 = c2e * tn * st;
            c2 = 2.0 * tn;
            st = tn;
        } else {
            const double rn = 1.0 / (2.0 * sigma - st);
            c1 = rn * st;
            c2 = 2.0 * rn / delta;
            st = rn;
        }
        alpha[k - 1] = c1 * sc / c2;
        scale[k - 1] = c2;
        sc = c2;
    }
}

// The first Chebyshev step of level l's pre-smoothing (of the diagonal solve for subsolver 2), to be
// fused into the product that writes the level's right-hand side; false where there is none (the
// coarsest level's dense solve, the DD(0)-ILU(0) sweep).  inv_theta is computed as cheb_coefs does.
template <class XT>
bool first_step_of(Hier &H, int l, FirstStep<XT> &f) {
    if (H.solver == 1 || (H.solver == 2 && l != 0)) return false;
    Level &Lv = H.L[l];
    double inv_theta = 1.0;
    if (H.solver == 0) {
        if (l >= (int)H.L.size() - 1) return false;
        const double theta = (Lv.lmax + Lv.lmin) / 2.0;
        inv_theta = 1.0 / theta;
    }
    f = FirstStep<XT>{Buf<XT>::dinv(Lv), Buf<XT>::x0(Lv), Buf<XT>::d(Lv), inv_theta};
    return true;
}

// One V-cycle on level l from x = 0.  first_done: the first pre-smoothing step was fused into the
// product that wrote b (first_step_of).  out (finest level only, may be null): where the last
// post-smoothing step writes, instead of the level's own x buffers.
template <class VT, class XT>
XT *vcycle(bgs_ctx *h, Hier &H, int l, bool transposed, bool first_done = false, XT *out = nullptr) {
    cudaStream_t s = h->s;
    Level &Lv = H.L[l];
    const int n = Lv.A.n;
    XT *b = Buf<XT>::b(Lv), *x0 = Buf<XT>::x0(Lv), *x1 = Buf<XT>::x1(Lv), *d = Buf<XT>::d(Lv),
       *r = Buf<XT>::r(Lv);
    if (l != 0) out = nullptr;
    if (l == (int)H.L.size() - 1) {
        XT *dst = out ? out : x0;
        dense_gemv<XT>(n, transposed ? H.inv_T().p : H.inv.p, b, dst, s);
        return dst;
    }
    const DCsr &A = transposed ? Lv.AT : Lv.A;
    const XT *dinv = Buf<XT>::dinv(Lv);
    const int deg = H.degree;
    double inv_theta;
    std::vector<double> alpha((size_t)deg), scale((size_t)deg);
    cheb_coefs(Lv, deg, inv_theta, alpha.data(), scale.data());
    const int vb = sizeof(VT), xb = sizeof(XT);
    const double cbytes = spmv_bytes(A, vb, xb, 4);
    const int ccls = l == 0 ? 1 : 4;   // fine-level vs coarse-level Chebyshev steps
    // pre-smoothing from x = 0
    if (!first_done) cheb_first<XT>(n, b, dinv, inv_theta, x0, d, s);
    XT *cur = x0, *oth = x1;
    for (int k = 1; k < deg; k++) {
        Prof pf(h, ccls, cbytes);
        cheb_step<VT, XT>(A, b, dinv, cur, oth, d, alpha[k - 1], scale[k - 1], false, s);
        std::swap(cur, oth);
    }
    // residual, restriction (with the coarse level's first smoothing step), coarse correction,
    // prolongation
    spmv_resid<VT, XT>(A, b, cur, r, s);
    Level &C = H.L[l + 1];
    FirstStep<XT> fc;
    const bool fuse = first_step_of<XT>(H, l + 1, fc);
    if (fuse) spmv_store_first<VT, XT>(Lv.R, r, Buf<XT>::b(C), fc, s);
    else spmv_store<VT, XT>(Lv.R, r, Buf<XT>::b(C), s);
    XT *xc = vcycle<VT, XT>(h, H, l + 1, transposed, fuse);
    spmv_addto<VT, XT>(Lv.P, xc, cur, s);
    // post-smoothing (the first step with alpha = 0 from the corrected x)
    for (int k = 0; k < deg; k++) {
        XT *dst = (out && k == deg - 1) ? out : oth;
        Prof pf(h, ccls, cbytes);
        if (k == 0) cheb_step<VT, XT>(A, b, dinv, cur, dst, d, 0.0, inv_theta, true, s);
        else cheb_step<VT, XT>(A, b, dinv, cur, dst, d, alpha[k - 1], scale[k - 1], false, s);
        oth = cur;
        cur = dst;
    }
    return cur;
}

// The block solve of one diagonal block on L[0].b: one V-cycle, the DD(0)-ILU(0) sweep, or the
// diagonal solve x = D^-1 b (its own transpose).  first_done and out as for vcycle (first_done:
// the first step of first_step_of(H, 0) has run).
template <class VT, class XT>
XT *block_solve(bgs_ctx *h, Hier &H, bool transposed, bool first_done = false, XT *out = nullptr) {
    if (H.solver == 2) {
        Level &L0 = H.L[0];
        if (!first_done)
            cheb_first<XT>(L0.A.n, Buf<XT>::b(L0), Buf<XT>::dinv(L0), 1.0, Buf<XT>::x0(L0), Buf<XT>::d(L0), h->s);
        return Buf<XT>::x0(L0);
    }
    if (H.solver == 1) {
        Level &L0 = H.L[0];
        const IluFactors &M = transposed ? H.iluT : H.ilu;
        const int vb = sizeof(XT) == 8 ? 8 : 4;
        Prof pf(h, 5, 2.0 * ((double)M.F.nnz * (vb + 4) + 4.0 * (M.F.n + 1)) + 2.0 * sizeof(XT) * M.F.n);
        ilu_apply<XT>(M, transposed, Buf<XT>::b(L0), Buf<XT>::x0(L0), h->s);
        return Buf<XT>::x0(L0);
    }
    return vcycle<VT, XT>(h, H, 0, transposed, first_done, out);
}

template <class XT>
void copy_in(const double *src, XT *dst, int64_t n, cudaStream_t s);
template <>
void copy_in<double>(const double *src, double *dst, int64_t n, cudaStream_t s) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
}
template <>
void copy_in<float>(const double *src, float *dst, int64_t n, cudaStream_t s) { copy_d2f(src, dst, n, s); }
template <class XT>
void copy_out(const XT *src, double *dst, int64_t n, cudaStream_t s);
template <>
void copy_out<double>(const double *src, double *dst, int64_t n, cudaStream_t s) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
}
template <>
void copy_out<float>(const float *src, double *dst, int64_t n, cudaStream_t s) { copy_f2d(src, dst, n, s); }

// ------------------------------------------------------------------ block Gauss-Seidel sweep
// block Jacobi: z_k = V_k(v_k) for every k, each block's V-cycle on its own stream (forked from
// and joined back into the solve stream, so a captured graph holds F parallel branches)
template <class VT, class XT>
void jacobi_sweep(bgs_ctx *h, const double *v, double *z, bool transposed) {
    cudaStream_t s = h->s;
    const bool fork = !h->prof;   // per-class event timing needs a single stream
    if (fork && !h->fork_ev) {
        CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
        for (int k = 0; k < h->F; k++) CK(cudaEventCreateWithFlags(&h->join_ev[k], cudaEventDisableTiming));
    }
    if (fork) CK(cudaEventRecord(h->fork_ev, s));
    for (int k = 0; k < h->F; k++) {
        cudaStream_t sk = fork ? h->bs[k] : s;
        if (fork) CK(cudaStreamWaitEvent(sk, h->fork_ev, 0));
        h->s = sk;
        try {
            Hier &H = h->H[k];
            FirstStep<XT> f0;
            const bool fuse0 = first_step_of<XT>(H, 0, f0);
            if (fuse0) copy_in_first<XT>(v + h->offs[k], Buf<XT>::b(H.L[0]), h->sizes[k], f0, sk);
            else copy_in<XT>(v + h->offs[k], Buf<XT>::b(H.L[0]), h->sizes[k], sk);
            XT *out = nullptr;
            if constexpr (std::is_same<XT, double>::value) out = z + h->offs[k];
            XT *xk = block_solve<VT, XT>(h, H, transposed, fuse0, out);
            if (xk != out) copy_out<XT>(xk, z + h->offs[k], h->sizes[k], sk);
        } catch (...) {
            h->s = s;
            throw;
        }
        h->s = s;
        if (fork) {
            CK(cudaEventRecord(h->join_ev[k], sk));
            CK(cudaStreamWaitEvent(s, h->join_ev[k], 0));
        }
    }
}

template <class VT, class XT, class CVT>
void sweep(bgs_ctx *h, const double *v, double *z, bool transposed) {
    if (h->opt.jacobi) {
        jacobi_sweep<VT, XT>(h, v, z, transposed);
        return;
    }
    cudaStream_t s = h->s;
    // FP32 block solves: each block's output is also kept in FP32 (zf), and the couplings of the
    // later blocks gather that copy (half the bytes of the FP64 z; the same values, since z holds
    // the FP32 results widened)
    float *zf = std::is_same<XT, float>::value ? h->zf.p : nullptr;
    for (int p = 0; p < h->F; p++) {
        const int k = transposed ? h->order[h->F - 1 - p] : h->order[p];
        Hier &H = h->H[k];
        Level &L0 = H.L[0];
        const int64_t nk = h->sizes[k];
        XT *b0 = Buf<XT>::b(L0);
        const DCsr &C = transposed ? h->upperT[k] : h->lower[k];
        // the block's right-hand side with the first step of its solve fused in
        FirstStep<XT> f0;
        const bool fuse0 = first_step_of<XT>(H, 0, f0);
        if (C.nnz > 0) {
            Prof pf(h, 3, spmv_bytes(C, sizeof(CVT), zf ? 4 : 8, 1) + (fuse0 ? 3.0 * sizeof(XT) * nk : 0.0));
            if constexpr (std::is_same<XT, float>::value) {
                if (zf) {
                    if (fuse0) coupling_sub_first<CVT, XT, float>(C, v + h->offs[k], zf, b0, f0, s);
                    else coupling_sub<CVT, XT, float>(C, v + h->offs[k], zf, b0, s);
                } else {
                    if (fuse0) coupling_sub_first<CVT, XT, double>(C, v + h->offs[k], z, b0, f0, s);
                    else coupling_sub<CVT, XT, double>(C, v + h->offs[k], z, b0, s);
                }
            } else {
                if (fuse0) coupling_sub_first<CVT, XT, double>(C, v + h->offs[k], z, b0, f0, s);
                else coupling_sub<CVT, XT, double>(C, v + h->offs[k], z, b0, s);
            }
        } else {
            if (fuse0) copy_in_first<XT>(v + h->offs[k], b0, nk, f0, s);
            else copy_in<XT>(v + h->offs[k], b0, nk, s);
        }
        // FP64: the last smoothing step writes the block's part of z itself
        XT *out = nullptr;
        if constexpr (std::is_same<XT, double>::value) out = z + h->offs[k];
        XT *xk = block_solve<VT, XT>(h, H, transposed, fuse0, out);
        if constexpr (std::is_same<XT, float>::value) {
            if (zf) copy_f2d_keep(xk, z + h->offs[k], zf + h->offs[k], nk, s);
            else copy_out<XT>(xk, z + h->offs[k], nk, s);
        } else {
            if (xk != out) copy_out<XT>(xk, z + h->offs[k], nk, s);
        }
    }
}

void apply_prec(bgs_ctx *h, const double *v, double *z, bool transposed) {
    if (h->opt.precision == 1) sweep<float, float, __nv_bfloat16>(h, v, z, transposed);
    else sweep<double, double, double>(h, v, z, transposed);
}


void drop_graphs(bgs_ctx *h) {
    for (auto &c : h->cyc)
        if (c.exec) {
            cudaGraphExecDestroy(c.exec);
            c.exec = nullptr;
        }
}

double host_dot(bgs_ctx *h, const double *a, const double *b, int64_t n) {
    dev_dot(a, b, n, h->sc.scal.p + 8, h->sc, h->s);
    CK(cudaMemcpyAsync(h->sc.h_scal + 8, h->sc.scal.p + 8, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    return h->sc.h_scal[8];
}

// ------------------------------------------------------------------ FGMRES(m)
// The scalar fields at the head of the device state (read back after a step or a cycle).
constexpr size_t kFgHead = offsetof(FgState, nw1);

FgState read_state(bgs_ctx *h, const Krylov &K) {
    double *buf = h->sc.h_scal + 16;   // pinned; slots 0..15 serve the other read-backs
    CK(cudaMemcpyAsync(buf, K.st.p, kFgHead, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    FgState hs;
    std::memcpy((void *)&hs, buf, kFgHead);
    return hs;
}

// Captures one restart cycle of the outer solve as a CUDA graph (a WHILE node over one step).
void build_cycle_graph(bgs_ctx *h, Krylov &K, const DCsr &A, int m, bool adjoint, CycleGraph &cg) {
    const int64_t n = K.n;
    if (!h->gs) CK(cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking));
    if (!h->gv.p) {
        h->gv.alloc((size_t)n, h->s);
        h->gz.alloc((size_t)n, h->s);
        CK(cudaStreamSynchronize(h->s));
    }
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaStream_t saved = h->s;
    const bool saved_prof = h->prof;
    bool capturing = false;
    try {
        CK(cudaGraphConditionalHandleCreate(&cg.cond, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cg.cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        h->s = h->gs;
        h->prof = false;
        const long long l0 = launch_count();
        CK(cudaStreamBeginCaptureToGraph(h->gs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        apply_prec(h, h->gv.p, h->gz.p, adjoint);
        fg_store_z(K.st.p, h->gz.p, K.Z.p, K.ld, n, h->gs);
        spmv_store<double, double>(A, h->gz.p, K.w.p, h->gs);
        fg_orthogonalise(K.st.p, K.V.p, K.ld, m, K.w.p, n, h->opt.reorth_eta >= 1.0, h->sc, h->gs);
        fg_step(K.st.p, cg.cond, true, K.w.p, K.V.p, K.ld, h->gv.p, n, h->gs);
        cudaGraph_t out = nullptr;
        capturing = false;
        CK(cudaStreamEndCapture(h->gs, &out));
        cg.body_launches = launch_count() - l0;
        h->s = saved;
        h->prof = saved_prof;
        CK(cudaGraphInstantiate(&cg.exec, g, 0));
        cudaGraphDestroy(g);
    } catch (...) {
        if (capturing) {
            cudaGraph_t out = nullptr;
            cudaStreamEndCapture(h->gs, &out);
        }
        h->s = saved;
        h->prof = saved_prof;
        cudaGraphDestroy(g);
        cg.exec = nullptr;
        throw;
    }
}

// Restarted right-preconditioned flexible GMRES on the workspace K: solves A x = K.b from x = 0
// into K.x.  prec(v, z) applies z = M^-1 v; A is the FP64 operator (w = A z and the true residual
// at every restart).  Gram-Schmidt with the selective re-orthogonalisation test of reorth_eta.
// Every step's arithmetic runs in device kernels; with cg the whole cycle is one graph launch
// (the preconditioner captured inside it), otherwise the host launches each step and reads the
// stop decision back.  Both orders of launches run the same kernels on the same data.
template <class Prec>
int fgmres_run(bgs_ctx *h, Krylov &K, const DCsr &A, int m, int maxit, double rtol, Prec &&prec, bgs_info *info,
               CycleGraph *cg) {
    cudaStream_t s = h->s;
    const int64_t n = K.n;
    const int64_t ld = K.ld;
    if (m > K.m || m > kMaxRestart) throw Error(BGS_INTERNAL, "restart longer than the Krylov workspace");
    double *V = K.V.p, *Z = K.Z.p, *w = K.w.p, *r = K.r.p, *x = K.x.p, *b = K.b.p;
    bgs_info inf{};
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    const double bn2 = host_dot(h, b, b, n);
    const double bnorm = std::sqrt(bn2);
    if (!std::isfinite(bnorm)) {
        inf.status = BGS_NAN_INF;
        if (info) *info = inf;
        return BGS_NAN_INF;
    }
    if (bnorm == 0.0) {
        inf.converged = 1;
        inf.status = BGS_OK;
        if (info) *info = inf;
        return BGS_OK;
    }
    const double eta = h->opt.reorth_eta;
    fg_init(K.st.p, m, maxit, rtol, eta * eta, bnorm, s);
    CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    double beta = bnorm, rel = 1.0;
    int status = BGS_NO_CONVERGENCE, restarts = 0;
    FgState hs{};
    for (;;) {
        fg_begin(K.st.p, r, beta, V, cg ? h->gv.p : nullptr, n, s);
        if (cg) {
            CK(cudaGraphLaunch(cg->exec, s));
            hs = read_state(h, K);
            for (long long i = 0; i < cg->body_launches * hs.jend; i++) count_launch();
        } else {
            for (int j = 0;; j++) {
                double *vj = V + (size_t)j * ld, *zj = Z + (size_t)j * ld;
                prec((const double *)vj, zj);
                {
                    Prof pf(h, 0, spmv_bytes(A, 8, 8, 0));
                    spmv_store<double, double>(A, zj, w, s);
                }
                {
                    Prof pf(h, 2, 8.0 * n * (2.0 * (j + 1) + 3.0));
                    fg_orthogonalise(K.st.p, V, ld, m, w, n, eta >= 1.0, h->sc, s);
                }
                fg_step(K.st.p, cudaGraphConditionalHandle{}, false, w, V, ld, nullptr, n, s);
                hs = read_state(h, K);
                if (hs.stop) break;
            }
        }
        if (hs.flag == 4) {
            status = BGS_NAN_INF;
            break;
        }
        fg_finish_cycle(K.st.p, Z, ld, x, n, s);
        spmv_resid<double, double>(A, b, x, r, s);
        beta = std::sqrt(host_dot(h, r, r, n));
        rel = beta / bnorm;
        if (!std::isfinite(rel)) {
            status = BGS_NAN_INF;
            break;
        }
        if (rel <= rtol) {
            status = BGS_OK;
            break;
        }
        if (hs.it >= maxit) {
            status = BGS_NO_CONVERGENCE;
            break;
        }
        restarts++;
    }
    inf.iters = hs.it;
    inf.converged = status == BGS_OK;
    inf.status = status;
    inf.restarts = restarts;
    inf.reorth = hs.reorth;
    inf.rel_true_resid = rel;
    inf.rel_est_resid = hs.est;
    if (info) *info = inf;
    return status;
}

void vstack(const std::vector<DCsr *> &parts, int ncols, DCsr &C, cudaStream_t s);

// ------------------------------------------------------------------ nested variant
// Sweep inside group G on group-local vectors (the inner FGMRES preconditioner): forward over the
// group's positions with the couplings inside the group, or the transposed sweep in reverse.
template <class VT, class XT, class CVT>
void group_sweep(bgs_ctx *h, const Group &G, const double *v, double *z, bool transposed) {
    cudaStream_t s = h->s;
    for (int t = G.p0; t < G.p1; t++) {
        const int p = transposed ? G.p1 - 1 - (t - G.p0) : t;
        const int k = h->order[p];
        Hier &H = h->H[k];
        const int64_t nk = h->sizes[k], off = h->offs[k] - G.base;
        XT *b0 = Buf<XT>::b(H.L[0]);
        const DCsr &C = transposed ? h->gi_upperT[k] : h->gi_lower[k];
        if (C.nnz > 0 && !h->opt.jacobi) {
            Prof pf(h, 3, spmv_bytes(C, sizeof(CVT), 8, 1));
            coupling_sub<CVT, XT, double>(C, v + off, z, b0, s);
        } else {
            copy_in<XT>(v + off, b0, nk, s);
        }
        XT *xk = block_solve<VT, XT>(h, H, transposed);
        copy_out<XT>(xk, z + off, nk, s);
    }
}

// Nested preconditioner (Sec. 2.2, Eq. hierarchical-bgs over the groups): for each group in order,
// r_g = v_g minus the couplings to the groups already solved, then A_gg z_g = r_g by an inner
// FGMRES(inner_restart) to inner_rtol (at most inner_maxit iterations) preconditioned by the
// group's own sweep.  The adjoint runs the groups in reverse with transposed operators.
void apply_nested(bgs_ctx *h, const double *v, double *z, bool adjoint) {
    cudaStream_t s = h->s;
    const int G = (int)h->groups.size();
    const bool mixed = h->opt.precision == 1;
    for (int t = 0; t < G; t++) {
        Group &g = h->groups[adjoint ? G - 1 - t : t];
        for (int p = g.p0; p < g.p1; p++) {
            const int k = h->order[p];
            double *rk = g.K.b.p + (h->offs[k] - g.base);
            const DCsr &C = adjoint ? h->go_upperT[k] : h->go_lower[k];
            if (C.nnz > 0 && !h->opt.jacobi) {
                Prof pf(h, 3, spmv_bytes(C, 8, 8, 1));
                coupling_sub<double, double, double>(C, v + h->offs[k], z, rk, s);
            } else {
                CK(cudaMemcpyAsync(rk, v + h->offs[k], sizeof(double) * (size_t)h->sizes[k],
                                   cudaMemcpyDeviceToDevice, s));
            }
        }
        fgmres_run(h, g.K, adjoint ? g.AT : g.A, h->opt.inner_restart, h->opt.inner_maxit, h->opt.inner_rtol,
                   [&](const double *vi, double *zi) {
                       if (mixed) group_sweep<float, float, __nv_bfloat16>(h, g, vi, zi, adjoint);
                       else group_sweep<double, double, double>(h, g, vi, zi, adjoint);
                   },
                   nullptr, nullptr);
        CK(cudaMemcpyAsync(z + g.base, g.K.x.p, sizeof(double) * (size_t)g.n, cudaMemcpyDeviceToDevice, s));
    }
}

// Rows of field k: the blocks (k, j) for the listed j, columns shifted by col_off(j); transposed:
// the blocks (j, k) transposed.
template <class Keep, class Off>
void coupling_rows(bgs_ctx *h, int k, bool transposed, Keep &&keep, Off &&col_off, DCsr &out, bool bf16) {
    cudaStream_t s = h->s;
    std::vector<DCsr> tr;
    tr.reserve(h->F);
    std::vector<CsrView> parts;
    std::vector<int> offs;
    for (int j = 0; j < h->F; j++) {
        if (!keep(j)) continue;
        const DCsr &B = transposed ? h->blk[(size_t)j * h->F + k] : h->blk[(size_t)k * h->F + j];
        if (B.nnz == 0) continue;
        if (transposed) {
            tr.emplace_back();
            transpose_csr(view(B), tr.back(), h->sc, s);
            parts.push_back(view(tr.back()));
        } else {
            parts.push_back(view(B));
        }
        offs.push_back((int)col_off(j));
    }
    out = DCsr();
    concat_rows((int)h->sizes[k], (int)parts.size(), parts.data(), offs.data(), out, h->sc, s);
    build_sell(out, kMaxPad, h->sc, s);
    if (bf16 && out.nnz) {
        out.vb.alloc((size_t)out.nnz, s);
        convert_d2bf(out.v.p, out.vb.p, out.nnz, s);
        sell_refresh(out, s);
    }
    CK(cudaStreamSynchronize(s));
}

void build_groups(bgs_ctx *h) {
    h->groups.clear();
    const int G = h->opt.ngroups;
    if (G <= 0) return;
    cudaStream_t s = h->s;
    const bool mixed = h->opt.precision == 1;
    std::vector<int> grp((size_t)h->F);
    h->groups.resize((size_t)G);
    for (int g = 0; g < G; g++) {
        Group &gr = h->groups[g];
        gr.p0 = g ? h->opt.group_end[g - 1] : 0;
        gr.p1 = h->opt.group_end[g];
        gr.base = INT64_MAX;
        gr.n = 0;
        for (int p = gr.p0; p < gr.p1; p++) {
            const int k = h->order[p];
            grp[k] = g;
            gr.base = std::min(gr.base, h->offs[k]);
            gr.n += h->sizes[k];
        }
    }
    for (int g = 0; g < G; g++) {
        Group &gr = h->groups[g];
        // the group's diagonal block: its fields' rows in field-id (memory) order, local columns
        std::vector<DCsr> rows((size_t)h->F);
        std::vector<DCsr *> rb;
        for (int k = 0; k < h->F; k++) {
            if (grp[k] != g) continue;
            coupling_rows(h, k, false, [&](int j) { return grp[j] == g; },
                          [&](int j) { return h->offs[j] - gr.base; }, rows[k], false);
            rb.push_back(&rows[k]);
        }
        vstack(rb, (int)gr.n, gr.A, s);
        gr.A.m = (int)gr.n;
        build_sell(gr.A, kMaxPad, h->sc, s);
        build_dia(gr.A, kMaxPadDia, h->sc, s);
        transpose_csr(view(gr.A), gr.AT, h->sc, s);
        build_sell(gr.AT, kMaxPad, h->sc, s);
        build_dia(gr.AT, kMaxPadDia, h->sc, s);
        gr.K.alloc(gr.n, h->opt.inner_restart, s);
    }
    for (int k = 0; k < h->F; k++) {
        const int g = grp[k];
        const Group &gr = h->groups[g];
        const int pk = h->pos[k];
        coupling_rows(h, k, false, [&](int j) { return grp[j] < g; }, [&](int j) { return h->offs[j]; },
                      h->go_lower[k], false);
        h->go_lower[k].m = (int)total_n(h);
        coupling_rows(h, k, true, [&](int j) { return grp[j] > g; }, [&](int j) { return h->offs[j]; },
                      h->go_upperT[k], false);
        h->go_upperT[k].m = (int)total_n(h);
        coupling_rows(h, k, false, [&](int j) { return grp[j] == g && h->pos[j] < pk; },
                      [&](int j) { return h->offs[j] - gr.base; }, h->gi_lower[k], mixed);
        h->gi_lower[k].m = (int)gr.n;
        coupling_rows(h, k, true, [&](int j) { return grp[j] == g && h->pos[j] > pk; },
                      [&](int j) { return h->offs[j] - gr.base; }, h->gi_upperT[k], mixed);
        h->gi_upperT[k].m = (int)gr.n;
    }
    CK(cudaStreamSynchronize(s));
}

int fgmres(bgs_ctx *h, bool adjoint, bgs_info *info) {
    const DCsr &A = adjoint ? h->fullT : h->full;
    const bool nested = !h->groups.empty();
    const bool graph = !nested && h->opt.graph && !h->prof;
    CycleGraph *cg = graph ? &h->cyc[adjoint ? 1 : 0] : nullptr;
    if (cg && !cg->exec) build_cycle_graph(h, h->K, A, h->opt.restart, adjoint, *cg);
    const int st = fgmres_run(h, h->K, A, h->opt.restart, h->opt.maxit, h->opt.rtol,
                              [&](const double *v, double *z) {
                                  if (nested) apply_nested(h, v, z, adjoint);
                                  else apply_prec(h, v, z, adjoint);
                              },
                              info, cg);
    if (info) h->last_reorth = info->reorth;
    return st;
}

// ------------------------------------------------------------------ helpers for create/setup
void alloc_block(const bgs_csr &in, int64_t nr, int64_t nc, DCsr &out, cudaStream_t s) {
    out.n = (int)nr;
    out.m = (int)nc;
    out.nnz = in.nnz;
    out.rp.alloc((size_t)nr + 1, s);
    out.ci.alloc((size_t)in.nnz, s);
    out.v.alloc((size_t)in.nnz, s);
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// BGS_TRACE set (not "async"): wall time of the phases of bgs_create (stream synchronised at each
// mark)
struct CreateTrace {
    bool on = getenv("BGS_TRACE") != nullptr && strcmp(getenv("BGS_TRACE"), "async") != 0;
    cudaStream_t s;
    double t;
    explicit CreateTrace(cudaStream_t st) : s(st) {
        if (on) {
            cudaStreamSynchronize(s);
            t = now_ms();
        }
    }
    void mark(const char *what) {
        if (!on) return;
        cudaStreamSynchronize(s);
        const double n = now_ms();
        fprintf(stderr, "bgs-trace create %-22s %8.3f ms\n", what, n - t);
        t = n;
    }
};

// The stored blocks' copies (pinned host sources pulled by the SMs over the host link, device and
// pageable sources by cudaMemcpyAsync), then each block's validation, the error bits one slot per
// block, read back once.
int copy_and_validate(bgs_ctx *h, const int64_t *sizes, const bgs_csr *blocks, cudaStream_t s) {
    const int F = h->F;
    CreateTrace tr(s);
    std::vector<int> todo;   // r * F + c of the stored blocks
    std::vector<XferSeg> segs;
    for (int r = 0; r < F; r++)
        for (int c = 0; c < F; c++) {
            const bgs_csr &B = blocks[r * F + c];
            DCsr &D = h->blk[(size_t)r * F + c];
            if (B.nrows == 0 && B.nnz == 0) {
                D.n = (int)sizes[r];
                D.m = (int)sizes[c];
                D.nnz = 0;
                D.rp.alloc((size_t)sizes[r] + 1, s);
                CK(cudaMemsetAsync(D.rp.p, 0, sizeof(int) * ((size_t)sizes[r] + 1), s));
                continue;
            }
            alloc_block(B, sizes[r], sizes[c], D, s);
            todo.push_back(r * F + c);
            segs.push_back({B.rowptr, D.rp.p, sizeof(int) * ((size_t)D.n + 1)});
            if (B.nnz) {
                segs.push_back({B.col, D.ci.p, sizeof(int) * (size_t)B.nnz});
                segs.push_back({B.val, D.v.p, sizeof(double) * (size_t)B.nnz});
            }
        }
    DBuf<int> flags(std::max<size_t>(todo.size(), 1), s);
    tr.mark("  allocate block copies");
    // block by block: each block's copy on s, its validation on the side stream once the copy is
    // done, so a block's validation runs under the next block's copy (bound by the host link)
    h->sc.ensure_side();
    cudaStream_t vs = h->sc.side;
    CK(cudaEventRecord(h->sc.fork, s));
    CK(cudaStreamWaitEvent(vs, h->sc.fork, 0));   // the flags' allocation and the empty blocks
    size_t seg0 = 0;
    for (size_t i = 0; i < todo.size(); i++) {
        const int b = todo[i];
        const size_t nseg = h->blk[(size_t)b].nnz ? 3 : 1;
        transfer(std::vector<XferSeg>(segs.begin() + seg0, segs.begin() + seg0 + nseg), s);
        seg0 += nseg;
        CK(cudaEventRecord(h->sc.fork, s));
        CK(cudaStreamWaitEvent(vs, h->sc.fork, 0));
        validate_csr_launch(view(h->blk[(size_t)b]), b / F == b % F, flags.p + i, vs);
    }
    CK(cudaEventRecord(h->sc.fork, vs));
    CK(cudaStreamWaitEvent(s, h->sc.fork, 0));
    std::vector<int> hf(todo.size(), 0);
    if (!todo.empty())
        CK(cudaMemcpyAsync(hf.data(), flags.p, sizeof(int) * todo.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    tr.mark("  copies + validation");
    for (int f : hf)
        if (int st = validate_status(f)) return st;
    return BGS_OK;
}

__global__ void k_shift_rowptr(int n, const int *in, int off, int *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = in[i] + off;
}

// vertical stack of row blocks into one CSR
void vstack(const std::vector<DCsr *> &parts, int ncols, DCsr &C, cudaStream_t s) {
    int64_t n = 0, nnz = 0;
    for (auto *p : parts) {
        n += p->n;
        nnz += p->nnz;
    }
    if (nnz >= INT32_MAX) throw Error(BGS_INVALID_ARG, "operator has 2^31 or more entries");
    C.n = (int)n;
    C.m = ncols;
    C.nnz = nnz;
    C.rp.alloc((size_t)n + 1, s);
    C.ci.alloc((size_t)nnz, s);
    C.v.alloc((size_t)nnz, s);
    int64_t r0 = 0, e0 = 0;
    for (auto *p : parts) {
        if (p->n) {
            k_shift_rowptr<<<grid_for(p->n, 256), 256, 0, s>>>(p->n, p->rp.p, (int)e0, C.rp.p + r0);
            CK_LAUNCH();
        }
        if (p->nnz) {
            CK(cudaMemcpyAsync(C.ci.p + e0, p->ci.p, sizeof(int) * p->nnz, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(C.v.p + e0, p->v.p, sizeof(double) * p->nnz, cudaMemcpyDeviceToDevice, s));
        }
        r0 += p->n;
        e0 += p->nnz;
    }
    int last = (int)nnz;
    CK(cudaMemcpyAsync(C.rp.p + n, &last, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
}

// The full operator (field-blocked rows: row i of field r is blocks (r, 0..F-1) with global
// columns) and, per field k, the lower couplings {A_kj : pos(j) < pos(k)} with global columns,
// from the stored blocks (Sec. 2.2, Eq. block-splitting).
void assemble_operators(bgs_ctx *h, DCsr &full, DCsr *lower, cudaStream_t s) {
    const int F = h->F;
    const int64_t tot = total_n(h);
    // the full operator in place: every block row's row lengths into its rows of the row
    // pointer, one scan, then every block row's entries
    std::vector<std::vector<CsrView>> parts((size_t)F);
    std::vector<std::vector<int>> coffs((size_t)F);
    for (int r = 0; r < F; r++)
        for (int c = 0; c < F; c++) {
            DCsr &B = h->blk[(size_t)r * F + c];
            if (B.nnz == 0) continue;
            parts[r].push_back(view(B));
            coffs[r].push_back((int)h->offs[c]);
        }
    full.n = (int)tot;
    full.m = (int)tot;
    full.rp.alloc((size_t)tot + 1, s);
    for (int r = 0; r < F; r++)
        concat_count((int)h->sizes[r], (int)parts[r].size(), parts[r].data(), full.rp.p + h->offs[r], s);
    full.nnz = scan_exclusive(full.rp.p, full.rp.p, tot, h->sc, s);   // throws past 2^31 - 1 entries
    full.ci.alloc((size_t)full.nnz, s);
    full.v.alloc((size_t)full.nnz, s);
    for (int r = 0; r < F; r++)
        concat_fill((int)h->sizes[r], (int)parts[r].size(), parts[r].data(), coffs[r].data(),
                    full.rp.p + h->offs[r], full.ci.p, full.v.p, s);
    for (int k = 0; k < F; k++) {
        std::vector<CsrView> parts;
        std::vector<int> offs;
        for (int j = 0; j < F; j++) {
            if (h->pos[j] >= h->pos[k]) continue;
            DCsr &B = h->blk[(size_t)k * F + j];
            if (B.nnz == 0) continue;
            parts.push_back(view(B));
            offs.push_back((int)h->offs[j]);
        }
        concat_rows((int)h->sizes[k], (int)parts.size(), parts.data(), offs.data(), lower[k], h->sc, s);
        lower[k].m = (int)tot;
    }
}

void build_adjoint(bgs_ctx *h) {
    if (h->adjoint_ready) return;
    cudaStream_t s = h->s;
    // rebuilt from scratch: the targets may hold SELL copies of earlier values
    h->fullT = DCsr();
    for (int k = 0; k < h->F; k++) {
        h->upperT[k] = DCsr();
        for (auto &Lv : h->H[k].L) Lv.AT = DCsr();
    }
    transpose_csr(view(h->full), h->fullT, h->sc, s);
    build_sell(h->fullT, kMaxPad, h->sc, s);
    build_dia(h->fullT, kMaxPadDia, h->sc, s);
    for (int k = 0; k < h->F; k++) {
        // rows of field k: sum over pos(j) > pos(k) of A_jk^T (global columns)
        std::vector<DCsr> tr;
        std::vector<CsrView> parts;
        std::vector<int> offs;
        tr.reserve(h->F);
        for (int j = 0; j < h->F; j++) {
            if (h->pos[j] <= h->pos[k]) continue;
            DCsr &B = h->blk[(size_t)j * h->F + k];
            if (B.nnz == 0) continue;
            tr.emplace_back();
            transpose_csr(view(B), tr.back(), h->sc, s);
        }
        size_t t = 0;
        for (int j = 0; j < h->F; j++) {
            if (h->pos[j] <= h->pos[k]) continue;
            DCsr &B = h->blk[(size_t)j * h->F + k];
            if (B.nnz == 0) continue;
            parts.push_back(view(tr[t++]));
            offs.push_back((int)h->offs[j]);
        }
        concat_rows((int)h->sizes[k], (int)parts.size(), parts.data(), offs.data(), h->upperT[k], h->sc, s);
        h->upperT[k].m = (int)total_n(h);
        build_sell(h->upperT[k], kMaxPad, h->sc, s);
        if (h->opt.precision == 1 && h->upperT[k].nnz) {
            h->upperT[k].vb.alloc((size_t)h->upperT[k].nnz, s);
            convert_d2bf(h->upperT[k].v.p, h->upperT[k].vb.p, h->upperT[k].nnz, s);
            sell_refresh(h->upperT[k], s);
        }
        Hier &H = h->H[k];
        if (H.solver == 1) {
            ilu_build_transposed(H.ilu, H.iluT, h->sc, s);
            continue;
        }
        if (H.solver == 2) continue;   // a diagonal solve is its own transpose
        for (size_t l = 0; l + 1 < H.L.size(); l++) {
            transpose_csr(view(H.L[l].A), H.L[l].AT, h->sc, s);
            build_sell(H.L[l].AT, kMaxPad, h->sc, s);
            if (l == 0) build_dia(H.L[l].AT, kMaxPadDia, h->sc, s);
            if (h->opt.precision == 1) {
                H.L[l].AT.vf.alloc((size_t)H.L[l].AT.nnz, s);
                convert_d2f(H.L[l].AT.v.p, H.L[l].AT.vf.p, H.L[l].AT.nnz, s);
                sell_refresh(H.L[l].AT, s);
            }
        }
        H.build_inv_T(s);
    }
    CK(cudaStreamSynchronize(s));
    h->adjoint_ready = true;
}

AmgParams params_for(const bgs_ctx *h, int k) {
    return AmgParams{h->opt.theta[k], h->opt.cheb_degree[k], h->opt.max_coarse, h->opt.max_levels,
                     h->opt.power_iters, h->opt.filter_diag, h->opt.cheb_ratio, h->opt.cheb_boost,
                     h->opt.cheb_ellipse, h->opt.precision == 1 ? 1 : 0};
}

// Runs fn(k, stream, scratch) for every diagonal block: the hierarchies are independent, so
// each gets a host thread and a stream of its own (BGS_SERIAL_SETUP=1 runs them one by one).
template <class Fn>
int run_per_block(bgs_ctx *h, Fn &&fn) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    // The blocks with the largest drop tolerance coarsen slowest (more levels: a longer chain of
    // small, latency-bound steps after the shared level-0 work), so their streams get the greatest
    // priority: where the blocks share the GPU, their work is scheduled first and their tail
    // overlaps the others' bulk.  With equal tolerances every stream has the default priority.
    double tmin = 1e300, tmax = -1e300;
    for (int k = 0; k < h->F; k++) {
        tmin = std::min(tmin, h->opt.theta[k]);
        tmax = std::max(tmax, h->opt.theta[k]);
    }
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    for (int k = 0; k < h->F; k++)
        if (!h->bs[k]) {
            const int prio = (tmax > tmin && h->opt.theta[k] == tmax) ? greatest : least;
            CK(cudaStreamCreateWithPriority(&h->bs[k], cudaStreamNonBlocking, prio));
            h->bsc[k].init(h->bs[k]);
        }
    std::vector<int> st((size_t)h->F, BGS_OK);
    auto work = [&](int k) {
        try {
            CK(cudaSetDevice(dev));
            fn(k, h->bs[k], h->bsc[k]);
        } catch (const Error &e) {
            if (getenv("BGS_VERBOSE")) fprintf(stderr, "libbgs: block %d: %s\n", k, e.what());
            st[k] = e.status;
        } catch (const std::bad_alloc &) {
            st[k] = BGS_OOM;
        } catch (...) {
            st[k] = BGS_INTERNAL;
        }
    };
    if (h->F > 1 && !getenv("BGS_SERIAL_SETUP")) {
        std::vector<std::thread> th;
        for (int k = 0; k < h->F; k++) th.emplace_back(work, k);
        for (auto &t : th) t.join();
    } else {
        for (int k = 0; k < h->F; k++) work(k);
    }
    for (int k = 0; k < h->F; k++)
        if (st[k]) return st[k];
    return BGS_OK;
}

template <class F>
int guarded(F &&f) {
    try {
        return f();
    } catch (const Error &e) {
        if (getenv("BGS_VERBOSE")) fprintf(stderr, "libbgs: %s\n", e.what());
        return e.status;
    } catch (const std::bad_alloc &) {
        return BGS_OOM;
    } catch (...) {
        return BGS_INTERNAL;
    }
}


}  // namespace

// ================================================================== C ABI
extern "C" {

int bgs_default_options(bgs_options *o) {
    if (!o) return BGS_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->restart = 50;
    o->maxit = 1000;
    o->rtol = 1e-8;
    o->precision = 0;
    o->graph = 1;
    o->autotune = 1;
    for (int k = 0; k < 8; k++) {
        o->cheb_degree[k] = 2;
        o->theta[k] = 0.0;
    }
    o->theta[0] = 0.04;
    o->cheb_degree[0] = 4;
    o->cheb_degree[1] = 4;
    o->max_coarse = 500;        /* dense coarsest solve on the GPU; the paper's 5000 fits a sparse CPU solver */
    o->max_levels = 10;
    o->cheb_ratio = 30.0;
    o->cheb_boost = 1.1;
    o->power_iters = 10;
    o->filter_diag = 1;
    o->reorth_eta = 0.01;
    o->jacobi = 0;
    for (int k = 0; k < 8; k++) o->subsolver[k] = 0;
    o->ilu_rows = 4096;
    o->ngroups = 0;
    for (int k = 0; k < 8; k++) o->group_end[k] = 0;
    o->inner_restart = 30;
    o->inner_maxit = 30;
    o->inner_rtol = 1e-6;
    o->cheb_ellipse = 0;
    return BGS_OK;
}

const char *bgs_status_string(int st) {
    switch (st) {
        case BGS_OK: return "ok";
        case BGS_INVALID_ARG: return "invalid argument";
        case BGS_NOT_SETUP: return "bgs_setup has not run";
        case BGS_NO_CONVERGENCE: return "no convergence within maxit";
        case BGS_BREAKDOWN: return "Arnoldi breakdown";
        case BGS_NAN_INF: return "NaN or Inf encountered";
        case BGS_ZERO_PIVOT: return "zero pivot in the coarsest LU or a zero diagonal";
        case BGS_CUDA_ERROR: return "CUDA error";
        case BGS_OOM: return "device out of memory";
        case BGS_INTERNAL: return "internal error";
        default: return "unknown status";
    }
}

int bgs_create(bgs_handle *out, int F, const int64_t *sizes, const bgs_csr *blocks, const int *order,
               const bgs_options *opt, void *stream) {
    if (!out || !sizes || !blocks || !order || F < 1 || F > 8) return BGS_INVALID_ARG;
    *out = nullptr;
    bgs_options o;
    if (opt) o = *opt;
    else bgs_default_options(&o);
    if (o.restart < 1 || o.restart > 63 || o.maxit < 1 || !(o.rtol > 0) || o.max_coarse < 1 || o.max_levels < 1 ||
        o.max_levels > kMaxLevels ||
        o.precision < 0 || o.precision > 1 || o.power_iters < 1 || !(o.cheb_ratio > 1.0) || !(o.cheb_boost > 0) ||
        !(o.reorth_eta >= 0.0) || o.jacobi < 0 || o.jacobi > 1 || o.ilu_rows < 1 || o.ilu_rows > kIluMaxRows ||
        o.cheb_ellipse < 0 || o.cheb_ellipse > 1)
        return BGS_INVALID_ARG;
    // host-side shape checks
    int seen[8] = {};
    for (int p = 0; p < F; p++) {
        if (order[p] < 0 || order[p] >= F || seen[order[p]]) return BGS_INVALID_ARG;
        seen[order[p]] = 1;
    }
    int64_t tot = 0;
    for (int k = 0; k < F; k++) {
        if (sizes[k] < 1 || sizes[k] >= INT32_MAX) return BGS_INVALID_ARG;
        tot += sizes[k];
        if (o.cheb_degree[k] < 1 || o.theta[k] < 0 || o.subsolver[k] < 0 || o.subsolver[k] > 2)
            return BGS_INVALID_ARG;
    }
    if (tot >= INT32_MAX) return BGS_INVALID_ARG;
    if (o.ngroups < 0 || o.ngroups > F) return BGS_INVALID_ARG;
    if (o.ngroups > 0) {
        if (o.inner_restart < 1 || o.inner_restart > 63 || o.inner_maxit < 1 || !(o.inner_rtol > 0))
            return BGS_INVALID_ARG;
        int prev = 0;
        for (int g = 0; g < o.ngroups; g++) {
            const int e = o.group_end[g];
            if (e <= prev || e > F) return BGS_INVALID_ARG;
            int lo = F, hi = -1;   // the group's field ids must be consecutive
            for (int p = prev; p < e; p++) {
                lo = std::min(lo, order[p]);
                hi = std::max(hi, order[p]);
            }
            if (hi - lo + 1 != e - prev) return BGS_INVALID_ARG;
            prev = e;
        }
        if (prev != F) return BGS_INVALID_ARG;
    }
    for (int r = 0; r < F; r++)
        for (int c = 0; c < F; c++) {
            const bgs_csr &B = blocks[r * F + c];
            const bool zero = B.nrows == 0 && B.nnz == 0;
            if (r == c && zero) return BGS_INVALID_ARG;
            if (zero) continue;
            if (B.nrows != sizes[r] || B.ncols != sizes[c] || B.nnz < 0 || B.nnz >= INT32_MAX || !B.rowptr)
                return BGS_INVALID_ARG;
            if (B.nnz > 0 && (!B.col || !B.val)) return BGS_INVALID_ARG;
        }
    std::unique_ptr<bgs_ctx> h(new bgs_ctx());
    return guarded([&]() -> int {
        h->s = (cudaStream_t)stream;
        h->F = F;
        h->opt = o;
        h->offs[0] = 0;
        for (int k = 0; k < F; k++) {
            h->sizes[k] = sizes[k];
            h->offs[k + 1] = h->offs[k] + sizes[k];
            h->order[k] = order[k];
            h->pos[order[k]] = k;
        }
        cudaStream_t s = h->s;
        CreateTrace tr(s);
        h->sc.init(s);
        h->blk.resize((size_t)F * F);
        if (int st = copy_and_validate(h.get(), sizes, blocks, s)) return st;
        tr.mark("copy+validate blocks");
        assemble_operators(h.get(), h->full, h->lower, s);
        tr.mark("full operator + couplings");
        // the layouts the autotuner will choose from (only its cached choice when it has one)
        const bool tune = o.autotune != 0;
        bool equal = F >= 2;
        for (int k = 1; k < F; k++) equal = equal && sizes[k] == sizes[0];
        build_formats(h->full, 8, true, tune, h->sc, s, true, equal ? F : 0);
        for (int k = 0; k < F; k++) build_formats(h->lower[k], o.precision == 1 ? 2 : 8, false, tune, h->sc, s);
        CK(cudaStreamSynchronize(s));
        tr.mark("sell");
        *out = h.release();
        return BGS_OK;
    });
}

namespace {

__global__ void k_diag_recip(int n, const int *rp, const int *ci, const double *v, double *dinv, int *zero) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; e++)
            if (ci[e] == i) d = v[e];
        if (d == 0.0) *zero = 1;
        dinv[i] = 1.0 / d;
    }
}

// Lv.dinv = 1 / diag(Lv.A) (and its FP32 copy in mixed precision); a zero diagonal entry is a zero
// pivot of the diagonal solve.
void diag_reciprocal(Level &Lv, bool mixed, Scratch &sc, cudaStream_t s) {
    const int n = Lv.A.n;
    if (Lv.dinv.n != (size_t)n) Lv.dinv.alloc((size_t)n, s);
    CK(cudaMemsetAsync(sc.flags.p + 13, 0, sizeof(int), s));
    if (n > 0) {
        k_diag_recip<<<grid_for(n, 256), 256, 0, s>>>(n, Lv.A.rp.p, Lv.A.ci.p, Lv.A.v.p, Lv.dinv.p, sc.flags.p + 13);
        CK_LAUNCH();
    }
    if (mixed) {
        if (Lv.dinvf.n != (size_t)n) Lv.dinvf.alloc((size_t)n, s);
        convert_d2f(Lv.dinv.p, Lv.dinvf.p, n, s);
    }
    CK(cudaMemcpyAsync(sc.h_flags + 13, sc.flags.p + 13, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sc.h_flags[13]) throw Error(BGS_ZERO_PIVOT, "zero diagonal entry in a block on the diagonal solve");
}

// Builds block k's hierarchy and its solve-side copies on stream sk (no timing-based tuning here).
void build_block(bgs_ctx *h, int k, cudaStream_t sk, Scratch &sck) {
    const bool mixed = h->opt.precision == 1;
    Hier &H = h->H[k];
    H = Hier();
    H.L.reserve(32);
    H.L.emplace_back();
    DCsr &B = h->blk[(size_t)k * h->F + k];
    DCsr &A0 = H.L[0].A;
    A0.n = B.n;
    A0.m = B.m;
    A0.nnz = B.nnz;
    A0.rp.alloc((size_t)B.n + 1, sk);
    A0.ci.alloc((size_t)B.nnz, sk);
    A0.v.alloc((size_t)B.nnz, sk);
    CK(cudaMemcpyAsync(A0.rp.p, B.rp.p, sizeof(int) * ((size_t)B.n + 1), cudaMemcpyDeviceToDevice, sk));
    CK(cudaMemcpyAsync(A0.ci.p, B.ci.p, sizeof(int) * B.nnz, cudaMemcpyDeviceToDevice, sk));
    CK(cudaMemcpyAsync(A0.v.p, B.v.p, sizeof(double) * B.nnz, cudaMemcpyDeviceToDevice, sk));
    if (h->opt.subsolver[k] == 2) {   // diagonal solve: 1 / diag(A_kk) on level 0 only
        H.solver = 2;
        diag_reciprocal(H.L[0], mixed, sck, sk);
        if (mixed) Buf<float>::alloc(H.L[0], A0.n, sk);
        else Buf<double>::alloc(H.L[0], A0.n, sk);
        CK(cudaStreamSynchronize(sk));
        return;
    }
    if (h->opt.subsolver[k] == 1) {   // DD(0)-ILU(0): factors of level 0 only
        H.solver = 1;
        ilu_setup(H.ilu, A0, h->opt.ilu_rows, mixed, sck, sk);
        if (mixed) Buf<float>::alloc(H.L[0], A0.n, sk);
        else Buf<double>::alloc(H.L[0], A0.n, sk);
        CK(cudaStreamSynchronize(sk));
        return;
    }
    amg_build(H, params_for(h, k), sck, sk);
    timeline_mark("hierarchy built", sk);
    if (H.status) throw Error(H.status, "coarsest-level factorisation");
    // the SpMV layouts of the level operators (the diagonal-offset form for the level-0 stencil
    // operator only, whose offsets repeat); only the autotuner's cached choice when it has one
    for (size_t l = 0; l + 1 < H.L.size(); l++)
        for (DCsr *M : {&H.L[l].A, &H.L[l].P, &H.L[l].R})
            build_formats(*M, mixed ? 4 : 8, M == &H.L[0].A, h->opt.autotune != 0, sck, sk);
    for (size_t l = 0; l < H.L.size(); l++) {
        Level &Lv = H.L[l];
        if (mixed) {
            Buf<float>::alloc(Lv, Lv.A.n, sk);
            if (l + 1 < H.L.size()) {
                for (DCsr *M : {&Lv.A, &Lv.P, &Lv.R}) {
                    if (M->vf.n != (size_t)M->nnz) {   // the FP32 Galerkin products made most already
                        M->vf.alloc((size_t)M->nnz, sk);
                        convert_d2f(M->v.p, M->vf.p, M->nnz, sk);
                    }
                    sell_refresh(*M, sk);
                }
                Lv.dinvf.alloc((size_t)Lv.A.n, sk);
                convert_d2f(Lv.dinv.p, Lv.dinvf.p, Lv.A.n, sk);
            }
        } else {
            Buf<double>::alloc(Lv, Lv.A.n, sk);
        }
    }
    CK(cudaStreamSynchronize(sk));
    timeline_mark("block done", sk);
}

}  // namespace

extern "C" int bgs_setup(bgs_handle h) {
    if (!h) return BGS_INVALID_ARG;
    return guarded([&]() -> int {
        cudaStream_t s = h->s;
        CK(cudaStreamSynchronize(s));
        const double t0 = now_ms();
        const bool mixed = h->opt.precision == 1;
        const int st = run_per_block(h, [&](int k, cudaStream_t sk, Scratch &sck) { build_block(h, k, sk, sck); });
        if (st) return st;
        timeline_mark("all blocks built", s);
        // kernel choice by timing runs alone, after the concurrent build
        for (int k = 0; k < h->F; k++)
            if (mixed && h->lower[k].nnz) {
                h->lower[k].vb.alloc((size_t)h->lower[k].nnz, s);
                convert_d2bf(h->lower[k].v.p, h->lower[k].vb.p, h->lower[k].nnz, s);
                sell_refresh(h->lower[k], s);
            }
        if (h->opt.autotune) {
            const int hb = mixed ? 4 : 8, cb = mixed ? 2 : 8;
            for (int k = 0; k < h->F; k++) {
                Hier &H = h->H[k];
                for (size_t l = 0; l + 1 < H.L.size(); l++)
                    for (DCsr *M : {&H.L[l].A, &H.L[l].P, &H.L[l].R}) autotune_spmv(*M, hb, h->sc, s);
                if (h->lower[k].nnz) autotune_spmv(h->lower[k], cb, h->sc, s);
            }
            autotune_spmv(h->full, 8, h->sc, s, true);   // applied only as a product
        }
        h->K.alloc(total_n(h), h->opt.restart, s);
        if (mixed) h->zf.alloc((size_t)total_n(h), s);
        build_groups(h);
        h->adjoint_ready = false;
        drop_graphs(h);
        CK(cudaStreamSynchronize(s));
        h->t_setup_ms = now_ms() - t0;
        h->setup_done = true;
        timeline_mark("setup done", s);
        return BGS_OK;
    });
}

extern "C" int bgs_update_values(bgs_handle h, const double *const *values) {
    if (!h || !values) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    return guarded([&]() -> int {
        cudaStream_t s = h->s;
        CK(cudaStreamSynchronize(s));
        const double t0 = now_ms();
        const int F = h->F;
        const bool mixed = h->opt.precision == 1;
        std::vector<XferSeg> segs;
        for (int b = 0; b < F * F; b++)
            if (values[b] && h->blk[b].nnz) segs.push_back({values[b], h->blk[b].v.p, sizeof(double) * (size_t)h->blk[b].nnz});
        transfer(segs, s);
        {
            // the full operator and the couplings: re-assembled, then their values taken over so
            // that their SELL layouts and tuned kernels stay
            DCsr full2, lower2[8];
            assemble_operators(h, full2, lower2, s);
            CK(cudaMemsetAsync(h->sc.flags.p + 10, 0, sizeof(int), s));
            take_values(h->full, full2, h->sc, s);
            for (int k = 0; k < F; k++)
                if (h->lower[k].nnz) take_values(h->lower[k], lower2[k], h->sc, s);
            CK(cudaMemcpyAsync(h->sc.h_flags + 10, h->sc.flags.p + 10, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (h->sc.h_flags[10]) throw Error(BGS_INTERNAL, "re-assembled operator has a different pattern");
        }
        const int st = run_per_block(h, [&](int k, cudaStream_t sk, Scratch &sck) {
            Hier &H = h->H[k];
            const DCsr &B = h->blk[(size_t)k * F + k];
            DCsr &A0 = H.L[0].A;
            CK(cudaMemcpyAsync(A0.v.p, B.v.p, sizeof(double) * (size_t)B.nnz, cudaMemcpyDeviceToDevice, sk));
            refresh_values(A0, sk);
            if (H.solver == 2) {
                diag_reciprocal(H.L[0], mixed, sck, sk);
                CK(cudaStreamSynchronize(sk));
                return;
            }
            if (H.solver == 1) {
                ilu_update(H.ilu, A0, sck, sk);
                CK(cudaStreamSynchronize(sk));
                return;
            }
            amg_update(H, params_for(h, k), sck, sk);
            if (H.status) throw Error(H.status, "coarsest-level factorisation");
            if (mixed)
                for (size_t l = 0; l + 1 < H.L.size(); l++)
                    convert_d2f(H.L[l].dinv.p, H.L[l].dinvf.p, H.L[l].A.n, sk);
            CK(cudaStreamSynchronize(sk));
        });
        if (st) return st;
        build_groups(h);
        h->adjoint_ready = false;
        drop_graphs(h);
        CK(cudaStreamSynchronize(s));
        h->t_setup_ms = now_ms() - t0;
        return BGS_OK;
    });
}

static int solve_common(bgs_handle h, const double *b, double *x, bgs_info *info, bool adjoint) {
    if (!h || !b || !x) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    return guarded([&]() -> int {
        cudaStream_t s = h->s;
        const int64_t n = total_n(h);
        if (adjoint) build_adjoint(h);
        CK(cudaStreamSynchronize(s));
        const double t0 = now_ms();
        for (auto &k : h->stats) k = KStats();
        transfer({{b, h->K.b.p, sizeof(double) * (size_t)n}}, s);
        bgs_info inf{};
        int st = fgmres(h, adjoint, &inf);
        transfer({{h->K.x.p, x, sizeof(double) * (size_t)n}}, s);
        CK(cudaStreamSynchronize(s));
        inf.t_solve_ms = now_ms() - t0;
        inf.t_setup_ms = h->t_setup_ms;
        for (int k = 0; k < h->F; k++) inf.nlevels[k] = (int)h->H[k].L.size();
        prof_collect(h);
        if (info) *info = inf;
        return st;
    });
}

int bgs_solve(bgs_handle h, const double *b, double *x, bgs_info *info) {
    return solve_common(h, b, x, info, false);
}

int bgs_solve_adjoint(bgs_handle h, const double *g, double *lambda, bgs_info *info) {
    return solve_common(h, g, lambda, info, true);
}

int bgs_grad_values_all(bgs_handle h, const double *lambda, const double *x, double *const *dvals) {
    if (!h || !lambda || !x || !dvals) return BGS_INVALID_ARG;
    return guarded([&]() -> int {
        for (int r = 0; r < h->F; r++)
            for (int c = 0; c < h->F; c++) {
                DCsr &B = h->blk[(size_t)r * h->F + c];
                double *d = dvals[r * h->F + c];
                if (!d || B.nnz == 0) continue;
                grad_outer(view(B), lambda + h->offs[r], x + h->offs[c], d, h->s);
            }
        CK(cudaStreamSynchronize(h->s));
        return BGS_OK;
    });
}

int bgs_grad_values(bgs_handle h, int rf, int cf, const double *lambda, const double *x, double *dvals) {
    if (!h || rf < 0 || cf < 0 || rf >= h->F || cf >= h->F || !lambda || !x || !dvals) return BGS_INVALID_ARG;
    return guarded([&]() -> int {
        DCsr &B = h->blk[(size_t)rf * h->F + cf];
        grad_outer(view(B), lambda + h->offs[rf], x + h->offs[cf], dvals, h->s);
        CK(cudaStreamSynchronize(h->s));
        return BGS_OK;
    });
}

int bgs_apply_preconditioner(bgs_handle h, const double *v, double *z) {
    if (!h || !v || !z) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    return guarded([&]() -> int {
        if (!h->groups.empty()) apply_nested(h, v, z, false);
        else apply_prec(h, v, z, false);
        CK(cudaStreamSynchronize(h->s));
        return BGS_OK;
    });
}

int bgs_apply_vcycle(bgs_handle h, int field, const double *b, double *x) {
    if (!h || field < 0 || field >= h->F || !b || !x) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    return guarded([&]() -> int {
        Hier &H = h->H[field];
        const int64_t n = h->sizes[field];
        if (h->opt.precision == 1) {
            copy_in<float>(b, Buf<float>::b(H.L[0]), n, h->s);
            float *r = block_solve<float, float>(h, H, false);
            copy_out<float>(r, x, n, h->s);
        } else {
            copy_in<double>(b, Buf<double>::b(H.L[0]), n, h->s);
            double *r = block_solve<double, double>(h, H, false);
            copy_out<double>(r, x, n, h->s);
        }
        CK(cudaStreamSynchronize(h->s));
        return BGS_OK;
    });
}

int bgs_full_spmv(bgs_handle h, const double *x, double *y) {
    if (!h || !x || !y) return BGS_INVALID_ARG;
    return guarded([&]() -> int {
        spmv_store<double, double>(h->full, x, y, h->s);
        CK(cudaStreamSynchronize(h->s));
        return BGS_OK;
    });
}

int bgs_num_levels(bgs_handle h, int field, int *nlevels) {
    if (!h || field < 0 || field >= h->F || !nlevels) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    *nlevels = (int)h->H[field].L.size();
    return BGS_OK;
}

int bgs_level_info(bgs_handle h, int field, int level, int64_t *rows, int64_t *nnz, int64_t *p_nnz, int *nagg,
                   int *mis_rounds, double *omega, double *lmin, double *lmax) {
    if (!h || field < 0 || field >= h->F) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    Hier &H = h->H[field];
    if (level < 0 || level >= (int)H.L.size()) return BGS_INVALID_ARG;
    Level &L = H.L[level];
    if (rows) *rows = L.A.n;
    if (nnz) *nnz = L.A.nnz;
    if (p_nnz) *p_nnz = L.P.nnz;
    if (nagg) *nagg = L.nagg;
    if (mis_rounds) *mis_rounds = L.mis_rounds;
    if (omega) *omega = L.omega;
    if (lmin) *lmin = L.lmin;
    if (lmax) *lmax = L.lmax;
    return BGS_OK;
}

int bgs_level_copy(bgs_handle h, int field, int level, int which, int32_t *rowptr, int32_t *col, double *val) {
    if (!h || field < 0 || field >= h->F || which < 0 || which > 2) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    Hier &H = h->H[field];
    if (level < 0 || level >= (int)H.L.size()) return BGS_INVALID_ARG;
    if (which > 0 && level + 1 >= (int)H.L.size()) return BGS_INVALID_ARG;
    return guarded([&]() -> int {
        Level &L = H.L[level];
        const DCsr &M = which == 0 ? L.A : (which == 1 ? L.P : L.R);
        cudaStream_t s = h->s;
        if (rowptr) CK(cudaMemcpyAsync(rowptr, M.rp.p, sizeof(int) * ((size_t)M.n + 1), cudaMemcpyDeviceToHost, s));
        if (col && M.nnz) CK(cudaMemcpyAsync(col, M.ci.p, sizeof(int) * M.nnz, cudaMemcpyDeviceToHost, s));
        if (val && M.nnz) CK(cudaMemcpyAsync(val, M.v.p, sizeof(double) * M.nnz, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return BGS_OK;
    });
}

int bgs_level_ellipse(bgs_handle h, int field, int level, double *imag) {
    if (!h || field < 0 || field >= h->F || !imag) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    const Hier &H = h->H[field];
    if (level < 0 || level >= (int)H.L.size()) return BGS_INVALID_ARG;
    *imag = H.L[level].lim;
    return BGS_OK;
}

int bgs_ilu_factors(bgs_handle h, int field, int64_t *nnz, int32_t *rowptr, int32_t *col, double *val) {
    if (!h || field < 0 || field >= h->F || !nnz) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    const Hier &H = h->H[field];
    if (H.solver != 1) return BGS_INVALID_ARG;
    return guarded([&]() -> int {
        const DCsr &F = H.ilu.F;
        *nnz = F.nnz;
        if (rowptr) CK(cudaMemcpyAsync(rowptr, F.rp.p, sizeof(int) * ((size_t)F.n + 1), cudaMemcpyDefault, h->s));
        if (col && F.nnz) CK(cudaMemcpyAsync(col, F.ci.p, sizeof(int) * (size_t)F.nnz, cudaMemcpyDefault, h->s));
        if (val && F.nnz) CK(cudaMemcpyAsync(val, F.v.p, sizeof(double) * (size_t)F.nnz, cudaMemcpyDefault, h->s));
        CK(cudaStreamSynchronize(h->s));
        return BGS_OK;
    });
}

int bgs_level_format(bgs_handle h, int field, int level, int which, int *format, int *threads_per_block) {
    if (!h || which < 0 || which > 3 || !format) return BGS_INVALID_ARG;
    if (!h->setup_done && which != 3) return BGS_NOT_SETUP;   // the full operator exists from create on
    const DCsr *Mp = &h->full;
    if (which < 3) {
        if (field < 0 || field >= h->F) return BGS_INVALID_ARG;
        Hier &H = h->H[field];
        if (level < 0 || level >= (int)H.L.size()) return BGS_INVALID_ARG;
        if (which > 0 && level + 1 >= (int)H.L.size()) return BGS_INVALID_ARG;
        Mp = which == 0 ? &H.L[level].A : (which == 1 ? &H.L[level].P : &H.L[level].R);
    }
    const DCsr &M = *Mp;
    *format = M.bsr_active() ? -2 : (M.dia ? -1 : (M.sell ? 0 : (M.lanes ? M.lanes : choose_lanes(M.n, M.nnz))));
    if (threads_per_block) *threads_per_block = M.tpb;
    return BGS_OK;
}

int bgs_level_aggregates(bgs_handle h, int field, int level, int32_t *agg) {
    if (!h || field < 0 || field >= h->F || !agg) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    Hier &H = h->H[field];
    if (level < 0 || level + 1 >= (int)H.L.size()) return BGS_INVALID_ARG;
    return guarded([&]() -> int {
        Level &L = H.L[level];
        CK(cudaMemcpyAsync(agg, L.agg.p, sizeof(int) * (size_t)L.A.n, cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        return BGS_OK;
    });
}

int bgs_level_strength(bgs_handle h, int field, int level, uint8_t *strong) {
    if (!h || field < 0 || field >= h->F || !strong) return BGS_INVALID_ARG;
    if (!h->setup_done) return BGS_NOT_SETUP;
    Hier &H = h->H[field];
    if (level < 0 || level + 1 >= (int)H.L.size()) return BGS_INVALID_ARG;
    return guarded([&]() -> int {
        Level &L = H.L[level];
        if (L.A.nnz)
            CK(cudaMemcpyAsync(strong, L.strong.p, (size_t)L.A.nnz, cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        return BGS_OK;
    });
}

int bgs_set_profiling(bgs_handle h, int on) {
    if (!h) return BGS_INVALID_ARG;
    h->prof = on != 0;
    return BGS_OK;
}

int bgs_kernel_stats(bgs_handle h, int cls, int64_t *launches, double *ms, double *bytes) {
    if (!h || cls < 0 || cls > 5) return BGS_INVALID_ARG;
    if (launches) *launches = h->stats[cls].launches;
    if (ms) *ms = h->stats[cls].ms;
    if (bytes) *bytes = h->stats[cls].bytes;
    return BGS_OK;
}

int bgs_csr_spmv(int64_t nrows, int64_t nnz, const int32_t *rowptr, const int32_t *col, const double *val,
                 const double *x, double *y, int lanes, void *stream) {
    if (nrows < 0 || nnz < 0 || nrows >= INT32_MAX || nnz >= INT32_MAX) return BGS_INVALID_ARG;
    if (nrows > 0 && (!rowptr || !x || !y)) return BGS_INVALID_ARG;
    if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32)
        return BGS_INVALID_ARG;
    return guarded([&]() -> int {
        CsrView A{(int)nrows, 0, nnz, rowptr, col, val};
        spmv_f64(A, lanes, x, y, (cudaStream_t)stream);
        return BGS_OK;
    });
}

int bgs_arnoldi_dots(const double *V, int64_t ld, int cnt, const double *w, int64_t n, double *h, void *stream) {
    if (!V || !w || !h || n < 1 || cnt < 1 || cnt > 64 || ld < n || (ld & 1)) return BGS_INVALID_ARG;
    if (((uintptr_t)V | (uintptr_t)w) & 15) return BGS_INVALID_ARG;   // read as 16-byte pairs
    return guarded([&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        DBuf<double> part(arnoldi_dots_scratch(cnt, n, 0), s);
        arnoldi_dots_into(V, ld, cnt, w, n, h, part.p, part.n, 0, s);
        return BGS_OK;
    });
}

int bgs_gram_schmidt_pass(const double *V, int64_t ld, int cnt, double *w, int64_t n, double *h, double *nw,
                          void *stream) {
    if (!V || !w || !h || !nw || n < 1 || cnt < 1 || cnt > 64 || ld < n || (ld & 1)) return BGS_INVALID_ARG;
    if (((uintptr_t)V | (uintptr_t)w) & 15) return BGS_INVALID_ARG;   // read as 16-byte pairs
    return guarded([&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        DBuf<double> part(gs_pass_scratch(cnt, n), s);
        gs_pass(V, ld, cnt, w, n, h, nw, part.p, part.n, s);
        return BGS_OK;
    });
}

int64_t bgs_launch_count(void) { return (int64_t)launch_count(); }

int bgs_release_cached_memory(void) {
    return guarded([&]() -> int {
        release_cached_memory();
        return BGS_OK;
    });
}

void bgs_destroy(bgs_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->s);
    for (int k = 0; k < 8; k++) {
        if (!h->bs[k]) continue;
        cudaStreamSynchronize(h->bs[k]);
        h->H[k] = Hier();   // released on the block's stream
        cudaStreamSynchronize(h->bs[k]);
    }
    if (h->gs) cudaStreamSynchronize(h->gs);
    drop_graphs(h);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    for (auto &e : h->join_ev)
        if (e) cudaEventDestroy(e);
    if (h->gs) cudaStreamDestroy(h->gs);
    for (auto &e : h->ev) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    cudaStream_t s = h->s;
    cudaStream_t bs[8];
    for (int k = 0; k < 8; k++) bs[k] = h->bs[k];
    delete h;
    cudaStreamSynchronize(s);
    for (int k = 0; k < 8; k++)
        if (bs[k]) {
            cudaStreamSynchronize(bs[k]);
            cudaStreamDestroy(bs[k]);
        }
}

}  // extern "C"
