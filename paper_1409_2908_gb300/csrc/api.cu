// C ABI entry points (include/fmm.h): argument validation, peeling geometry
// (Section 3.5) and the launch sequence of one fast product.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fmm_internal.h"

using namespace fmm;

namespace {

thread_local int t_launches = 0;

// Optional event pairs around the leaf launch (fmm_timing_enable).
struct Timing {
    bool on = false;
    int device = -1;
    std::vector<cudaEvent_t> ev;   // 2 per call
    int used = 0;
    ~Timing() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    cudaEvent_t next() {
        if (used >= 2048) return nullptr;
        if (used >= (int)ev.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            ev.push_back(e);
        }
        return ev[used++];
    }
};
thread_local Timing t_timing;

}  // namespace

namespace fmm {
cudaEvent_t timing_mark(cudaStream_t s) {
    if (!t_timing.on) return nullptr;
    cudaEvent_t e = t_timing.next();
    if (e) cudaEventRecord(e, s);
    return e;
}
void timing_unmark() {
    if (t_timing.used > 0) --t_timing.used;
}
void set_last_launch_count(int n) { t_launches = n; }
}  // namespace fmm

namespace {

int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes) {
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + bbytes && y < x + abytes;
}

// Bytes spanned by an m x n row-major matrix with leading dimension ld.
size_t span(int64_t m, int64_t n, int64_t ld) { return size_t(((m - 1) * ld + n) * 8); }

fmm_status check_operands(const double *A, int64_t lda, const double *B, int64_t ldb,
                          const double *C, int64_t ldc, int64_t m, int64_t k, int64_t n) {
    if (!A || !B || !C) return FMM_ERR_ARG;
    if (m < 1 || k < 1 || n < 1) return FMM_ERR_ARG;
    if (m > (int64_t(1) << 31) || k > (int64_t(1) << 31) || n > (int64_t(1) << 31))
        return FMM_ERR_ARG;
    if (lda < k || ldb < n || ldc < n) return FMM_ERR_ARG;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 7) return FMM_ERR_ARG;
    if (overlaps(C, span(m, n, ldc), A, span(m, k, lda)) ||
        overlaps(C, span(m, n, ldc), B, span(k, n, ldb)))
        return FMM_ERR_ARG;
    return FMM_OK;
}

struct Geometry {
    int64_t mp, kp, np, mL, kL, nL;
    bool fast;  // a nonempty core for the fast algorithm
};

Geometry geometry(const fmm_plan *p, int64_t m, int64_t k, int64_t n) {
    Geometry g{};
    const int64_t sm = ipow(p->M, p->L), sk = ipow(p->K, p->L), sn = ipow(p->N, p->L);
    g.mp = (m / sm) * sm;
    g.kp = (k / sk) * sk;
    g.np = (n / sn) * sn;
    g.mL = g.mp / sm;
    g.kL = g.kp / sk;
    g.nL = g.np / sn;
    g.fast = p->L > 0 && g.mp > 0 && g.kp > 0 && g.np > 0;
    if (p->L == 0) {
        g.mp = m; g.kp = k; g.np = n; g.mL = m; g.kL = k; g.nL = n;
    }
    return g;
}

struct WsLayout {
    size_t slotA = 0, slotB = 0, prod = 0, oz = 0, total = 0;
    // level-by-level scheme: offsets of each level's S, T and product buffers
    std::vector<size_t> lvS, lvT, lvP;
};

// Leaf products on the TF32 tensor path: one TF32 product per leaf, or three
// (TF32 pairs) for FP32 accuracy.
bool tf32_family(const fmm_plan *p) { return p->prec == FMM_PREC_TF32 || p->prec == FMM_PREC_FP32; }
int tf32_split(const fmm_plan *p) { return p->prec == FMM_PREC_FP32 ? 3 : 1; }

// The whole recursion runs on residues when the base coefficients are
// integers (the plan layer checks) and per-leaf emulation was not asked for.
bool residue_space(const fmm_plan *p) {
    if (!p->integer_coefs || (p->flags & FMM_FLAG_LEAF_EMULATION)) return false;
    // the residue kernels stage one level's term lists in shared memory
    auto nnz = [](const std::vector<double> &F) {
        size_t c = 0;
        for (double x : F) c += x != 0.0;
        return c;
    };
    return p->R <= 64 && p->M * p->N <= 64 && nnz(p->U) <= 512 && nnz(p->V) <= 512 && nnz(p->W) <= 512;
}

ResPlan res_plan(const fmm_plan *p) {
    ResPlan rp{};
    rp.M = p->M; rp.K = p->K; rp.N = p->N; rp.R = p->R; rp.L = p->L;
    rp.u_ptr = p->dev.lu_ptr; rp.u_code = p->dev.lu_code; rp.u_icoef = p->dev.lu_icoef;
    rp.v_ptr = p->dev.lv_ptr; rp.v_code = p->dev.lv_code; rp.v_icoef = p->dev.lv_icoef;
    rp.vt_code = p->dev.lvt_code;
    rp.w_ptr = p->dev.lw_ptr; rp.w_r = p->dev.lw_r; rp.w_icoef = p->dev.lw_icoef;
    rp.tile = p->tile;
    rp.fused_s = (p->flags & FMM_FLAG_TC_FUSED_S) != 0;
    rp.hU = p->U.data();
    rp.w_absmax = 0;
    for (int q = 0; q < p->M * p->N; ++q) {
        double sum = 0;
        for (int r = 0; r < p->R; ++r) sum += std::fabs(p->W[size_t(q) * p->R + r]);
        rp.w_absmax = std::max(rp.w_absmax, int(sum));
    }
    rp.u_absmax = rp.v_absmax = 0;
    for (int r = 0; r < p->R; ++r) {
        double su = 0, sv = 0;
        for (int i = 0; i < p->M * p->K; ++i) su += std::fabs(p->U[size_t(i) * p->R + r]);
        for (int j = 0; j < p->K * p->N; ++j) sv += std::fabs(p->V[size_t(j) * p->R + r]);
        rp.u_absmax = std::max(rp.u_absmax, int(su));
        rp.v_absmax = std::max(rp.v_absmax, int(sv));
    }
    return rp;
}

WsLayout ws_layout(const fmm_plan *p, const Geometry &g) {
    WsLayout w;
    const bool tf = tf32_family(p);
    const bool oz = p->prec == FMM_PREC_OZAKI_BF16 || tf;
    if (tf && p->L == 0) {
        w.oz = 0;
        w.total = tf32_workspace(1, g.mp, g.kp, g.np, tf32_split(p));
        return w;
    }
    if (!tf && oz && p->L > 0 && g.fast && residue_space(p)) {
        w.oz = 0;
        w.total = ozaki_fast_workspace(res_plan(p), g.mp, g.kp, g.np, p->nmod);
        return w;
    }
    if (oz && p->L == 0) {
        // the whole product is one emulated product (the residue path with no level)
        w.oz = 0;
        w.total = ozaki_fast_workspace(res_plan(p), g.mp, g.kp, g.np, p->nmod);
        return w;
    }
    if (!g.fast) return w;
    size_t off = 0;
    const bool lw = oz || (p->flags & FMM_FLAG_LEVELWISE);
    if (oz || !(p->flags & FMM_FLAG_FUSED_ST)) {
        if (lw) {
            int64_t cnt = 1;
            for (int l = 1; l <= p->L; ++l) {
                cnt *= p->R;
                w.lvS.push_back(off);
                off = align256(off + size_t(cnt) * (g.mp / ipow(p->M, l)) * (g.kp / ipow(p->K, l)) * 8);
            }
            cnt = 1;
            for (int l = 1; l <= p->L; ++l) {
                cnt *= p->R;
                w.lvT.push_back(off);
                off = align256(off + size_t(cnt) * (g.kp / ipow(p->K, l)) * (g.np / ipow(p->N, l)) * 8);
            }
        } else {
            w.slotA = off;
            off = align256(off + size_t(p->slots_a) * g.mL * g.kL * 8);
            w.slotB = off;
            off = align256(off + size_t(p->slots_b) * g.kL * g.nL * 8);
        }
    }
    if (oz || !(p->flags & FMM_FLAG_FUSED_W)) {
        if (lw) {
            int64_t cnt = 1;
            for (int l = 1; l <= p->L; ++l) {
                cnt *= p->R;
                w.lvP.push_back(off);
                off = align256(off + size_t(cnt) * (g.mp / ipow(p->M, l)) * (g.np / ipow(p->N, l)) * 8);
            }
            w.prod = w.lvP.back();
        } else {
            w.prod = off;
            off = align256(off + size_t(p->leaves) * g.mL * g.nL * 8);
        }
    }
    if (oz) {
        w.oz = off;
        off = align256(off + (tf ? tf32_workspace(p->leaves, g.mL, g.kL, g.nL, tf32_split(p))
                                 : ozaki_workspace(p->leaves, p->nmod, g.mL, g.kL, g.nL)));
    }
    w.total = off;
    return w;
}

fmm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return FMM_OK;
    return e == cudaErrorMemoryAllocation ? FMM_ERR_NO_MEMORY : FMM_ERR_CUDA;
}

int device_sms() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Copy the unrolled lists to the device on first use (plan creation itself
// needs no GPU).
fmm_status ensure_uploaded(fmm_plan *p) {
    std::lock_guard<std::mutex> g(p->upload_mu);
    if (p->uploaded) return FMM_OK;
    fmm_status st;
    try {
        st = upload_plan(p);
    } catch (const std::bad_alloc &) {
        st = FMM_ERR_NO_MEMORY;
    }
    if (st == FMM_OK) {
        p->uploaded = true;
        cudaGetDevice(&p->upload_device);
    }
    return st;
}

// Record a timing pair around one launch sequence (no-op unless enabled).
template <class F>
cudaError_t timed(cudaStream_t s, F &&f) {
    cudaEvent_t a = timing_mark(s);
    cudaError_t e = f();
    cudaEvent_t b = timing_mark(s);
    if (a && !b) timing_unmark();   // keep pairs aligned
    return e;
}

// Where a path has no place for the host overlap: wait for B now and drop
// the hooks (the caller then copies C out after the whole product).
cudaError_t settle_pipe(const HostPipe *&pipe, cudaStream_t s) {
    if (!pipe) return cudaSuccess;
    // A's bands follow B on one stream: the last of them implies all
    const cudaEvent_t last = pipe->a_bands > 0 ? pipe->a_ready[pipe->a_bands - 1] : pipe->b_ready;
    const cudaError_t e = last ? cudaStreamWaitEvent(s, last, 0) : cudaSuccess;
    pipe = nullptr;
    return e;
}

// Side stream and events of the host entry point, one set per thread and
// device (created on first use).
constexpr int kMaxABands = 8;
struct HostSide {
    int device = -1;
    cudaStream_t side = nullptr;
    cudaEvent_t start = nullptr, b_in = nullptr, band = nullptr, side_done = nullptr;
    cudaEvent_t a_in[kMaxABands] = {};
    void release() {
        for (cudaEvent_t *ev : {&start, &b_in, &band, &side_done})
            if (*ev) cudaEventDestroy(*ev), *ev = nullptr;
        for (cudaEvent_t &ev : a_in)
            if (ev) cudaEventDestroy(ev), ev = nullptr;
        if (side) cudaStreamDestroy(side), side = nullptr;
        device = -1;
    }
    ~HostSide() { release(); }
};
thread_local HostSide t_host;

HostSide *host_side() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (t_host.device == dev) return &t_host;
    t_host.release();
    if (cudaStreamCreateWithFlags(&t_host.side, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    for (cudaEvent_t *ev : {&t_host.start, &t_host.b_in, &t_host.band, &t_host.side_done})
        if (cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) {
            t_host.release();
            return nullptr;
        }
    for (cudaEvent_t &ev : t_host.a_in)
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            t_host.release();
            return nullptr;
        }
    t_host.device = dev;
    return &t_host;
}

// rows x cols doubles between host and device, one flat copy when both sides
// are packed
cudaError_t copy_rows(void *dst, int64_t dld, const void *src, int64_t sld, int64_t rows, int64_t cols,
                      cudaMemcpyKind kind, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (dld == cols && sld == cols) return cudaMemcpyAsync(dst, src, size_t(rows * cols * 8), kind, s);
    return cudaMemcpy2DAsync(dst, size_t(dld * 8), src, size_t(sld * 8), size_t(cols * 8), size_t(rows), kind, s);
}

// fmm_set_host_pipeline (0: from the sizes)
thread_local int t_bands = 0, t_gemm_bands = 0;

// Row bands of C copied out while the last pass still writes the next ones:
// about 32 MiB of C per band, at most 8.
int host_bands(int64_t m, int64_t n) {
    if (t_bands > 0) return t_bands;
    const double mib = double(m) * double(n) * 8.0 / 1048576.0;
    return (int)std::min(8.0, std::max(1.0, std::floor(mib / 32.0)));
}

// Row bands of the residue products: each band of S is multiplied by all of
// T, so T is read once per band.
int host_gemm_bands(int bands) {
    if (t_gemm_bands > 0) return t_gemm_bands;
    return std::min(bands, 4);
}

struct BandCopy {
    cudaStream_t s, side;
    cudaEvent_t ev;
    double *hostC;
    int64_t ldc;
    const double *devC;
    int64_t n;
    int64_t rows_done;
};

// HostPipe::band_done of the host entry point: the band's rows of every
// block row, copied on the side stream after the pass that wrote them.
cudaError_t copy_band(void *ctx, int64_t r0, int64_t r1, int64_t block_rows, int count) {
    BandCopy *b = (BandCopy *)ctx;
    cudaError_t e;
    if ((e = cudaEventRecord(b->ev, b->s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(b->side, b->ev, 0)) != cudaSuccess) return e;
    for (int a = 0; a < count; ++a) {
        const int64_t row = a * block_rows + r0;
        if ((e = copy_rows(b->hostC + row * b->ldc, b->ldc, b->devC + row * b->n, b->n, r1 - r0, b->n,
                           cudaMemcpyDeviceToHost, b->side)) != cudaSuccess)
            return e;
    }
    b->rows_done += (r1 - r0) * count;
    return cudaSuccess;
}

// One recursive level of S (side 0, from parents with an M x K block grid)
// or T (side 1, K x N) in the plan's addition scheme (Section 3.2):
// write-once, streaming or pairwise.
cudaError_t form_level(const fmm_plan *p, int side, const double *par, int64_t pld, int64_t pst,
                       int64_t parents, int64_t rows, int64_t cols, double *out, cudaStream_t s, int *launches) {
    const int gR = side ? p->K : p->M, gC = side ? p->N : p->K;
    const int *ptr = side ? p->dev.lv_ptr : p->dev.lu_ptr, *code = side ? p->dev.lv_code : p->dev.lu_code;
    const double *coef = side ? p->dev.lv_coef : p->dev.lu_coef;
    const std::vector<double> &F = side ? p->V : p->U;
    size_t nnz = 0;
    for (double x : F) nnz += x != 0.0;
    if ((p->flags & FMM_FLAG_STREAMING) && nnz <= 512 && p->R <= 128 && gR * gC <= 64)
        return launch_level_stream(par, pld, pst, parents, rows, cols, gR, gC, p->R, ptr, code, coef, out, s,
                                   launches);
    if (p->flags & FMM_FLAG_PAIRWISE) {
        const int64_t per = rows * cols;
        for (int r = 0; r < p->R; ++r) {
            bool first = true;
            for (int i = 0; i < gR * gC; ++i) {
                const double c = F[size_t(i) * p->R + r];
                if (c == 0.0) continue;
                const double *X = par + (int64_t)(i / gC) * rows * pld + (int64_t)(i % gC) * cols;
                cudaError_t e = launch_block_axpy(X, pld, pst, out + r * per, cols, p->R * per, parents, rows,
                                                  cols, c, first ? 1 : 0, s, launches);
                if (e != cudaSuccess) return e;
                first = false;
            }
            if (first) {   // no terms: the child is zero (0 x, inputs are finite)
                cudaError_t e = launch_block_axpy(par, pld, pst, out + r * per, cols, p->R * per, parents, rows,
                                                  cols, 0.0, 1, s, launches);
                if (e != cudaSuccess) return e;
            }
        }
        return cudaSuccess;
    }
    return launch_level_form(par, pld, pst, parents, rows, cols, p->R, ptr, code, coef, out, s, launches);
}

// One recursive level of the W combination in the plan's addition scheme:
// the MN blocks of each parent (ld pld, parents pst apart) from its R child
// products (packed rows x cols, consecutive).
cudaError_t w_level(const fmm_plan *p, const double *child, int64_t rows, int64_t cols, double *parent,
                    int64_t pld, int64_t pst, int64_t parents, int accumulate, cudaStream_t s, int *launches) {
    const int MN = p->M * p->N;
    size_t nnz = 0;
    for (double x : p->W) nnz += x != 0.0;
    if ((p->flags & FMM_FLAG_STREAMING) && nnz <= 512 && p->R <= 128 && MN <= 128)
        return launch_level_w_stream(child, rows, cols, p->R, p->N, MN, parent, pld, pst, parents, p->dev.lw_ptr,
                                     p->dev.lw_r, p->dev.lw_coef, accumulate, s, launches);
    if (p->flags & FMM_FLAG_PAIRWISE) {
        const int64_t per = rows * cols;
        for (int q = 0; q < MN; ++q) {
            double *Y = parent + (int64_t)(q / p->N) * rows * pld + (int64_t)(q % p->N) * cols;
            bool first = !accumulate;
            bool any = false;
            for (int r = 0; r < p->R; ++r) {
                const double w = p->W[size_t(q) * p->R + r];
                if (w == 0.0) continue;
                cudaError_t e = launch_block_axpy(child + r * per, cols, p->R * per, Y, pld, pst, parents, rows,
                                                  cols, w, first ? 1 : 0, s, launches);
                if (e != cudaSuccess) return e;
                first = false;
                any = true;
            }
            if (!any && !accumulate) {
                cudaError_t e = launch_block_axpy(child, cols, p->R * per, Y, pld, pst, parents, rows, cols, 0.0, 1,
                                                  s, launches);
                if (e != cudaSuccess) return e;
            }
        }
        return cudaSuccess;
    }
    return launch_level_w(child, rows, cols, p->R, p->N, MN, parent, pld, pst, parents, p->dev.lw_ptr, p->dev.lw_r,
                          p->dev.lw_coef, accumulate, s, launches);
}

// Emulated-FP64 leaves: FP64 level-by-level S/T, tensor-core residue
// products, FP64 level-by-level W; classical FP64 fringe.
fmm_status run_gemm_ozaki(fmm_plan *p, const Geometry &g, const WsLayout &wl, const double *A,
                          int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc,
                          int64_t m, int64_t k, int64_t n, char *wsb, cudaStream_t s,
                          int *launches, const HostPipe *pipe, GemmDefer *defer = nullptr) {
    cudaError_t e;
    // the overlap hooks reach only the residue-space path without a fringe
    const bool fringe = g.mp < m || g.kp < k || g.np < n;
    if (tf32_family(p) || (p->L > 0 && (!residue_space(p) || fringe)))
        if ((e = settle_pipe(pipe, s)) != cudaSuccess) return cuda_status(e);
    // (the timing pair, when enabled, brackets the tensor-core GEMM inside)
    const bool tf = tf32_family(p);
    auto leaf_products = [&](const double *S_, int64_t lds, int64_t ss, const double *T_, int64_t ldt,
                             int64_t ts, double *Out, int64_t ldo, int64_t os, int64_t leaves,
                             int64_t mm, int64_t kk, int64_t nn) {
        return tf ? tf32_products(S_, lds, ss, T_, ldt, ts, Out, ldo, os, leaves, mm, kk, nn, 0,
                                  wsb + wl.oz, s, launches, tf32_split(p), p->tile)
                  : ozaki_products(S_, lds, ss, T_, ldt, ts, Out, ldo, os, leaves, mm, kk, nn, p->nmod,
                                   wsb + wl.oz, s, launches, p->tile);
    };
    if (defer && (tf || (p->L > 0 && !residue_space(p)))) return FMM_ERR_UNSUPPORTED;
    if (p->L == 0)
        return cuda_status(tf ? leaf_products(A, lda, 0, B, ldb, 0, C, ldc, 0, 1, m, k, n)
                              : ozaki_fast(res_plan(p), A, lda, B, ldb, C, ldc, m, k, n, p->nmod, 0, wsb, s,
                                           launches, pipe, defer));
    if (!tf && residue_space(p)) {
        const bool kfr = g.kp < k;
        // (two phases: the k-fringe before, the row and column fringes after the GEMM)
        const bool first = !defer || defer->phase == 0, last = !defer || defer->phase == 1;
        if (first && kfr && (e = launch_classical(A + g.kp, lda, B + g.kp * ldb, ldb, C, ldc, g.mp, k - g.kp,
                                                  g.np, FMM_TILE_AUTO, s, launches)) != cudaSuccess)
            return cuda_status(e);
        if ((e = ozaki_fast(res_plan(p), A, lda, B, ldb, C, ldc, g.mp, g.kp, g.np, p->nmod,
                            kfr ? 1 : 0, wsb + wl.oz, s, launches, pipe, defer)) != cudaSuccess)
            return cuda_status(e);
        if (!last) return FMM_OK;
        if (g.mp < m &&
            (e = launch_classical(A + g.mp * lda, lda, B, ldb, C + g.mp * ldc, ldc, m - g.mp, k, n,
                                  FMM_TILE_AUTO, s, launches)) != cudaSuccess)
            return cuda_status(e);
        if (g.np < n &&
            (e = launch_classical(A, lda, B + g.np, ldb, C + g.np, ldc, g.mp, k, n - g.np,
                                  FMM_TILE_AUTO, s, launches)) != cudaSuccess)
            return cuda_status(e);
        return FMM_OK;
    }
    const double *pa = A, *pb = B;
    int64_t pld_a = lda, pld_b = ldb, pst_a = 0, pst_b = 0, parents = 1;
    double *prod = (double *)(wsb + wl.lvP.back());
    // TF32-family leaves one level deep: the level fused with the conversion
    // (each operand read once, S and T formed in FP32), no FP64 S/T levels
    auto nnz = [](const std::vector<double> &F) {
        size_t c = 0;
        for (double x : F) c += x != 0.0;
        return c;
    };
    auto grid_ok = [](int nb) { return nb == 4 || nb == 6 || nb == 8 || nb == 9; };
    const bool tf_fused = tf && p->L == 1 && p->R <= 64 && grid_ok(p->M * p->K) && grid_ok(p->K * p->N) &&
                          nnz(p->U) <= 512 && nnz(p->V) <= 512;
    if (tf_fused) {
        if ((e = tf32_first_level_products(A, lda, B, ldb, g.mL, g.kL, g.nL, p->M, p->K, p->N, p->R, p->dev.lu_ptr,
                                           p->dev.lu_code, p->dev.lu_coef, p->dev.lv_ptr, p->dev.lv_code,
                                           p->dev.lv_coef, (float *)prod, g.nL, g.mL * g.nL, wsb + wl.oz, s,
                                           launches, tf32_split(p), p->tile)) != cudaSuccess)
            return cuda_status(e);
    }
    for (int l = 1; l <= p->L && !tf_fused; ++l) {
        const int64_t ml = g.mp / ipow(p->M, l), kl = g.kp / ipow(p->K, l), nl = g.np / ipow(p->N, l);
        double *oa = (double *)(wsb + wl.lvS[l - 1]);
        double *ob = (double *)(wsb + wl.lvT[l - 1]);
        if ((e = form_level(p, 0, pa, pld_a, pst_a, parents, ml, kl, oa, s, launches)) != cudaSuccess)
            return cuda_status(e);
        if ((e = form_level(p, 1, pb, pld_b, pst_b, parents, kl, nl, ob, s, launches)) != cudaSuccess)
            return cuda_status(e);
        pa = oa; pld_a = kl; pst_a = ml * kl;
        pb = ob; pld_b = nl; pst_b = kl * nl;
        parents *= p->R;
    }
    if (!tf_fused && (e = leaf_products(pa, g.kL, g.mL * g.kL, pb, g.nL, g.kL * g.nL, prod, g.nL, g.mL * g.nL,
                                        p->leaves, g.mL, g.kL, g.nL)) != cudaSuccess)
        return cuda_status(e);
    const bool kfringe = g.kp < k;
    if (kfringe &&
        (e = launch_classical(A + g.kp, lda, B + g.kp * ldb, ldb, C, ldc, g.mp, k - g.kp, g.np,
                              FMM_TILE_AUTO, s, launches)) != cudaSuccess)
        return cuda_status(e);
    // the fused level's FP32 products: W in FP32 straight into C
    if (tf_fused && (e = tf32_w_level((const float *)prod, g.mL, g.nL, p->M, p->N, p->dev.lw_ptr, p->dev.lw_r,
                                      p->dev.lw_coef, C, ldc, kfringe ? 1 : 0, s, launches)) != cudaSuccess)
        return cuda_status(e);
    int64_t lparents = ipow(p->R, p->L - 1);
    for (int l = p->L; l >= 1 && !tf_fused; --l) {
        const int64_t ml = g.mp / ipow(p->M, l), nl = g.np / ipow(p->N, l);
        const double *child = (const double *)(wsb + wl.lvP[l - 1]);
        double *parent = l == 1 ? C : (double *)(wsb + wl.lvP[l - 2]);
        const int64_t pld = l == 1 ? ldc : nl * p->N;
        const int64_t pst = l == 1 ? 0 : (ml * p->M) * (nl * p->N);
        if ((e = w_level(p, child, ml, nl, parent, pld, pst, lparents, (l == 1 && kfringe) ? 1 : 0, s,
                         launches)) != cudaSuccess)
            return cuda_status(e);
        lparents /= p->R;
    }
    if (g.mp < m &&
        (e = launch_classical(A + g.mp * lda, lda, B, ldb, C + g.mp * ldc, ldc, m - g.mp, k, n,
                              FMM_TILE_AUTO, s, launches)) != cudaSuccess)
        return cuda_status(e);
    if (g.np < n &&
        (e = launch_classical(A, lda, B + g.np, ldb, C + g.np, ldc, g.mp, k, n - g.np,
                              FMM_TILE_AUTO, s, launches)) != cudaSuccess)
        return cuda_status(e);
    return FMM_OK;
}

// The fast core plus the classical fringe, all on one stream.  pipe: the
// host entry point's overlap hooks (or null); paths that cannot use them wait
// for B first and drop them.
fmm_status run_gemm(fmm_plan *p, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *C, int64_t ldc, int64_t m, int64_t k, int64_t n, void *ws,
                    size_t ws_bytes, cudaStream_t s, int *launches, const HostPipe *pipe = nullptr,
                    GemmDefer *defer = nullptr) {
    const Geometry g = geometry(p, m, k, n);
    const bool emulated = (p->prec == FMM_PREC_OZAKI_BF16 || tf32_family(p)) && (p->L == 0 || g.fast);
    if (defer && !emulated) return FMM_ERR_UNSUPPORTED;
    if (!emulated) {
        const cudaError_t pe = settle_pipe(pipe, s);
        if (pe != cudaSuccess) return cuda_status(pe);
    }
    if (emulated) {
        // int32 drain sums stay below 2^31 for k_L <= 65536 (2^23 per 512-chunk)
        if (g.kL > 65536) return FMM_ERR_UNSUPPORTED;
        const WsLayout wl = ws_layout(p, g);
        if (wl.total > 0 && (!ws || ws_bytes < wl.total)) return FMM_ERR_NO_MEMORY;
        if (wl.total > 0 && ((uintptr_t)ws & 255)) return FMM_ERR_ARG;
        const fmm_status us = ensure_uploaded(p);
        if (us != FMM_OK) return us;
        return run_gemm_ozaki(p, g, wl, A, lda, B, ldb, C, ldc, m, k, n, (char *)ws, s, launches, pipe, defer);
    }
    if (!g.fast)
        return cuda_status(timed(s, [&] {
            return launch_classical(A, lda, B, ldb, C, ldc, m, k, n, FMM_TILE_AUTO, s, launches);
        }));
    const WsLayout wl = ws_layout(p, g);
    if (wl.total > 0 && (!ws || ws_bytes < wl.total)) return FMM_ERR_NO_MEMORY;
    {
        const fmm_status us = ensure_uploaded(p);
        if (us != FMM_OK) return us;
    }
    if (wl.total > 0 && ((uintptr_t)ws & 255)) return FMM_ERR_ARG;
    char *wsb = (char *)ws;
    const bool fused_st = p->flags & FMM_FLAG_FUSED_ST;
    const bool fused_w = p->flags & FMM_FLAG_FUSED_W;
    cudaError_t e;

    const bool lw = p->flags & FMM_FLAG_LEVELWISE;
    // write-once S_r and T_r (unfused scheme)
    double *slotA = nullptr, *slotB = nullptr;
    if (!fused_st && lw) {
        // one recursive level at a time: level l forms R^l operands from R^(l-1)
        const double *pa = A, *pb = B;
        int64_t pld_a = lda, pld_b = ldb, pst_a = 0, pst_b = 0, parents = 1;
        for (int l = 1; l <= p->L; ++l) {
            const int64_t ml = g.mp / ipow(p->M, l), kl = g.kp / ipow(p->K, l), nl = g.np / ipow(p->N, l);
            double *oa = (double *)(wsb + wl.lvS[l - 1]);
            double *ob = (double *)(wsb + wl.lvT[l - 1]);
            if ((e = form_level(p, 0, pa, pld_a, pst_a, parents, ml, kl, oa, s, launches)) != cudaSuccess)
                return cuda_status(e);
            if ((e = form_level(p, 1, pb, pld_b, pst_b, parents, kl, nl, ob, s, launches)) != cudaSuccess)
                return cuda_status(e);
            pa = oa; pld_a = kl; pst_a = ml * kl;
            pb = ob; pld_b = nl; pst_b = kl * nl;
            parents *= p->R;
        }
        slotA = (double *)(wsb + wl.lvS.back());
        slotB = (double *)(wsb + wl.lvT.back());
    } else if (!fused_st) {
        slotA = (double *)(wsb + wl.slotA);
        slotB = (double *)(wsb + wl.slotB);
        if (p->slots_a > 0 &&
            (e = launch_form_slots(A, lda, g.mL, g.kL, p->slots_a, p->dev.sa_leaf, p->dev.a_ptr,
                                   p->dev.a_code, p->dev.a_coef, slotA, g.mL * g.kL, s,
                                   launches)) != cudaSuccess)
            return cuda_status(e);
        if (p->slots_b > 0 &&
            (e = launch_form_slots(B, ldb, g.kL, g.nL, p->slots_b, p->dev.sb_leaf, p->dev.b_ptr,
                                   p->dev.b_code, p->dev.b_coef, slotB, g.kL * g.nL, s,
                                   launches)) != cudaSuccess)
            return cuda_status(e);
    }
    // C[:m',:n'] starts as the k-fringe product A[:m',k':] B[k':,:n'], or zero
    const bool kfringe = g.kp < k;
    if (fused_w) {
        if (kfringe) {
            if ((e = launch_classical(A + g.kp, lda, B + g.kp * ldb, ldb, C, ldc, g.mp, k - g.kp,
                                      g.np, FMM_TILE_AUTO, s, launches)) != cudaSuccess)
                return cuda_status(e);
        } else {
            if ((e = cudaMemset2DAsync(C, ldc * 8, 0, g.np * 8, g.mp, s)) != cudaSuccess)
                return cuda_status(e);
        }
    }
    LeafLaunch L{};
    L.A = A; L.lda = lda; L.B = B; L.ldb = ldb; L.C = C; L.ldc = ldc;
    L.mL = g.mL; L.kL = g.kL; L.nL = g.nL; L.leaves = p->leaves;
    // Operand chains and the epilogue coefficient must agree: normalised
    // chains (first coefficient 1) pair with W * sA * sB; true-valued
    // operands (level-wise slots, or raw chains feeding level-wise W) pair
    // with the plain W.
    bool raw_values = false;
    if (fused_st) {
        raw_values = lw && !fused_w;
        L.a_ptr = p->dev.a_ptr; L.a_code = p->dev.a_code;
        L.a_coef = raw_values ? p->dev.a_coef_raw : p->dev.a_coef;
        L.b_ptr = p->dev.b_ptr; L.b_code = p->dev.b_code;
        L.b_coef = raw_values ? p->dev.b_coef_raw : p->dev.b_coef;
    } else if (lw) {
        raw_values = true;
        L.a_ptr = p->dev.ua_ptr; L.a_code = p->dev.leaf_slot; L.a_coef = p->dev.u_one;
        L.b_ptr = p->dev.ub_ptr; L.b_code = p->dev.leaf_slot; L.b_coef = p->dev.u_one;
        L.slotA = slotA; L.slotA_stride = g.mL * g.kL;
        L.slotB = slotB; L.slotB_stride = g.kL * g.nL;
    } else {
        L.a_ptr = p->dev.ua_ptr; L.a_code = p->dev.ua_code; L.a_coef = p->dev.u_one;
        L.b_ptr = p->dev.ub_ptr; L.b_code = p->dev.ub_code; L.b_coef = p->dev.u_one;
        L.slotA = slotA; L.slotA_stride = g.mL * g.kL;
        L.slotB = slotB; L.slotB_stride = g.kL * g.nL;
    }
    L.c_ptr = p->dev.c_ptr; L.c_code = p->dev.c_code;
    L.c_coef = raw_values ? p->dev.c_coef_raw : p->dev.c_coef;
    double *wsM = fused_w ? nullptr : (double *)(wsb + wl.prod);
    L.wsM = wsM;
    L.epi = fused_w ? EPI_ATOMIC : EPI_WORKSPACE;
    const double extra_a = fused_st ? double(p->a.row.size()) / double(p->leaves) - 1.0 : 0.0;
    const double extra_b = fused_st ? double(p->b.row.size()) / double(p->leaves) - 1.0 : 0.0;
    L.tile = resolve_tile(p->tile, g.mL, g.nL, g.kL, p->leaves, extra_a, extra_b, device_sms());
    if ((e = timed(s, [&] { return launch_leaf_gemm(L, s, launches); })) != cudaSuccess)
        return cuda_status(e);
    if (!fused_w) {
        if (kfringe &&
            (e = launch_classical(A + g.kp, lda, B + g.kp * ldb, ldb, C, ldc, g.mp, k - g.kp, g.np,
                                  FMM_TILE_AUTO, s, launches)) != cudaSuccess)
            return cuda_status(e);
        if (lw) {
            // combine level by level, from the leaf products up to C
            int64_t parents = ipow(p->R, p->L - 1);
            for (int l = p->L; l >= 1; --l) {
                const int64_t ml = g.mp / ipow(p->M, l), nl = g.np / ipow(p->N, l);
                const double *child = (const double *)(wsb + wl.lvP[l - 1]);
                double *parent = l == 1 ? C : (double *)(wsb + wl.lvP[l - 2]);
                const int64_t pld = l == 1 ? ldc : nl * p->N;
                const int64_t pst = l == 1 ? 0 : (ml * p->M) * (nl * p->N);
                if ((e = w_level(p, child, ml, nl, parent, pld, pst, parents, (l == 1 && kfringe) ? 1 : 0, s,
                                 launches)) != cudaSuccess)
                    return cuda_status(e);
                parents /= p->R;
            }
        } else {
            const int64_t gridN = ipow(p->N, p->L), blocks = ipow(p->M, p->L) * gridN;
            if ((e = launch_w_pass(C, ldc, g.mL, g.nL, int(gridN), blocks, p->dev.cq_ptr,
                                   p->dev.cq_leaf, p->dev.cq_coef, wsM, kfringe ? 1 : 0, s,
                                   launches)) != cudaSuccess)
                return cuda_status(e);
        }
    }
    // fringe rows and columns (Section 3.5)
    if (g.mp < m &&
        (e = launch_classical(A + g.mp * lda, lda, B, ldb, C + g.mp * ldc, ldc, m - g.mp, k, n,
                              FMM_TILE_AUTO, s, launches)) != cudaSuccess)
        return cuda_status(e);
    if (g.np < n &&
        (e = launch_classical(A, lda, B + g.np, ldb, C + g.np, ldc, g.mp, k, n - g.np,
                              FMM_TILE_AUTO, s, launches)) != cudaSuccess)
        return cuda_status(e);
    return FMM_OK;
}

}  // namespace

extern "C" {

const char *fmm_status_string(fmm_status st) {
    switch (st) {
        case FMM_OK: return "ok";
        case FMM_ERR_ARG: return "invalid argument";
        case FMM_ERR_INVALID_ALGORITHM: return "factor matrices fail the Brent equations";
        case FMM_ERR_UNSUPPORTED: return "unsupported request";
        case FMM_ERR_NO_MEMORY: return "out of memory or workspace too small";
        case FMM_ERR_CUDA: return "CUDA error";
        case FMM_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

int fmm_last_launch_count(void) { return t_launches; }

fmm_status fmm_plan_create(fmm_plan_t *out, int M, int K, int N, int R, const double *U,
                           const double *V, const double *W, int levels, fmm_precision prec,
                           unsigned flags) {
    if (!out || !U || !V || !W) return FMM_ERR_ARG;
    if (M < 1 || K < 1 || N < 1 || R < 1 || R > 4096) return FMM_ERR_ARG;
    if (int64_t(M) * K * K * N * M * N > (int64_t(1) << 22)) return FMM_ERR_UNSUPPORTED;
    if (levels < 0 || levels > 6) return FMM_ERR_ARG;
    if (prec != FMM_PREC_FP64 && prec != FMM_PREC_OZAKI_BF16 && prec != FMM_PREC_TF32 && prec != FMM_PREC_FP32)
        return FMM_ERR_UNSUPPORTED;
    if (flags & ~unsigned(FMM_FLAG_FUSED_ST | FMM_FLAG_FUSED_W | FMM_FLAG_LEVELWISE |
                          FMM_FLAG_LEAF_EMULATION | FMM_FLAG_STREAMING | FMM_FLAG_PAIRWISE |
                          FMM_FLAG_TC_FUSED_S))
        return FMM_ERR_ARG;
    if ((flags & FMM_FLAG_STREAMING) && (flags & FMM_FLAG_PAIRWISE)) return FMM_ERR_ARG;
    bool representable = true;
    if (!brent_exact(M, K, N, R, U, V, W, &representable))
        return representable ? FMM_ERR_INVALID_ALGORITHM : FMM_ERR_UNSUPPORTED;
    fmm_plan *p = new (std::nothrow) fmm_plan();
    if (!p) return FMM_ERR_NO_MEMORY;
    p->flags = flags;
    p->prec = prec;
    cudaGetDevice(&p->device);
    fmm_status st;
    try {
        st = build_plan(p, M, K, N, R, U, V, W, levels);
    } catch (const std::bad_alloc &) {
        st = FMM_ERR_NO_MEMORY;
    }
    if (st != FMM_OK) {
        free_plan_device(p);
        delete p;
        return st;
    }
    *out = p;
    return FMM_OK;
}

fmm_status fmm_plan_load(fmm_plan_t *out, const char *path, int levels, fmm_precision prec,
                         unsigned flags) {
    if (!out || !path) return FMM_ERR_ARG;
    int M, K, N, R;
    std::vector<double> U, V, W;
    fmm_status st;
    try {
        st = parse_fmm_file(path, &M, &K, &N, &R, &U, &V, &W);
    } catch (const std::bad_alloc &) {
        return FMM_ERR_NO_MEMORY;
    }
    if (st != FMM_OK) return st;
    return fmm_plan_create(out, M, K, N, R, U.data(), V.data(), W.data(), levels, prec, flags);
}

void fmm_plan_destroy(fmm_plan_t p) {
    if (!p) return;
    free_plan_device(p);
    delete p;
}

fmm_status fmm_plan_set_tile(fmm_plan_t p, fmm_tile tile) {
    if (!p || tile < FMM_TILE_AUTO || tile > FMM_TILE_64x128) return FMM_ERR_ARG;
    p->tile = tile;
    return FMM_OK;
}

fmm_status fmm_plan_prepare(fmm_plan_t p) {
    if (!p) return FMM_ERR_ARG;
    fmm_status st = ensure_uploaded(p);
    if (st != FMM_OK) return st;
    if (p->prec == FMM_PREC_OZAKI_BF16 && ozaki_prepare(p->nmod) != cudaSuccess) return FMM_ERR_CUDA;
    if (tf32_family(p) && tf32_prepare() != cudaSuccess) return FMM_ERR_CUDA;
    if (prepare_fp64_kernels() != cudaSuccess) return FMM_ERR_CUDA;
    return FMM_OK;
}

fmm_status fmm_plan_set_moduli(fmm_plan_t p, int n_moduli) {
    if (!p || p->prec != FMM_PREC_OZAKI_BF16 || n_moduli < 3 || n_moduli > 16) return FMM_ERR_ARG;
    p->nmod = n_moduli;
    return FMM_OK;
}

fmm_status fmm_check_device_error(void) {
    int flag = 0, flag2 = 0;
    if (read_device_error(&flag, true) != cudaSuccess) return FMM_ERR_CUDA;
    if (read_tf32_error(&flag2, true) != cudaSuccess) return FMM_ERR_CUDA;
    return (flag || flag2) ? FMM_ERR_TIMEOUT : FMM_OK;
}

fmm_status fmm_set_wait_limit(uint64_t ns) {
    if (ns == 0) return FMM_ERR_ARG;
    set_wait_limit_ns(ns);
    return FMM_OK;
}

fmm_status fmm_selftest_wait_timeout(int kernel, uint64_t ns, void *stream) {
    if ((kernel != 0 && kernel != 1) || ns == 0) return FMM_ERR_ARG;
    const cudaError_t e = kernel == 0 ? residue_gemm_timeout_probe(ns, (cudaStream_t)stream)
                                      : tf32_gemm_timeout_probe(ns, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? FMM_ERR_NO_MEMORY : FMM_ERR_CUDA;
    }
    return fmm_check_device_error();
}

fmm_status fmm_plan_info(fmm_plan_t p, fmm_plan_info_t *info) {
    if (!p || !info) return FMM_ERR_ARG;
    info->M = p->M; info->K = p->K; info->N = p->N; info->R = p->R; info->levels = p->L;
    info->flags = p->flags;
    info->leaves = p->leaves;
    info->nnz_a_terms = (int64_t)p->a.row.size();
    info->nnz_b_terms = (int64_t)p->b.row.size();
    info->nnz_c_terms = (int64_t)p->c.row.size();
    info->max_a_terms = p->a.max_terms();
    info->max_b_terms = p->b.max_terms();
    info->max_c_terms = p->c.max_terms();
    return FMM_OK;
}

fmm_status fmm_plan_leaf_terms(fmm_plan_t p, int which, int64_t *ptr, int32_t *row, int32_t *col,
                               double *coef, int64_t capacity) {
    if (!p || which < 0 || which > 2) return FMM_ERR_ARG;
    const TermList &t = which == 0 ? p->a : (which == 1 ? p->b : p->c);
    const int64_t n = (int64_t)t.row.size();
    if ((row || col || coef) && capacity < n) return FMM_ERR_ARG;
    if (ptr) std::memcpy(ptr, t.ptr.data(), t.ptr.size() * sizeof(int64_t));
    if (row) std::memcpy(row, t.row.data(), n * sizeof(int32_t));
    if (col) std::memcpy(col, t.col.data(), n * sizeof(int32_t));
    if (coef) std::memcpy(coef, t.coef.data(), n * sizeof(double));
    return FMM_OK;
}

fmm_status fmm_workspace_size(fmm_plan_t p, int64_t m, int64_t k, int64_t n, size_t *bytes) {
    if (!p || !bytes || m < 1 || k < 1 || n < 1) return FMM_ERR_ARG;
    *bytes = ws_layout(p, geometry(p, m, k, n)).total;
    return FMM_OK;
}

fmm_status fmm_gemm(fmm_plan_t p, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *C, int64_t ldc, int64_t m, int64_t k, int64_t n, void *ws,
                    size_t ws_bytes, void *stream) {
    t_launches = 0;
    if (!p) return FMM_ERR_ARG;
    fmm_status st = check_operands(A, lda, B, ldb, C, ldc, m, k, n);
    if (st != FMM_OK) return st;
    int launches = 0;
    st = run_gemm(p, A, lda, B, ldb, C, ldc, m, k, n, ws, ws_bytes, (cudaStream_t)stream,
                  &launches);
    t_launches = launches;
    return st;
}

fmm_status fmm_gemm_grouped(int64_t count, const fmm_plan_t *plans, const double *const *A, const int64_t *lda,
                            const double *const *B, const int64_t *ldb, double *const *C, const int64_t *ldc,
                            const int64_t *m, const int64_t *k, const int64_t *n, void *const *ws,
                            const size_t *ws_bytes, void *stream) {
    t_launches = 0;
    if (count < 1 || count > 4096 || !plans || !A || !lda || !B || !ldb || !C || !ldc || !m || !k || !n ||
        !ws_bytes || !ws)
        return FMM_ERR_ARG;
    std::vector<int> grouped;
    for (int64_t i = 0; i < count; ++i) {
        fmm_plan *p = plans[i];
        if (!p) return FMM_ERR_ARG;
        fmm_status st = check_operands(A[i], lda[i], B[i], ldb[i], C[i], ldc[i], m[i], k[i], n[i]);
        if (st != FMM_OK) return st;
        const Geometry g = geometry(p, m[i], k[i], n[i]);
        const size_t need = ws_layout(p, g).total;
        if (need > 0 && (!ws[i] || ws_bytes[i] < need)) return FMM_ERR_NO_MEMORY;
        if (need > 0 && ((uintptr_t)ws[i] & 255)) return FMM_ERR_ARG;
        // the GEMMs of emulated residue-space products (at most one recursive
        // level) are grouped; everything else runs as fmm_gemm would
        if (p->prec == FMM_PREC_OZAKI_BF16 && p->L <= 1 && (p->L == 0 || (g.fast && residue_space(p))) &&
            g.kL <= 65536 && !(p->flags & FMM_FLAG_TC_FUSED_S))
            grouped.push_back(int(i));
    }
    for (int64_t i = 0; i < count; ++i)
        for (int64_t j = 0; j < count; ++j) {
            if (j == i) continue;
            const size_t ci = span(m[i], n[i], ldc[i]);
            if (overlaps(C[i], ci, C[j], span(m[j], n[j], ldc[j])) ||
                overlaps(C[i], ci, A[j], span(m[j], k[j], lda[j])) ||
                overlaps(C[i], ci, B[j], span(k[j], n[j], ldb[j])))
                return FMM_ERR_ARG;
        }
    cudaStream_t s = (cudaStream_t)stream;
    int launches = 0;
    std::vector<char> is_grouped(count, 0);
    for (int i : grouped) is_grouped[i] = 1;
    for (int64_t i = 0; i < count; ++i) {
        if (is_grouped[i]) continue;
        const fmm_status st = run_gemm(plans[i], A[i], lda[i], B[i], ldb[i], C[i], ldc[i], m[i], k[i], n[i], ws[i],
                                       ws_bytes[i], s, &launches);
        if (st != FMM_OK) return st;
    }
    int *err = nullptr;
    if (!grouped.empty() && device_error_flag(&err) != cudaSuccess) return FMM_ERR_CUDA;
    for (size_t c0 = 0; c0 < grouped.size(); c0 += RG_MAX_PROBLEMS) {
        const size_t c1 = std::min(grouped.size(), c0 + RG_MAX_PROBLEMS);
        std::vector<GemmDefer> d(c1 - c0);
        bool narrow = false;
        for (size_t t = c0; t < c1; ++t) {
            const int i = grouped[t];
            d[t - c0].phase = 0;
            const fmm_status st = run_gemm(plans[i], A[i], lda[i], B[i], ldb[i], C[i], ldc[i], m[i], k[i], n[i],
                                           ws[i], ws_bytes[i], s, &launches, nullptr, &d[t - c0]);
            if (st != FMM_OK) return st;
            narrow = narrow || d[t - c0].narrow;
        }
        std::vector<RgDesc> gd;
        for (auto &x : d) gd.push_back(x.gemm);
        cudaError_t e = launch_residue_gemm_group(gd.data(), int(gd.size()), err, s, &launches, narrow);
        if (e != cudaSuccess) return cuda_status(e);
        for (size_t t = c0; t < c1; ++t) {
            const int i = grouped[t];
            d[t - c0].phase = 1;
            const fmm_status st = run_gemm(plans[i], A[i], lda[i], B[i], ldb[i], C[i], ldc[i], m[i], k[i], n[i],
                                           ws[i], ws_bytes[i], s, &launches, nullptr, &d[t - c0]);
            if (st != FMM_OK) return st;
        }
    }
    t_launches = launches;
    return FMM_OK;
}

fmm_status fmm_workspace_size_batched(fmm_plan_t p, int64_t count, int64_t m, int64_t k,
                                      int64_t n, size_t *bytes) {
    if (!p || !bytes || count < 1 || m < 1 || k < 1 || n < 1) return FMM_ERR_ARG;
    *bytes = align256(size_t(count) * 3 * sizeof(void *));
    return FMM_OK;
}

fmm_status fmm_gemm_batched(fmm_plan_t p, int64_t count, const double *const *A, int64_t lda,
                            const double *const *B, int64_t ldb, double *const *C, int64_t ldc,
                            int64_t m, int64_t k, int64_t n, void *ws, size_t ws_bytes,
                            void *stream) {
    t_launches = 0;
    if (!p || !A || !B || !C || count < 1 || count > 65535) return FMM_ERR_ARG;
    if (p->prec != FMM_PREC_FP64) return FMM_ERR_UNSUPPORTED;
    for (int64_t b = 0; b < count; ++b) {
        fmm_status st = check_operands(A[b], lda, B[b], ldb, C[b], ldc, m, k, n);
        if (st != FMM_OK) return st;
        for (int64_t o = 0; o < count; ++o)
            if (overlaps(C[b], span(m, n, ldc), A[o], span(m, k, lda)) ||
                overlaps(C[b], span(m, n, ldc), B[o], span(k, n, ldb)))
                return FMM_ERR_ARG;
    }
    const size_t need = align256(size_t(count) * 3 * sizeof(void *));
    if (!ws || ws_bytes < need) return FMM_ERR_NO_MEMORY;
    if ((uintptr_t)ws & 255) return FMM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int launches = 0;
    cudaError_t e;
    const Geometry g = geometry(p, m, k, n);
    if (!g.fast) {
        for (int64_t b = 0; b < count; ++b)
            if ((e = launch_classical(A[b], lda, B[b], ldb, C[b], ldc, m, k, n, FMM_TILE_AUTO, s,
                                      &launches)) != cudaSuccess) {
                t_launches = launches;
                return cuda_status(e);
            }
        t_launches = launches;
        return FMM_OK;
    }
    {
        const fmm_status us = ensure_uploaded(p);
        if (us != FMM_OK) return us;
    }
    // pointer arrays to the device (pageable source: copied before return)
    std::vector<const void *> host(size_t(count) * 3);
    for (int64_t b = 0; b < count; ++b) {
        host[b] = A[b];
        host[count + b] = B[b];
        host[2 * count + b] = C[b];
    }
    if ((e = cudaMemcpyAsync(ws, host.data(), host.size() * sizeof(void *), cudaMemcpyHostToDevice,
                             s)) != cudaSuccess)
        return cuda_status(e);
    const bool kfringe = g.kp < k;
    for (int64_t b = 0; b < count; ++b) {
        if (kfringe)
            e = launch_classical(A[b] + g.kp, lda, B[b] + g.kp * ldb, ldb, C[b], ldc, g.mp, k - g.kp,
                                 g.np, FMM_TILE_AUTO, s, &launches);
        else
            e = cudaMemset2DAsync(C[b], ldc * 8, 0, g.np * 8, g.mp, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    LeafLaunch L{};
    L.lda = lda; L.ldb = ldb; L.ldc = ldc;
    L.mL = g.mL; L.kL = g.kL; L.nL = g.nL; L.leaves = p->leaves;
    L.a_ptr = p->dev.a_ptr; L.a_code = p->dev.a_code; L.a_coef = p->dev.a_coef;
    L.b_ptr = p->dev.b_ptr; L.b_code = p->dev.b_code; L.b_coef = p->dev.b_coef;
    L.c_ptr = p->dev.c_ptr; L.c_code = p->dev.c_code; L.c_coef = p->dev.c_coef;
    L.epi = EPI_ATOMIC;
    L.Ab = (const double *const *)ws;
    L.Bb = (const double *const *)ws + count;
    L.Cb = (double *const *)ws + 2 * count;
    L.batch = count;
    const double extra_a = double(p->a.row.size()) / double(p->leaves) - 1.0;
    const double extra_b = double(p->b.row.size()) / double(p->leaves) - 1.0;
    L.tile = resolve_tile(p->tile, g.mL, g.nL, g.kL, p->leaves * count, extra_a, extra_b,
                          device_sms());
    if ((e = timed(s, [&] { return launch_leaf_gemm(L, s, &launches); })) != cudaSuccess)
        return cuda_status(e);
    for (int64_t b = 0; b < count; ++b) {
        if (g.mp < m &&
            (e = launch_classical(A[b] + g.mp * lda, lda, B[b], ldb, C[b] + g.mp * ldc, ldc, m - g.mp,
                                  k, n, FMM_TILE_AUTO, s, &launches)) != cudaSuccess)
            return cuda_status(e);
        if (g.np < n &&
            (e = launch_classical(A[b], lda, B[b] + g.np, ldb, C[b] + g.np, ldc, g.mp, k, n - g.np,
                                  FMM_TILE_AUTO, s, &launches)) != cudaSuccess)
            return cuda_status(e);
    }
    t_launches = launches;
    return FMM_OK;
}

fmm_status fmm_classical_gemm(const double *A, int64_t lda, const double *B, int64_t ldb,
                              double *C, int64_t ldc, int64_t m, int64_t k, int64_t n,
                              void *stream) {
    t_launches = 0;
    fmm_status st = check_operands(A, lda, B, ldb, C, ldc, m, k, n);
    if (st != FMM_OK) return st;
    int launches = 0;
    cudaStream_t s = (cudaStream_t)stream;
    st = cuda_status(timed(s, [&] {
        return launch_classical(A, lda, B, ldb, C, ldc, m, k, n, FMM_TILE_AUTO, s, &launches);
    }));
    t_launches = launches;
    return st;
}

fmm_status fmm_timing_enable(int on) {
    t_timing.on = on != 0;
    t_timing.used = 0;
    return FMM_OK;
}

fmm_status fmm_timing_leaf_ms(double *total_ms, int *count) {
    if (!total_ms || !count) return FMM_ERR_ARG;
    double tot = 0.0;
    int n = 0;
    for (int i = 0; i + 1 < t_timing.used; i += 2) {
        if (cudaEventSynchronize(t_timing.ev[i + 1]) != cudaSuccess) return FMM_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t_timing.ev[i], t_timing.ev[i + 1]) != cudaSuccess)
            return FMM_ERR_CUDA;
        tot += ms;
        ++n;
    }
    t_timing.used = 0;
    *total_ms = tot;
    *count = n;
    return FMM_OK;
}

fmm_status fmm_host_workspace_size(fmm_plan_t p, int64_t m, int64_t k, int64_t n, size_t *bytes) {
    if (!bytes || m < 1 || k < 1 || n < 1) return FMM_ERR_ARG;
    size_t ws = 0;
    if (p) ws = ws_layout(p, geometry(p, m, k, n)).total;
    *bytes = align256(size_t(m * k * 8)) + align256(size_t(k * n * 8)) +
             align256(size_t(m * n * 8)) + ws;
    return FMM_OK;
}

fmm_status fmm_set_host_pipeline(int bands, int gemm_bands) {
    if (bands < 0 || bands > 64 || gemm_bands < 0 || gemm_bands > 64) return FMM_ERR_ARG;
    t_bands = bands;
    t_gemm_bands = gemm_bands;
    return FMM_OK;
}

fmm_status fmm_gemm_host(fmm_plan_t p, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, int64_t m, int64_t k, int64_t n,
                         void *dev_ws, size_t ws_bytes, void *stream) {
    t_launches = 0;
    if (!A || !B || !C || !dev_ws) return FMM_ERR_ARG;
    if (m < 1 || k < 1 || n < 1 || lda < k || ldb < n || ldc < n) return FMM_ERR_ARG;
    if ((uintptr_t)dev_ws & 255) return FMM_ERR_ARG;
    size_t need = 0;
    fmm_host_workspace_size(p, m, k, n, &need);
    if (ws_bytes < need) return FMM_ERR_NO_MEMORY;
    HostSide *hs = host_side();
    if (!hs) return FMM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)dev_ws;
    double *dA = (double *)w;
    double *dB = (double *)(w + align256(size_t(m * k * 8)));
    double *dC = (double *)((char *)dB + align256(size_t(k * n * 8)));
    char *rest = (char *)dC + align256(size_t(m * n * 8));
    // All copies in on the side stream (one after the other: they would only
    // share the link), once the caller's earlier work on `stream` is done
    // with the buffers: B first, then A in bands of first-level child rows,
    // each with an event, so that the kernels reading B run while A arrives
    // and each band of A is formed as soon as it is in.
    cudaError_t e;
    auto fail = [&](fmm_status st) {
        cudaStreamSynchronize(hs->side);   // no copy into the caller's buffers left in flight
        cudaStreamSynchronize(s);
        return st;
    };
    const int gM = (p && p->L > 0) ? p->M : 1;
    const int64_t ml1 = m / gM;   // rows of a first-level block (banding is used only without a fringe)
    const int a_bands = (int)std::max<int64_t>(1, std::min<int64_t>({4, ml1, m * k * 8 / (64 << 20)}));
    if ((e = cudaEventRecord(hs->start, s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(hs->side, hs->start, 0)) != cudaSuccess ||
        (e = copy_rows(dB, n, B, ldb, k, n, cudaMemcpyHostToDevice, hs->side)) != cudaSuccess ||
        (e = cudaEventRecord(hs->b_in, hs->side)) != cudaSuccess)
        return fail(cuda_status(e));
    for (int j = 0; j < a_bands; ++j) {
        // rows [r0, r1) of every block row; the last band also takes rows
        // past gM ml1 (none when the path bands A)
        const int64_t r0 = ml1 * j / a_bands, r1 = ml1 * (j + 1) / a_bands;
        for (int a = 0; a < gM; ++a) {
            const int64_t row = a * ml1 + r0;
            if ((e = copy_rows(dA + row * k, k, A + row * lda, lda, r1 - r0, k, cudaMemcpyHostToDevice,
                               hs->side)) != cudaSuccess)
                return fail(cuda_status(e));
        }
        if (j == a_bands - 1 && gM * ml1 < m &&
            (e = copy_rows(dA + gM * ml1 * k, k, A + gM * ml1 * lda, lda, m - gM * ml1, k,
                           cudaMemcpyHostToDevice, hs->side)) != cudaSuccess)
            return fail(cuda_status(e));
        if ((e = cudaEventRecord(hs->a_in[j], hs->side)) != cudaSuccess) return fail(cuda_status(e));
    }
    // C leaves in row bands, each copied on the side stream as soon as the
    // last pass has written it (when the path runs in bands at all)
    BandCopy bc{s, hs->side, hs->band, C, ldc, dC, n, 0};
    const int bands = host_bands(m, n);
    HostPipe pipe{hs->b_in, a_bands, hs->a_in, bands, host_gemm_bands(bands), copy_band, &bc};
    fmm_status st;
    int launches = 0;
    if (p) {
        st = run_gemm(p, dA, k, dB, n, dC, n, m, k, n, rest, ws_bytes - (rest - w), s, &launches, &pipe);
    } else {
        st = cuda_status(cudaStreamWaitEvent(s, hs->a_in[a_bands - 1], 0));
        if (st == FMM_OK)
            st = cuda_status(launch_classical(dA, k, dB, n, dC, n, m, k, n, FMM_TILE_AUTO, s, &launches));
    }
    t_launches = launches;
    if (st != FMM_OK) return fail(st);
    if (bc.rows_done == m) {
        if ((e = cudaEventRecord(hs->side_done, hs->side)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, hs->side_done, 0)) != cudaSuccess)
            return fail(cuda_status(e));
    } else if (bc.rows_done != 0) {
        return fail(FMM_ERR_CUDA);
    } else if ((e = copy_rows(C, ldc, dC, n, m, n, cudaMemcpyDeviceToHost, s)) != cudaSuccess) {
        return fail(cuda_status(e));
    }
    return cuda_status(cudaStreamSynchronize(s));
}

}  // extern "C"
