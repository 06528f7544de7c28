// FP64 kernels of the fast-multiplication hot path on sm_103a.
//
//   leaf_gemm      grouped GEMM over all R^L leaf products M_r = S_r T_r
//                  (Section 3.1; one launch for every leaf, the GPU analogue
//                  of running all leaves of the recursion tree as tasks,
//                  Section 4.2).  Operand staging forms S_r and T_r from the
//                  A and B blocks while filling shared memory (the write-once
//                  chains of Section 3.2 moved on chip); the epilogue applies
//                  the W coefficients.
//   form_slots     write-once formation of S_r / T_r into workspace
//                  (Section 3.2, "write-once"), for the unfused scheme.
//   w_pass         write-once formation of the C blocks from stored M_r.
//
// The FP64 pipe of GB300 retires 2 DFMA per SM per clock, so the leaf GEMM
// is bound by FP64 issue, not by memory: the tile is sized so that each warp
// has 16-64 independent FMAs per shared-memory fragment, and shared-memory
// layouts are chosen to keep fragment reads broadcast or conflict-free.
#include <cuda_runtime.h>

#include <algorithm>

#include <cstdint>

#include "fmm_internal.h"

namespace fmm {

namespace {

constexpr int BK = 16;        // k-depth of one shared-memory stage
constexpr int THREADS = 256;  // 16 x 16 threads

struct KParams {
    const double *A; int64_t lda;
    const double *B; int64_t ldb;
    double *C; int64_t ldc;
    int64_t mL, kL, nL;
    const int *a_ptr; const int *a_code; const double *a_coef;
    const int *b_ptr; const int *b_code; const double *b_coef;
    const int *c_ptr; const int *c_code; const double *c_coef;
    const double *slotA; int64_t slotA_stride;
    const double *slotB; int64_t slotB_stride;
    double *wsM;
    int epi;
    int tiles_n;
    int64_t leaf_base;
    // batched products: per blockIdx.z operand bases (device arrays) or null
    const double *const *Ab; const double *const *Bb; double *const *Cb;
};

// Base address and leading dimension of one operand term.
__device__ __forceinline__ const double *term_base(int code, const double *X, int64_t ld,
                                                    int64_t brows, int64_t bcols,
                                                    const double *slot, int64_t slot_stride,
                                                    int64_t slot_ld, int64_t *ld_out) {
    if (code >= 0) {
        *ld_out = ld;
        return X + (int64_t)(code >> 16) * brows * ld + (int64_t)(code & 0xffff) * bcols;
    }
    *ld_out = slot_ld;
    return slot + (int64_t)(-code - 1) * slot_stride;
}

// Coefficient tests on the integer pipe: on this GPU the FP64 pipe retires
// 1/64 of the FP32 rate, and an FP64 compare per term and element costs as
// much as the addition itself.
__device__ __forceinline__ bool is_one(double c) { return __double_as_longlong(c) == 0x3FF0000000000000ll; }
__device__ __forceinline__ bool is_minus_one(double c) {
    return __double_as_longlong(c) == (long long)0xBFF0000000000000ull;
}
__device__ __forceinline__ bool is_zero(double c) { return (__double_as_longlong(c) << 1) == 0; }

// Add coef * x into v with one FP64 operation whatever the coefficient: for
// c = +-1, fma(c, x, v) rounds v +- x once, the same bits as the addition,
// and avoids a data-dependent choice between several FP64 results.
__device__ __forceinline__ double chain_step(double v, double c, double x) { return fma(c, x, v); }

// The first term of a chain: c x (exact for c = +-1, and for powers of two).
__device__ __forceinline__ double chain_first(double c, double x) { return c * x; }

template <int TM, int TN>
__global__ void __launch_bounds__(THREADS, 1) leaf_gemm(const KParams p) {
    constexpr int BM = 16 * TM, BN = 16 * TN;
    constexpr int EA = BM * BK / THREADS;   // A elements staged per thread
    constexpr int EB = BK * BN / THREADS;   // B elements staged per thread
    constexpr int LDA_S = BM + 1;           // padded: transposed stores
    extern __shared__ double smem[];
    double *As = smem;                      // [2][BK][LDA_S]
    double *Bs = smem + 2 * BK * LDA_S;     // [2][BK][BN]

    const int64_t leaf = p.leaf_base + blockIdx.y;
    const int tm = blockIdx.x / p.tiles_n, tn = blockIdx.x % p.tiles_n;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)tm * BM, col0 = (int64_t)tn * BN;
    const double *opA = p.Ab ? p.Ab[blockIdx.z] : p.A;
    const double *opB = p.Bb ? p.Bb[blockIdx.z] : p.B;
    double *opC = p.Cb ? p.Cb[blockIdx.z] : p.C;

    const int a0 = p.a_ptr[leaf], a1 = p.a_ptr[leaf + 1];
    const int b0 = p.b_ptr[leaf], b1 = p.b_ptr[leaf + 1];

    double acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

    double ra[EA], rb[EB];

    // Stage k-chunk k0: S_r and T_r entries combined from all their terms.
    auto gather = [&](int64_t k0) {
#pragma unroll
        for (int e = 0; e < EA; ++e) ra[e] = 0.0;
#pragma unroll
        for (int e = 0; e < EB; ++e) rb[e] = 0.0;
        for (int t = a0; t < a1; ++t) {
            int64_t ld;
            const double *X = term_base(p.a_code[t], opA, p.lda, p.mL, p.kL, p.slotA,
                                        p.slotA_stride, p.kL, &ld);
            const double c = p.a_coef[t];
#pragma unroll
            for (int e = 0; e < EA; ++e) {
                const int idx = tid + THREADS * e;
                const int r = idx / BK, kk = idx % BK;
                const int64_t gr = row0 + r, gk = k0 + kk;
                double x = 0.0;
                if (gr < p.mL && gk < p.kL) x = __ldg(X + gr * ld + gk);
                ra[e] = (t == a0) ? chain_first(c, x) : chain_step(ra[e], c, x);
            }
        }
        for (int t = b0; t < b1; ++t) {
            int64_t ld;
            const double *X = term_base(p.b_code[t], opB, p.ldb, p.kL, p.nL, p.slotB,
                                        p.slotB_stride, p.nL, &ld);
            const double c = p.b_coef[t];
#pragma unroll
            for (int e = 0; e < EB; ++e) {
                const int idx = tid + THREADS * e;
                const int kk = idx / BN, cc = idx % BN;
                const int64_t gk = k0 + kk, gc = col0 + cc;
                double x = 0.0;
                if (gk < p.kL && gc < p.nL) x = __ldg(X + gk * ld + gc);
                rb[e] = (t == b0) ? chain_first(c, x) : chain_step(rb[e], c, x);
            }
        }
    };
    auto stash = [&](int buf) {
        double *as = As + buf * BK * LDA_S;
        double *bs = Bs + buf * BK * BN;
#pragma unroll
        for (int e = 0; e < EA; ++e) {
            const int idx = tid + THREADS * e;
            as[(idx % BK) * LDA_S + idx / BK] = ra[e];
        }
#pragma unroll
        for (int e = 0; e < EB; ++e) {
            const int idx = tid + THREADS * e;
            bs[(idx / BN) * BN + idx % BN] = rb[e];
        }
    };

    gather(0);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = 0; k0 < p.kL; k0 += BK) {
        const bool more = k0 + BK < p.kL;
        if (more) gather(k0 + BK);
        const double *as = As + buf * BK * LDA_S;
        const double *bs = Bs + buf * BK * BN;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = as[kk * LDA_S + ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = bs[kk * BN + tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (more) stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }

    // Epilogue: the W coefficients of this leaf (Section 3.1, C_q = sum W_qr M_r).
    if (p.epi == EPI_WORKSPACE) {
        double *out = p.wsM + leaf * p.mL * p.nL;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t gr = row0 + ty + 16 * i;
            if (gr >= p.mL) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t gc = col0 + tx + 16 * j;
                if (gc < p.nL) out[gr * p.nL + gc] = acc[i][j];
            }
        }
        return;
    }
    const int c0 = p.c_ptr[leaf], c1 = p.c_ptr[leaf + 1];
    for (int t = c0; t < c1; ++t) {
        const int code = p.c_code[t];
        const double w = p.c_coef[t];
        if (is_zero(w)) continue;
        double *Cb = opC + (int64_t)(code >> 16) * p.mL * p.ldc + (int64_t)(code & 0xffff) * p.nL;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t gr = row0 + ty + 16 * i;
            if (gr >= p.mL) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t gc = col0 + tx + 16 * j;
                if (gc >= p.nL) continue;
                const double v = is_one(w) ? acc[i][j] : (is_minus_one(w) ? -acc[i][j] : w * acc[i][j]);
                if (p.epi == EPI_ATOMIC)
                    atomicAdd(Cb + gr * p.ldc + gc, v);
                else
                    Cb[gr * p.ldc + gc] = v;
            }
        }
    }
}

// Warp-specialised variant: PRODUCERS gather and combine S_r / T_r chunks
// into a STAGES-deep shared-memory ring while CONSUMERS run the DFMA loop, so
// the load latency of multi-term chains never idles the FP64 pipe.  Stage
// hand-off uses hardware named barriers (FULL: producers arrive, consumers
// wait; EMPTY: consumers arrive, producers wait); every thread takes part in
// the same number of phases, so each barrier completes.
constexpr int WS_CONSUMERS = 256;
constexpr int WS_PRODUCERS = 128;
constexpr int WS_THREADS = WS_CONSUMERS + WS_PRODUCERS;
constexpr int WS_STAGES = 4;

__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <int TM, int TN>
__global__ void __launch_bounds__(WS_THREADS, 1) leaf_gemm_ws(const KParams p) {
    constexpr int BM = 16 * TM, BN = 16 * TN;
    constexpr int LDA_S = BM + 1;
    constexpr int STAGE = BK * LDA_S + BK * BN;      // doubles per stage
    constexpr int PA = BM * BK / WS_PRODUCERS;       // A elements per producer thread
    constexpr int PB = BK * BN / WS_PRODUCERS;       // B elements per producer thread
    extern __shared__ double smem[];

    const int64_t leaf = p.leaf_base + blockIdx.y;
    const int tm = blockIdx.x / p.tiles_n, tn = blockIdx.x % p.tiles_n;
    const int64_t row0 = (int64_t)tm * BM, col0 = (int64_t)tn * BN;
    const int64_t nchunks = (p.kL + BK - 1) / BK;
    const int tid = threadIdx.x;
    const double *opA = p.Ab ? p.Ab[blockIdx.z] : p.A;
    const double *opB = p.Bb ? p.Bb[blockIdx.z] : p.B;
    double *opC = p.Cb ? p.Cb[blockIdx.z] : p.C;

    if (tid >= WS_CONSUMERS) {
        // ---------------- producers ----------------
        const int pt = tid - WS_CONSUMERS;
        const int a0 = p.a_ptr[leaf], a1 = p.a_ptr[leaf + 1];
        const int b0 = p.b_ptr[leaf], b1 = p.b_ptr[leaf + 1];
        // elements gathered per batch (bounded registers)
        constexpr int PBATCH = (PA % 8 == 0 && PB % 8 == 0) ? 8 : 4;
        static_assert(PA % PBATCH == 0 && PB % PBATCH == 0, "producer batching");
        for (int64_t c = 0; c < nchunks; ++c) {
            const int st = int(c % WS_STAGES);
            const int64_t k0 = c * BK;
            if (c >= WS_STAGES) named_sync(1 + WS_STAGES + st, WS_THREADS);   // EMPTY[st]
            double *as = smem + st * STAGE;
            double *bs = as + BK * LDA_S;
            for (int eb = 0; eb < PA; eb += PBATCH) {
                double v[PBATCH];
#pragma unroll 2
                for (int t = a0; t < a1; ++t) {
                    int64_t ld;
                    const double *X = term_base(p.a_code[t], opA, p.lda, p.mL, p.kL, p.slotA,
                                                p.slotA_stride, p.kL, &ld);
                    const double cf = p.a_coef[t];
                    double x[PBATCH];
#pragma unroll
                    for (int e = 0; e < PBATCH; ++e) {
                        const int idx = pt + WS_PRODUCERS * (eb + e);
                        const int64_t gr = row0 + idx / BK, gk = k0 + idx % BK;
                        x[e] = (gr < p.mL && gk < p.kL) ? __ldg(X + gr * ld + gk) : 0.0;
                    }
#pragma unroll
                    for (int e = 0; e < PBATCH; ++e)
                        v[e] = (t == a0) ? chain_first(cf, x[e]) : chain_step(v[e], cf, x[e]);
                }
                if (a0 == a1) {
#pragma unroll
                    for (int e = 0; e < PBATCH; ++e) v[e] = 0.0;
                }
#pragma unroll
                for (int e = 0; e < PBATCH; ++e) {
                    const int idx = pt + WS_PRODUCERS * (eb + e);
                    as[(idx % BK) * LDA_S + idx / BK] = v[e];
                }
            }
            for (int eb = 0; eb < PB; eb += PBATCH) {
                double v[PBATCH];
#pragma unroll 2
                for (int t = b0; t < b1; ++t) {
                    int64_t ld;
                    const double *X = term_base(p.b_code[t], opB, p.ldb, p.kL, p.nL, p.slotB,
                                                p.slotB_stride, p.nL, &ld);
                    const double cf = p.b_coef[t];
                    double x[PBATCH];
#pragma unroll
                    for (int e = 0; e < PBATCH; ++e) {
                        const int idx = pt + WS_PRODUCERS * (eb + e);
                        const int64_t gk = k0 + idx / BN, gc = col0 + idx % BN;
                        x[e] = (gk < p.kL && gc < p.nL) ? __ldg(X + gk * ld + gc) : 0.0;
                    }
#pragma unroll
                    for (int e = 0; e < PBATCH; ++e)
                        v[e] = (t == b0) ? chain_first(cf, x[e]) : chain_step(v[e], cf, x[e]);
                }
                if (b0 == b1) {
#pragma unroll
                    for (int e = 0; e < PBATCH; ++e) v[e] = 0.0;
                }
#pragma unroll
                for (int e = 0; e < PBATCH; ++e) {
                    const int idx = pt + WS_PRODUCERS * (eb + e);
                    bs[(idx / BN) * BN + idx % BN] = v[e];
                }
            }
            __threadfence_block();
            named_arrive(1 + st, WS_THREADS);                                  // FULL[st]
        }
        return;
    }

    // ---------------- consumers ----------------
    const int tx = tid & 15, ty = tid >> 4;
    double acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int st = int(c % WS_STAGES);
        named_sync(1 + st, WS_THREADS);                                        // FULL[st]
        const double *as = smem + st * STAGE + ty;
        const double *bs = smem + st * STAGE + BK * LDA_S + tx;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[TM];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = as[kk * LDA_S + 16 * i];
            // B fragment in halves keeps the live register set small
#pragma unroll
            for (int jh = 0; jh < TN; jh += TN / 2) {
                double b[TN / 2];
#pragma unroll
                for (int j = 0; j < TN / 2; ++j) b[j] = bs[kk * BN + 16 * (jh + j)];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN / 2; ++j)
                        acc[i][jh + j] = fma(a[i], b[j], acc[i][jh + j]);
            }
        }
        if (c + WS_STAGES < nchunks) named_arrive(1 + WS_STAGES + st, WS_THREADS);  // EMPTY[st]
    }

    if (p.epi == EPI_WORKSPACE) {
        double *out = p.wsM + leaf * p.mL * p.nL;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t gr = row0 + ty + 16 * i;
            if (gr >= p.mL) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t gc = col0 + tx + 16 * j;
                if (gc < p.nL) out[gr * p.nL + gc] = acc[i][j];
            }
        }
        return;
    }
    const int c0 = p.c_ptr[leaf], c1 = p.c_ptr[leaf + 1];
    for (int t = c0; t < c1; ++t) {
        const int code = p.c_code[t];
        const double w = p.c_coef[t];
        if (is_zero(w)) continue;
        double *Cb = opC + (int64_t)(code >> 16) * p.mL * p.ldc + (int64_t)(code & 0xffff) * p.nL;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t gr = row0 + ty + 16 * i;
            if (gr >= p.mL) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t gc = col0 + tx + 16 * j;
                if (gc >= p.nL) continue;
                const double v = is_one(w) ? acc[i][j] : (is_minus_one(w) ? -acc[i][j] : w * acc[i][j]);
                if (p.epi == EPI_ATOMIC)
                    atomicAdd(Cb + gr * p.ldc + gc, v);
                else
                    Cb[gr * p.ldc + gc] = v;
            }
        }
    }
}

// S_r (or T_r) = sum_t coef_t X_t for every slot, written once.
__global__ void form_slots_kernel(const double *X, int64_t ldx, int64_t rows, int64_t cols,
                                  int64_t slot_base, const int *slot_leaf, const int *ptr,
                                  const int *code, const double *coef, double *out,
                                  int64_t out_stride) {
    const int64_t s = slot_base + blockIdx.y;
    const int leaf = slot_leaf[s];
    const int t0 = ptr[leaf], t1 = ptr[leaf + 1];
    double *o = out + s * out_stride;
    for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
        for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) {
            double v = 0.0;
            for (int t = t0; t < t1; ++t) {
                const int cd = code[t];
                const double *Xt = X + (int64_t)(cd >> 16) * rows * ldx + (int64_t)(cd & 0xffff) * cols;
                const double x = __ldg(Xt + i * ldx + j);
                v = (t == t0) ? chain_first(coef[t], x) : chain_step(v, coef[t], x);
            }
            o[i * cols + j] = v;
        }
    }
}

// C block q = (C block q if accumulate) + sum over its leaves of w * M_leaf.
__global__ void w_pass_kernel(double *C, int64_t ldc, int64_t mL, int64_t nL, int gridN,
                              int64_t q_base, const int *cq_ptr, const int *cq_leaf,
                              const double *cq_coef, const double *wsM, int accumulate) {
    const int64_t q = q_base + blockIdx.y;
    const int64_t brow = q / gridN, bcol = q % gridN;
    const int t0 = cq_ptr[q], t1 = cq_ptr[q + 1];
    double *Cb = C + brow * mL * ldc + bcol * nL;
    for (int64_t i = blockIdx.x; i < mL; i += gridDim.x) {
        for (int64_t j = threadIdx.x; j < nL; j += blockDim.x) {
            double v = accumulate ? Cb[i * ldc + j] : 0.0;
            for (int t = t0; t < t1; ++t) {
                const double w = cq_coef[t];
                if (is_zero(w)) continue;
                const double x = __ldg(wsM + (int64_t)cq_leaf[t] * mL * nL + i * nL + j);
                v = chain_step(v, w, x);
            }
            Cb[i * ldc + j] = v;
        }
    }
}

// One recursive level of S (or T) formation, write-once: output o = s*R + r
// is sum_i U_ir (parent s)_i, where block i = (a, b) of parent s starts at
// row a*rows, column b*cols.  Parents are A itself (level 1) or the previous
// level's outputs, stored contiguously with leading dimension cols*K.
__global__ void level_form_kernel(const double *parent, int64_t pld, int64_t pstride, int64_t rows,
                                  int64_t cols, int R, int64_t o_base, const int *ptr,
                                  const int *code, const double *coef, double *out) {
    const int64_t o = o_base + blockIdx.y;
    const int64_t s = o / R;
    const int r = int(o % R);
    const double *P = parent + s * pstride;
    const int t0 = ptr[r], t1 = ptr[r + 1];
    double *O = out + o * rows * cols;
    for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
        for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) {
            double v = 0.0;
            for (int t = t0; t < t1; ++t) {
                const int cd = code[t];
                const double x = __ldg(P + ((int64_t)(cd >> 16) * rows + i) * pld +
                                       (int64_t)(cd & 0xffff) * cols + j);
                v = (t == t0) ? chain_first(coef[t], x) : chain_step(v, coef[t], x);
            }
            O[i * cols + j] = v;
        }
    }
}

// One recursive level of the W combination: parent s, block q = (a, c) of
// its M x N grid = (its old value if accumulate) + sum_r W_qr child_{s*R+r}.
__global__ void level_w_kernel(const double *child, int64_t rows, int64_t cols, int R, int gridN,
                               int MN, double *parent, int64_t pld, int64_t pstride, int64_t o_base,
                               const int *w_ptr, const int *w_r, const double *w_coef,
                               int accumulate) {
    const int64_t o = o_base + blockIdx.y;
    const int64_t s = o / MN;
    const int q = int(o % MN);
    const int a = q / gridN, c = q % gridN;
    double *Pout = parent + s * pstride + (int64_t)a * rows * pld + (int64_t)c * cols;
    const int t0 = w_ptr[q], t1 = w_ptr[q + 1];
    for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
        for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) {
            double v = accumulate ? Pout[i * pld + j] : 0.0;
            bool first = !accumulate;
            for (int t = t0; t < t1; ++t) {
                const double x = __ldg(child + ((s * R + w_r[t]) * rows + i) * cols + j);
                v = first ? chain_first(w_coef[t], x) : chain_step(v, w_coef[t], x);
                first = false;
            }
            Pout[i * pld + j] = v;
        }
    }
}

// Streaming additions (Section 3.2), one recursive level of S (or T): a
// thread reads its element of all NB blocks of its parent once and writes
// that element of every child, child r = sum_t c_t block(t) in list order
// (the same operations in the same order as level_form_kernel, so the same
// bits).  parent s: (gridR rows) x (gridC cols) blocks of rows x cols, ld
// pld, parents pstride apart; children out[s*R + r] packed rows x cols.
// Dynamic shared memory: NB x 256 doubles.
__global__ void __launch_bounds__(256) level_stream_kernel(const double *parent, int64_t pld, int64_t pstride,
                                                           int64_t rows, int64_t cols, int gridC, int NB,
                                                           int R, int64_t parents, const int *ptr,
                                                           const int *code, const double *coef,
                                                           double *out) {
    extern __shared__ double sx[];
    __shared__ int sb[512];
    __shared__ double sc[512];
    __shared__ int sp[129];
    const int nt = ptr[R];
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const int cd = code[t];
        sb[t] = (cd >> 16) * gridC + (cd & 0xffff);
        sc[t] = coef[t];
    }
    for (int t = threadIdx.x; t <= R; t += blockDim.x) sp[t] = ptr[t];
    __syncthreads();
    const int64_t per = rows * cols;
    const int64_t pos = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (pos >= parents * per) return;
    const int64_t sidx = pos / per, rem = pos % per, i = rem / cols, j = rem % cols;
    const double *P = parent + sidx * pstride;
    for (int b = 0; b < NB; ++b)
        sx[b * 256 + threadIdx.x] = __ldg(P + ((int64_t)(b / gridC) * rows + i) * pld + (int64_t)(b % gridC) * cols + j);
    double *O = out + sidx * R * per + rem;
    for (int r = 0; r < R; ++r) {
        const int t0 = sp[r], t1 = sp[r + 1];
        double v = 0.0;
        for (int t = t0; t < t1; ++t) {
            const double x = sx[sb[t] * 256 + threadIdx.x];
            v = (t == t0) ? chain_first(sc[t], x) : chain_step(v, sc[t], x);
        }
        O[(int64_t)r * per] = v;
    }
}

// Streaming W combination, one level: a thread reads its element of all R
// child products of parent s once and writes that element of each of the
// MN blocks of s, block q = (old value if accumulate) + sum_t W_t child(r_t)
// in list order (as level_w_kernel).  Dynamic shared memory: R x 128 doubles.
__global__ void __launch_bounds__(128) level_w_stream_kernel(const double *child, int64_t rows, int64_t cols,
                                                             int R, int gridN, int MN, double *parent,
                                                             int64_t pld, int64_t pstride, int64_t parents,
                                                             const int *w_ptr, const int *w_r,
                                                             const double *w_coef, int accumulate) {
    extern __shared__ double sx[];
    __shared__ int sr[512];
    __shared__ double sc[512];
    __shared__ int sp[129];
    const int nt = w_ptr[MN];
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        sr[t] = w_r[t];
        sc[t] = w_coef[t];
    }
    for (int t = threadIdx.x; t <= MN; t += blockDim.x) sp[t] = w_ptr[t];
    __syncthreads();
    const int64_t per = rows * cols;
    const int64_t pos = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (pos >= parents * per) return;
    const int64_t sidx = pos / per, rem = pos % per, i = rem / cols, j = rem % cols;
    const double *X = child + sidx * R * per + rem;
    for (int r = 0; r < R; ++r) sx[r * 128 + threadIdx.x] = __ldg(X + (int64_t)r * per);
    double *Pb = parent + sidx * pstride + i * pld + j;
    for (int q = 0; q < MN; ++q) {
        double *dst = Pb + (int64_t)(q / gridN) * rows * pld + (int64_t)(q % gridN) * cols;
        double v = accumulate ? *dst : 0.0;
        bool first = !accumulate;
        for (int t = sp[q]; t < sp[q + 1]; ++t) {
            const double x = sx[sr[t] * 128 + threadIdx.x];
            v = first ? chain_first(sc[t], x) : chain_step(v, sc[t], x);
            first = false;
        }
        *dst = v;
    }
}

// Pairwise additions (Section 3.2): one pass per term, Y_s = c X_s (first)
// or Y_s + c X_s, for every parent s; X_s and Y_s are rows x cols blocks with
// their own leading dimensions and parent strides.
__global__ void __launch_bounds__(256) block_axpy_kernel(const double *X, int64_t xld, int64_t xstride, double *Y,
                                                         int64_t yld, int64_t ystride, int64_t parents,
                                                         int64_t rows, int64_t cols, double c, int first) {
    const int64_t per = rows * cols;
    for (int64_t pos = (int64_t)blockIdx.x * 256 + threadIdx.x; pos < parents * per;
         pos += (int64_t)gridDim.x * 256) {
        const int64_t sidx = pos / per, rem = pos % per, i = rem / cols, j = rem % cols;
        const double x = __ldg(X + sidx * xstride + i * xld + j);
        double *y = Y + sidx * ystride + i * yld + j;
        *y = first ? chain_first(c, x) : chain_step(*y, c, x);
    }
}

__device__ int g_unit_ptr[2] = {0, 1};
__device__ int g_unit_code[1] = {0};
__device__ double g_unit_coef[1] = {1.0};

template <int TM, int TN, bool WS>
cudaError_t configure_tile(void (**kern_out)(const KParams), size_t *smem_out) {
    constexpr int BM = 16 * TM, BN = 16 * TN;
    const size_t smem = WS ? sizeof(double) * WS_STAGES * BK * ((BM + 1) + BN)
                           : sizeof(double) * 2 * BK * ((BM + 1) + BN);
    void (*kern)(const KParams);
    if constexpr (WS)
        kern = leaf_gemm_ws<TM, TN>;
    else
        kern = leaf_gemm<TM, TN>;
    static bool configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    if (kern_out) *kern_out = kern;
    if (smem_out) *smem_out = smem;
    return cudaSuccess;
}

template <int TM, int TN, bool WS>
cudaError_t launch_tile(const KParams &base, int64_t leaves, int64_t batch, cudaStream_t s,
                        int *launches) {
    constexpr int BM = 16 * TM, BN = 16 * TN;
    void (*kern)(const KParams);
    size_t smem;
    cudaError_t ce = configure_tile<TM, TN, WS>(&kern, &smem);
    if (ce != cudaSuccess) return ce;
    const int threads = WS ? WS_THREADS : THREADS;
    KParams p = base;
    const int64_t tiles_m = (p.mL + BM - 1) / BM, tiles_n = (p.nL + BN - 1) / BN;
    if (tiles_m * tiles_n > 0x7fffffffLL) return cudaErrorInvalidValue;
    p.tiles_n = (int)tiles_n;
    for (int64_t lb = 0; lb < leaves; lb += 65535) {
        const int64_t cnt = leaves - lb < 65535 ? leaves - lb : 65535;
        p.leaf_base = lb;
        dim3 grid((unsigned)(tiles_m * tiles_n), (unsigned)cnt, (unsigned)batch);
        kern<<<grid, threads, smem, s>>>(p);
        ++*launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t prepare_fp64_kernels() {
    cudaError_t e;
    if ((e = configure_tile<8, 8, true>(nullptr, nullptr)) != cudaSuccess) return e;
    if ((e = configure_tile<6, 6, true>(nullptr, nullptr)) != cudaSuccess) return e;
    if ((e = configure_tile<8, 4, true>(nullptr, nullptr)) != cudaSuccess) return e;
    if ((e = configure_tile<4, 8, true>(nullptr, nullptr)) != cudaSuccess) return e;
    if ((e = configure_tile<4, 4, false>(nullptr, nullptr)) != cudaSuccess) return e;
    if ((e = configure_tile<2, 2, false>(nullptr, nullptr)) != cudaSuccess) return e;
    int *uptr;
    return cudaGetSymbolAddress((void **)&uptr, g_unit_ptr);
}

void tile_dims(int tile, int *bm, int *bn) {
    switch (tile) {
        case FMM_TILE_96x96: *bm = 96; *bn = 96; break;
        case FMM_TILE_64x64: *bm = 64; *bn = 64; break;
        case FMM_TILE_32x32: *bm = 32; *bn = 32; break;
        case FMM_TILE_128x64: *bm = 128; *bn = 64; break;
        case FMM_TILE_64x128: *bm = 64; *bn = 128; break;
        default: *bm = 128; *bn = 128; break;
    }
}

// Pick the tile with the least estimated time: CTAs run in waves over the
// SMs, each CTA costs its padded FMAs plus its share of chain additions.
int resolve_tile(int requested, int64_t mL, int64_t nL, int64_t kL, int64_t leaves,
                 double extra_a, double extra_b, int num_sms) {
    if (requested != FMM_TILE_AUTO) return requested;
    const int cands[] = {FMM_TILE_128x128, FMM_TILE_128x64, FMM_TILE_64x128, FMM_TILE_96x96,
                         FMM_TILE_64x64, FMM_TILE_32x32};
    int best = FMM_TILE_128x128;
    double best_t = 1e300;
    for (int t : cands) {
        int bm, bn;
        tile_dims(t, &bm, &bn);
        const double tiles = double((mL + bm - 1) / bm) * double((nL + bn - 1) / bn);
        const double ctas = tiles * double(leaves);
        // CTAs resident per SM for this tile (register-limited)
        const int per_sm = (bm * bn >= 128 * 64) ? 1 : (bm * bn >= 64 * 64 ? 2 : 4);
        const double waves = std::ceil(ctas / double(num_sms * per_sm));
        const double cta_cost = double(bm) * bn * kL * (1.0 + extra_a / bn + extra_b / bm) * per_sm;
        // small tiles also pay more shared-memory traffic per FMA
        const double small = (bm * bn <= 32 * 32) ? 1.15 : (bm * bn <= 64 * 64 ? 1.03 : 1.0);
        const double est = waves * cta_cost * small;
        if (est < best_t * 0.999) {
            best_t = est;
            best = t;
        }
    }
    return best;
}

cudaError_t launch_leaf_gemm(const LeafLaunch &a, cudaStream_t s, int *launches) {
    KParams p{};
    p.A = a.A; p.lda = a.lda; p.B = a.B; p.ldb = a.ldb; p.C = a.C; p.ldc = a.ldc;
    p.mL = a.mL; p.kL = a.kL; p.nL = a.nL;
    p.a_ptr = a.a_ptr; p.a_code = a.a_code; p.a_coef = a.a_coef;
    p.b_ptr = a.b_ptr; p.b_code = a.b_code; p.b_coef = a.b_coef;
    p.c_ptr = a.c_ptr; p.c_code = a.c_code; p.c_coef = a.c_coef;
    p.slotA = a.slotA; p.slotA_stride = a.slotA_stride;
    p.slotB = a.slotB; p.slotB_stride = a.slotB_stride;
    p.wsM = a.wsM; p.epi = a.epi;
    p.Ab = a.Ab; p.Bb = a.Bb; p.Cb = a.Cb;
    const int64_t batch = a.batch > 0 ? a.batch : 1;
    if (batch > 65535) return cudaErrorInvalidValue;
    switch (a.tile) {
        case FMM_TILE_96x96: return launch_tile<6, 6, true>(p, a.leaves, batch, s, launches);
        case FMM_TILE_64x64: return launch_tile<4, 4, false>(p, a.leaves, batch, s, launches);
        case FMM_TILE_32x32: return launch_tile<2, 2, false>(p, a.leaves, batch, s, launches);
        case FMM_TILE_128x64: return launch_tile<8, 4, true>(p, a.leaves, batch, s, launches);
        case FMM_TILE_64x128: return launch_tile<4, 8, true>(p, a.leaves, batch, s, launches);
        default: return launch_tile<8, 8, true>(p, a.leaves, batch, s, launches);
    }
}

cudaError_t launch_form_slots(const double *X, int64_t ldx, int64_t rows, int64_t cols,
                              int64_t slots, const int *slot_leaf, const int *ptr,
                              const int *code, const double *coef, double *out,
                              int64_t out_stride, cudaStream_t s, int *launches) {
    const unsigned gx = (unsigned)(rows < 4096 ? rows : 4096);
    for (int64_t sb = 0; sb < slots; sb += 65535) {
        const int64_t cnt = slots - sb < 65535 ? slots - sb : 65535;
        form_slots_kernel<<<dim3(gx, (unsigned)cnt), 256, 0, s>>>(
            X, ldx, rows, cols, sb, slot_leaf, ptr, code, coef, out, out_stride);
        ++*launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_w_pass(double *C, int64_t ldc, int64_t mL, int64_t nL, int gridN,
                          int64_t blocks, const int *cq_ptr, const int *cq_leaf,
                          const double *cq_coef, const double *wsM, int accumulate,
                          cudaStream_t s, int *launches) {
    const unsigned gx = (unsigned)(mL < 4096 ? mL : 4096);
    for (int64_t qb = 0; qb < blocks; qb += 65535) {
        const int64_t cnt = blocks - qb < 65535 ? blocks - qb : 65535;
        w_pass_kernel<<<dim3(gx, (unsigned)cnt), 256, 0, s>>>(C, ldc, mL, nL, gridN, qb, cq_ptr,
                                                               cq_leaf, cq_coef, wsM, accumulate);
        ++*launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_level_form(const double *parent, int64_t parent_ld, int64_t parent_stride,
                              int64_t parents, int64_t rows, int64_t cols, int R, const int *ptr,
                              const int *code, const double *coef, double *out, cudaStream_t s,
                              int *launches) {
    const int64_t outs = parents * R;
    const unsigned gx = (unsigned)(rows < 1024 ? rows : 1024);
    const unsigned bx = cols >= 256 ? 256 : (cols >= 128 ? 128 : 64);
    for (int64_t ob = 0; ob < outs; ob += 65535) {
        const int64_t cnt = outs - ob < 65535 ? outs - ob : 65535;
        level_form_kernel<<<dim3(gx, (unsigned)cnt), bx, 0, s>>>(parent, parent_ld, parent_stride,
                                                                 rows, cols, R, ob, ptr, code, coef, out);
        ++*launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_level_w(const double *child, int64_t rows, int64_t cols, int R, int gridN,
                           int MN, double *parent, int64_t parent_ld, int64_t parent_stride,
                           int64_t parents, const int *w_ptr, const int *w_r, const double *w_coef,
                           int accumulate, cudaStream_t s, int *launches) {
    const int64_t outs = parents * MN;
    const unsigned gx = (unsigned)(rows < 1024 ? rows : 1024);
    const unsigned bx = cols >= 256 ? 256 : (cols >= 128 ? 128 : 64);
    for (int64_t ob = 0; ob < outs; ob += 65535) {
        const int64_t cnt = outs - ob < 65535 ? outs - ob : 65535;
        level_w_kernel<<<dim3(gx, (unsigned)cnt), bx, 0, s>>>(child, rows, cols, R, gridN, MN, parent,
                                                              parent_ld, parent_stride, ob, w_ptr,
                                                              w_r, w_coef, accumulate);
        ++*launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_level_stream(const double *parent, int64_t parent_ld, int64_t parent_stride,
                                int64_t parents, int64_t rows, int64_t cols, int gridR, int gridC, int R,
                                const int *ptr, const int *code, const double *coef, double *out,
                                cudaStream_t s, int *launches) {
    const int NB = gridR * gridC;
    if (NB > 64 || R > 128) return cudaErrorInvalidValue;
    const size_t smem = size_t(NB) * 256 * 8;
    static bool configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(level_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             64 * 256 * 8);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    const int64_t total = parents * rows * cols;
    level_stream_kernel<<<(unsigned)((total + 255) / 256), 256, smem, s>>>(
        parent, parent_ld, parent_stride, rows, cols, gridC, NB, R, parents, ptr, code, coef, out);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_level_w_stream(const double *child, int64_t rows, int64_t cols, int R, int gridN, int MN,
                                  double *parent, int64_t parent_ld, int64_t parent_stride, int64_t parents,
                                  const int *w_ptr, const int *w_r, const double *w_coef, int accumulate,
                                  cudaStream_t s, int *launches) {
    if (R > 128 || MN > 128) return cudaErrorInvalidValue;
    const size_t smem = size_t(R) * 128 * 8;
    static bool configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(level_w_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             128 * 128 * 8);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    const int64_t total = parents * rows * cols;
    level_w_stream_kernel<<<(unsigned)((total + 127) / 128), 128, smem, s>>>(
        child, rows, cols, R, gridN, MN, parent, parent_ld, parent_stride, parents, w_ptr, w_r, w_coef,
        accumulate);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_block_axpy(const double *X, int64_t xld, int64_t xstride, double *Y, int64_t yld,
                              int64_t ystride, int64_t parents, int64_t rows, int64_t cols, double c,
                              int first, cudaStream_t s, int *launches) {
    const int64_t total = parents * rows * cols;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
    block_axpy_kernel<<<blocks, 256, 0, s>>>(X, xld, xstride, Y, yld, ystride, parents, rows, cols, c, first);
    ++*launches;
    return cudaGetLastError();
}

// Thin classical products (the peeling fringes of Section 3.5: at most
// M^L - 1 rows or N^L - 1 columns), where a 2-D tile would mostly compute
// padding.  Both are deterministic: fixed k-slices reduced in a fixed order.

// k <= 32 (the k-fringe): C = A B as a short sum per element; a warp covers
// 32 consecutive columns of one row (A broadcast, B and C coalesced).
__global__ void __launch_bounds__(256) thin_k_kernel(const double *A, int64_t lda, const double *B, int64_t ldb,
                                                     double *C, int64_t ldc, int64_t m, int64_t k, int64_t n) {
    const int64_t colb = (n + 31) / 32;
    for (int64_t g = (int64_t)blockIdx.x * 8 + threadIdx.x / 32; g < m * colb; g += (int64_t)gridDim.x * 8) {
        const int64_t i = g / colb, j = (g % colb) * 32 + threadIdx.x % 32;
        if (j >= n) continue;
        double acc = 0.0;
        for (int64_t p = 0; p < k; ++p) acc = fma(__ldg(A + i * lda + p), __ldg(B + p * ldb + j), acc);
        C[i * ldc + j] = acc;
    }
}

// m <= 32 rows: CTA = 32 columns x 8 k-slices; rows in groups of 8.  grid ceil(n/32).
__global__ void __launch_bounds__(256) thin_rows_kernel(const double *A, int64_t lda, const double *B, int64_t ldb,
                                                        double *C, int64_t ldc, int64_t m, int64_t k, int64_t n) {
    __shared__ double red[8][8][33];
    const int col = threadIdx.x % 32, ks = threadIdx.x / 32;
    const int64_t j = (int64_t)blockIdx.x * 32 + col;
    for (int64_t i0 = 0; i0 < m; i0 += 8) {
        double acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = 0.0;
        if (j < n) {
            for (int64_t p = ks; p < k; p += 8) {
                const double b = B[p * ldb + j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (i0 + i < m) acc[i] = fma(__ldg(A + (i0 + i) * lda + p), b, acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) red[ks][i][col] = acc[i];
        __syncthreads();
        if (ks == 0 && j < n) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                double v = red[0][i][col];
#pragma unroll
                for (int t = 1; t < 8; ++t) v += red[t][i][col];
                if (i0 + i < m) C[(i0 + i) * ldc + j] = v;
            }
        }
        __syncthreads();
    }
}

// n <= 32 columns: one warp per row of C, lanes over k, columns in groups of
// 8, butterfly reduction across the warp.  grid ceil(m/8), 256 threads.
__global__ void __launch_bounds__(256) thin_cols_kernel(const double *A, int64_t lda, const double *B, int64_t ldb,
                                                        double *C, int64_t ldc, int64_t m, int64_t k, int64_t n) {
    const int lane = threadIdx.x % 32;
    const int64_t i = (int64_t)blockIdx.x * 8 + threadIdx.x / 32;
    if (i >= m) return;
    for (int64_t j0 = 0; j0 < n; j0 += 8) {
        double acc[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[jj] = 0.0;
        for (int64_t p = lane; p < k; p += 32) {
            const double a = A[i * lda + p];
            const double *b = B + p * ldb + j0;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
                if (j0 + jj < n) acc[jj] = fma(a, __ldg(b + jj), acc[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
            for (int o = 16; o > 0; o >>= 1) acc[jj] += __shfl_xor_sync(0xffffffffu, acc[jj], o);
        if (lane == 0)
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
                if (j0 + jj < n) C[i * ldc + j0 + jj] = acc[jj];
    }
}

cudaError_t launch_classical(const double *A, int64_t lda, const double *B, int64_t ldb,
                             double *C, int64_t ldc, int64_t m, int64_t k, int64_t n, int tile,
                             cudaStream_t s, int *launches) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (tile == FMM_TILE_AUTO && k > 0 && k <= 32 && m > 32 && n > 32) {
        const int64_t warps = m * ((n + 31) / 32);
        thin_k_kernel<<<(unsigned)std::min<int64_t>((warps + 7) / 8, 152 * 64), 256, 0, s>>>(A, lda, B, ldb, C, ldc,
                                                                                          m, k, n);
        ++*launches;
        return cudaGetLastError();
    }
    if (tile == FMM_TILE_AUTO && k > 0 && (m <= 32 || n <= 32)) {
        if (m <= 32)
            thin_rows_kernel<<<(unsigned)((n + 31) / 32), 256, 0, s>>>(A, lda, B, ldb, C, ldc, m, k, n);
        else
            thin_cols_kernel<<<(unsigned)((m + 7) / 8), 256, 0, s>>>(A, lda, B, ldb, C, ldc, m, k, n);
        ++*launches;
        return cudaGetLastError();
    }
    int *uptr, *ucode;
    double *ucoef;
    cudaError_t e;
    if ((e = cudaGetSymbolAddress((void **)&uptr, g_unit_ptr)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&ucode, g_unit_code)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&ucoef, g_unit_coef)) != cudaSuccess) return e;
    LeafLaunch a{};
    a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.C = C; a.ldc = ldc;
    a.mL = m; a.kL = k; a.nL = n; a.leaves = 1;
    a.a_ptr = a.b_ptr = a.c_ptr = uptr;
    a.a_code = a.b_code = a.c_code = ucode;
    a.a_coef = a.b_coef = a.c_coef = ucoef;
    a.epi = EPI_STORE;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    a.tile = resolve_tile(tile, m, n, k, 1, 0.0, 0.0, sms);
    return launch_leaf_gemm(a, s, launches);
}

}  // namespace fmm
