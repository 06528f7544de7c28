// TF32 leaf products on the tensor cores (precision variants FMM_PREC_TF32
// and, with three TF32 pair products per leaf, FMM_PREC_FP32):
// the FP64 leaf operands S_r, T_r are rounded to TF32 (10-bit significand,
// round to nearest) in FP32 K-major layout, multiplied by tcgen05
// (kind::tf32, FP32 accumulation in TMEM over the whole k), and the FP32
// products are widened back to FP64 for the W combination.  Expected
// relative error ~ 2^-11 per operand; stated per result by the benchmark.
//
// The FP32-accurate variant splits each operand into a TF32 pair and sums
// the three pair products in one launch over a tripled k, in chunks of 512 k
// (x3) that the drain warps add in FP32 registers (the tensor core's own FP32
// sums over a long k lose accuracy; see tf32_gemm<BN, true>).
//
// Same pipeline as the emulated-FP64 residue GEMM: persistent CTAs over
// 128 x 256 tiles (128 x 128 for narrow products) in groups of 16 tile rows,
// TMA (128-byte swizzle) into an mbarrier ring, one load thread, one MMA
// thread, eight drain warps; two TMEM accumulators let a tile's drain overlap
// the next tile's MMAs.  Every wait is bounded.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "fmm_internal.h"
#include "tcgen05.cuh"

namespace fmm {

__device__ int g_tf32_error = 0;   // set when a bounded wait gives up

namespace {

using namespace tc;

constexpr int TB_M = 128, TB_K = 32;   // TB_K fp32 = 128 bytes: one swizzled row
constexpr int TB_A = TB_M * TB_K * 4;

// BN = 256: 8 drain warps (two column halves), 4 stages of 48 KB; BN = 128:
// 4 drain warps, 6 stages of 32 KB.  Two TMEM accumulators of BN columns.
template <int BN>
struct TfCfg;
template <>
struct TfCfg<256> { static constexpr int DW = 8, STAGES = 4; };
template <>
struct TfCfg<128> { static constexpr int DW = 4, STAGES = 6; };
constexpr int TB_TBUF = 2;
// CH (k in chunks summed in drain-warp registers): twice the drain warps, so
// that each holds the running sums of 64 columns
template <int BN, bool CH>
__host__ __device__ constexpr int tf_dw() { return TfCfg<BN>::DW * (CH ? 2 : 1); }
template <int BN, bool CH>
constexpr int tf_threads() { return (tf_dw<BN, CH>() + 2) * 32; }
template <int BN>
constexpr int tf_smem() { return TfCfg<BN>::STAGES * (TB_A + BN * TB_K * 4) + 1024 + 256; }

// Tile t of the persistent sequence -> (plane, tile row, tile column), in
// groups of 16 tile rows taken column by column (panels shared in L2).
__device__ __forceinline__ void tf_tile(int64_t tile, int64_t per_plane, int tiles_m, int tiles_n, int &z, int &tm,
                                        int &tn) {
    constexpr int G = 16;
    z = int(tile / per_plane);
    const int rem = int(tile % per_plane);
    const int g = rem / (G * tiles_n);
    const int tm0 = g * G;
    const int gsz = min(G, tiles_m - tm0);
    const int within = rem - g * G * tiles_n;
    tn = within / gsz;
    tm = tm0 + within % gsz;
}

// OT: the products' element type (double, or float for the fused one-level
// path, whose W combination runs in FP32)
template <int BN, bool CH, typename OT = double>
__global__ void __launch_bounds__(tf_threads<BN, CH>(), 1)
tf32_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          OT *Out, int64_t m, int64_t n, int kblocks, int chunk_kb, int tiles_m, int tiles_n,
          int64_t tiles_total, int64_t ldo, int64_t out_stride, int accumulate, int *err,
          unsigned long long wait_ns, int dry) {
    constexpr int DW = tf_dw<BN, CH>(), STAGES = TfCfg<BN>::STAGES;
    constexpr int CW = 4 * BN / DW;   // accumulator columns per drain warp
    constexpr int TB_B = BN * TB_K * 4, STAGE = TB_A + TB_B;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + TB_TBUF;
    uint64_t *mdone = tempty + TB_TBUF;   // the MMA thread's last commit
    uint32_t *tmem_slot = (uint32_t *)(mdone + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t per_plane = (int64_t)tiles_m * tiles_n;
    // k in chunks of chunk_kb blocks: each chunk is summed in TMEM and added
    // to the drain warps' FP32 registers (round to nearest) before the next
    const int nchunks = (kblocks + chunk_kb - 1) / chunk_kb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < TB_TBUF; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], DW * 32); }
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(tmem_slot)), "r"(TB_TBUF * BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == DW) {
        if (lane == 0 && !dry) {
            int64_t g = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < tiles_total && ok; tile += gridDim.x) {
                int z, tm, tn;
                tf_tile(tile, per_plane, tiles_m, tiles_n, z, tm, tn);
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    const int s = int(g % STAGES);
                    if (g >= STAGES && !mbar_wait(&empty[s], uint32_t(((g / STAGES) - 1) & 1), wait_ns)) {
                        atomicExch(err, 1);
                        ok = false;
                        break;
                    }
                    unsigned char *sa = smem + s * STAGE, *sb = sa + TB_A;
                    mbar_expect_tx(&full[s], STAGE);
                    tma_load_3d(sa, &tmA, kb * TB_K, tm * TB_M, z, &full[s]);
                    tma_load_3d(sb, &tmB, kb * TB_K, tn * BN, z, &full[s]);
                }
            }
            // no bulk copy of this CTA may still be in flight when it exits
            for (int64_t j = g > STAGES ? g - STAGES : 0; j < g; ++j)
                if (!mbar_wait(&full[j % STAGES], uint32_t((j / STAGES) & 1), wait_ns)) atomicExch(err, 1);
        }
    } else if (warp == DW + 1) {
        if (lane == 0 && !dry) {
            // FP32 accumulator, TF32 A and B, both K-major
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                                   ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TB_M >> 4) << 24);
            bool ok = true;
            int64_t g = 0, cg = 0;   // global k-block and chunk counters
            for (int64_t tile = blockIdx.x; tile < tiles_total && ok; tile += gridDim.x) {
                int kb = 0;
                for (int c = 0; c < nchunks && ok; ++c, ++cg) {
                    const int b = int(cg % TB_TBUF);
                    if (cg >= TB_TBUF && !mbar_wait(&tempty[b], uint32_t(((cg / TB_TBUF) - 1) & 1), wait_ns)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t acc = tmem + (uint32_t)(b * BN);
                    const int kend = min(kblocks, (c + 1) * chunk_kb);
                    for (int first = 1; kb < kend; ++kb, ++g, first = 0) {
                        const int s = int(g % STAGES);
                        if (!mbar_wait(&full[s], uint32_t((g / STAGES) & 1), wait_ns)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t a0 = su32(smem + s * STAGE), b0 = a0 + TB_A;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)   // K = 8 tf32 (32 bytes) per MMA
                            mma_tf32(acc, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32), idesc,
                                     (first && kk == 0) ? 0u : 1u);
                        mma_commit(&empty[s]);
                    }
                    mma_commit(&tfull[b]);
                }
            }
            // every MMA issued here completes before TMEM is freed
            mma_commit(mdone);
            if (!mbar_wait(mdone, 0u, wait_ns)) ok = false;
            if (!ok) atomicExch(err, 1);
        }
    } else {
        // drain warps: warp w reads TMEM lanes 32*(w%4)..+31 (rows of the tile)
        // and the CW-column slice w/4 of the accumulator
        const int lg = warp % 4, ch = warp / 4;
        bool ok = true;
        int64_t cg = 0;
        for (int64_t tile = blockIdx.x; tile < tiles_total && ok; tile += gridDim.x) {
            int z, tm, tn;
            tf_tile(tile, per_plane, tiles_m, tiles_n, z, tm, tn);
            const int64_t row = (int64_t)tm * TB_M + lg * 32 + lane;
            const int64_t col0 = (int64_t)tn * BN + ch * CW;
            const int64_t cols = min((int64_t)CW, n - col0);
            OT *out = Out + (int64_t)z * out_stride + row * ldo + col0;
            const bool pairs = ((((uintptr_t)out) & 15) == 0);
            // 16 accumulated columns from c0 on, widened to FP64 (or kept in
            // FP32) and stored (added)
            auto store16 = [&](int c0, const float *v16) {
                if (row >= m || c0 >= cols) return;
                if constexpr (sizeof(OT) == 4) {
                    if (pairs && c0 + 16 <= cols) {
#pragma unroll
                        for (int j = 0; j < 16; j += 4) {
                            float4 v = make_float4(v16[j], v16[j + 1], v16[j + 2], v16[j + 3]);
                            float4 *dst = reinterpret_cast<float4 *>(out + c0 + j);
                            if (accumulate) {
                                const float4 o = *dst;
                                v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
                            }
                            *dst = v;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < cols) out[c0 + j] = accumulate ? out[c0 + j] + v16[j] : v16[j];
                    }
                    return;
                }
                if (pairs && c0 + 16 <= cols) {
                    // 16 consecutive columns as eight 16-byte stores
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        double2 v = make_double2((double)v16[j], (double)v16[j + 1]);
                        double2 *dst = reinterpret_cast<double2 *>(reinterpret_cast<double *>(out) + c0 + j);
                        if (accumulate) {
                            const double2 o = *dst;
                            v.x += o.x;
                            v.y += o.y;
                        }
                        *dst = v;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (c0 + j < cols) {
                            const double v = (double)v16[j];
                            double *od = reinterpret_cast<double *>(out);
                            od[c0 + j] = accumulate ? od[c0 + j] + v : v;
                        }
                    }
                }
            };
            if constexpr (!CH) {
                // the whole k summed in TMEM: one drain per tile
                const int b = int(cg % TB_TBUF);
                if (!mbar_wait(&tfull[b], uint32_t((cg / TB_TBUF) & 1), wait_ns)) { ok = false; break; }
                ++cg;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * BN + ch * CW);
#pragma unroll
                for (int c0 = 0; c0 < CW; c0 += 16) {
                    uint32_t r[16];
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                                 : "r"(base + (uint32_t)c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    float v16[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v16[j] = __uint_as_float(r[j]);
                    store16(c0, v16);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&tempty[b]);
            } else {
                // chunks of k summed in TMEM, added here in FP32 (round to nearest)
                float acc[CW];
#pragma unroll
                for (int j = 0; j < CW; ++j) acc[j] = 0.0f;
                for (int c = 0; c < nchunks; ++c, ++cg) {
                    const int b = int(cg % TB_TBUF);
                    if (!mbar_wait(&tfull[b], uint32_t((cg / TB_TBUF) & 1), wait_ns)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t base = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * BN + ch * CW);
#pragma unroll
                    for (int c0 = 0; c0 < CW; c0 += 16) {
                        uint32_t r[16];
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                                       "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                                     : "r"(base + (uint32_t)c0));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(r[j]);
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(&tempty[b]);
                }
                if (!ok) break;
#pragma unroll
                for (int c0 = 0; c0 < CW; c0 += 16) store16(c0, acc + c0);
            }
        }
        if (!ok && lane == 0) atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TB_TBUF * BN) : "memory");
}

__device__ __forceinline__ float to_tf32(float f) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    return __uint_as_float(r);
}

// The TF32 pair of x: hi = tf32(x) and lo = tf32(x - hi), x taken in FP32
// (hi + lo carries 22 significant bits of it).
__device__ __forceinline__ float2 tf32_pair(double x) {
    const float f = (float)x;
    const float hi = to_tf32(f);
    return make_float2(hi, to_tf32(f - hi));
}

// X (rows x cols per plane, ld, plane stride) -> TF32 in FP32, rows padded to
// kpad.  split 3 (FP32-accurate products): each row holds three segments of
// kpad, hi | hi | lo, against hi | lo | hi on the T side, so one product over
// 3 kpad sums hi hi + hi lo + lo hi (the lo lo term, 2^-22 relative, is left out).
__global__ void tf32_rows(const double *X, int64_t ldx, int64_t xs, int64_t rows, int64_t cols,
                          int64_t kpad, int64_t planes, int split, float *out) {
    const int64_t kk = kpad * split;
    const int64_t total = planes * rows * kk;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pl = g / (rows * kk), rem = g % (rows * kk), i = rem / kk, jj = rem % kk;
        const int64_t seg = jj / kpad, j = jj % kpad;
        float v = 0.0f;
        if (j < cols) {
            const double x = X[pl * xs + i * ldx + j];
            if (split == 1) {
                v = to_tf32((float)x);
            } else {
                const float2 hl = tf32_pair(x);
                v = seg == 2 ? hl.y : hl.x;
            }
        }
        out[g] = v;
    }
}

// Y (rows x cols per plane) -> TF32 of Y^T (cols x split kpad), through 32x32
// tiles; split 3: segments hi | lo | hi of each row of Y^T.
__global__ void tf32_cols_t(const double *Y, int64_t ldy, int64_t ys, int64_t rows, int64_t cols,
                            int64_t kpad, int split, float *out) {
    __shared__ float tile[32][33], tile_lo[32][33];
    const int64_t pl = blockIdx.z;
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + r, j = j0 + tx;
        float2 hl = make_float2(0.0f, 0.0f);
        if (i < rows && j < cols) {
            const double y = Y[pl * ys + i * ldy + j];
            hl = split == 1 ? make_float2(to_tf32((float)y), 0.0f) : tf32_pair(y);
        }
        tile[r][tx] = hl.x;
        tile_lo[r][tx] = hl.y;
    }
    __syncthreads();
    const int64_t kk = kpad * split;
    for (int r = ty; r < 32; r += 8) {
        const int64_t j = j0 + r, i = i0 + tx;
        if (j < cols && i < kpad) {
            float *o = out + (pl * cols + j) * kk + i;
            o[0] = tile[tx][r];
            if (split == 3) {
                o[kpad] = tile_lo[tx][r];
                o[2 * kpad] = tile[tx][r];
            }
        }
    }
}

// ---------------------------------------------------------------------
// First recursive level fused with the conversion (TF32-family leaves, one
// level): each FP64 operand is read once and every child S_r = sum_t c_t A_t
// (Section 3.1's S formation) is formed in FP32 from the block values rounded
// to FP32 once, then written as leaf r's TF32 operand (split 1) or its hi/lo
// pair segments (split 3), exactly the layout tf32_rows / tf32_cols_t write.
// The FP32 sums add at most a few units of 2^-24 relative to the operand,
// far below TF32's 2^-11 and the pair's 2^-22.  Term lists: CSR over the
// children, code = (block row << 16) | block column, FP64 coefficients.

constexpr int TF_MAX_TERMS = 512, TF_MAX_R = 64;

__device__ __forceinline__ void tf_stage_terms(int R, int gC, const int *ptr, const int *code, const double *coef,
                                               int *sb, float *sc, int *sp) {
    const int nt = __ldg(ptr + R);
    for (int t = threadIdx.x + blockDim.x * threadIdx.y; t < nt; t += blockDim.x * blockDim.y) {
        const int cd = __ldg(code + t);
        sb[t] = (cd >> 16) * gC + (cd & 0xffff);
        sc[t] = (float)__ldg(coef + t);
    }
    for (int o = threadIdx.x + blockDim.x * threadIdx.y; o <= R; o += blockDim.x * blockDim.y) sp[o] = __ldg(ptr + o);
}

// S side: A (ld lda) as a gR x gC grid of blocks rows x cols.  Thread: one row
// i of the child blocks and 4 consecutive columns j of the padded k (columns
// >= cols are zero).  out: R planes of rows x (split kpad) floats.
template <int NB>
__global__ void __launch_bounds__(256) tf32_form_rows(const double *A, int64_t lda, int64_t rows, int64_t cols,
                                                      int gC, int R, const int *ptr, const int *code,
                                                      const double *coef, int64_t kpad, int split, float *out) {
    __shared__ int sb[TF_MAX_TERMS];
    __shared__ float sc[TF_MAX_TERMS];
    __shared__ int sp[TF_MAX_R + 1];
    tf_stage_terms(R, gC, ptr, code, coef, sb, sc, sp);
    __syncthreads();
    const int64_t groups = kpad / 4;
    const int64_t pos = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (pos >= rows * groups) return;
    const int64_t i = pos / groups, j0 = (pos % groups) * 4;
    float v[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const double *x = A + ((int64_t)(b / gC) * rows + i) * lda + (int64_t)(b % gC) * cols + j0;
        if (j0 + 4 <= cols && ((uintptr_t)x & 15) == 0) {
            const double2 x0 = reinterpret_cast<const double2 *>(x)[0], x1 = reinterpret_cast<const double2 *>(x)[1];
            v[b][0] = (float)x0.x; v[b][1] = (float)x0.y; v[b][2] = (float)x1.x; v[b][3] = (float)x1.y;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[b][e] = (j0 + e < cols) ? (float)x[e] : 0.0f;
        }
    }
    const int64_t kk = kpad * split;
    for (int r = 0; r < R; ++r) {
        float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int t = sp[r]; t < sp[r + 1]; ++t) {
            const int bt = sb[t];
            const float c = sc[t];
#pragma unroll
            for (int b = 0; b < NB; ++b)
                if (b == bt) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) a[e] = fmaf(c, v[b][e], a[e]);
                }
        }
        float *o = out + ((int64_t)r * rows + i) * kk + j0;
        float4 hi, lo;
        hi.x = to_tf32(a[0]); hi.y = to_tf32(a[1]); hi.z = to_tf32(a[2]); hi.w = to_tf32(a[3]);
        *reinterpret_cast<float4 *>(o) = hi;
        if (split == 3) {
            lo.x = to_tf32(a[0] - hi.x); lo.y = to_tf32(a[1] - hi.y); lo.z = to_tf32(a[2] - hi.z);
            lo.w = to_tf32(a[3] - hi.w);
            *reinterpret_cast<float4 *>(o + kpad) = hi;      // segments hi | hi | lo
            *reinterpret_cast<float4 *>(o + 2 * kpad) = lo;
        }
    }
}

// T side, transposed: B (ld ldb) as a gR x gC grid of blocks krows x ncols;
// child r's T_r^T (ncols x split kpad, K-major).  CTA: 32 k x 32 n positions
// of the child blocks through shared memory (NB tiles of 32 x 33 floats);
// thread (tx, ty): loads rows ty, ty + 8, ..; writes k = k0 + tx.
template <int NB>
__global__ void __launch_bounds__(256) tf32_form_cols_t(const double *B, int64_t ldb, int64_t krows, int64_t ncols,
                                                        int gC, int R, const int *ptr, const int *code,
                                                        const double *coef, int64_t kpad, int split, float *out) {
    __shared__ int sb[TF_MAX_TERMS];
    __shared__ float sc[TF_MAX_TERMS];
    __shared__ int sp[TF_MAX_R + 1];
    __shared__ float tile[NB][32][33];
    tf_stage_terms(R, gC, ptr, code, coef, sb, sc, sp);
    const int64_t k0 = (int64_t)blockIdx.x * 32, n0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int b = 0; b < NB; ++b)
        for (int r = ty; r < 32; r += 8) {
            const int64_t kr = k0 + r, nc = n0 + tx;
            tile[b][r][tx] = (kr < krows && nc < ncols)
                                 ? (float)B[((int64_t)(b / gC) * krows + kr) * ldb + (int64_t)(b % gC) * ncols + nc]
                                 : 0.0f;
        }
    __syncthreads();
    const int64_t kk = kpad * split;
    const int64_t kc = k0 + tx;
    if (kc >= kpad) return;
    // this thread's four n positions (ty, ty + 8, ty + 16, ty + 24): every
    // block's values read from shared memory once, one walk over the terms
    float v[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) v[b][q] = tile[b][tx][ty + 8 * q];
    for (int r = 0; r < R; ++r) {
        float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int t = sp[r]; t < sp[r + 1]; ++t) {
            const int bt = sb[t];
            const float c = sc[t];
#pragma unroll
            for (int b = 0; b < NB; ++b)
                if (b == bt) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) a[q] = fmaf(c, v[b][q], a[q]);
                }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t nc = n0 + ty + 8 * q;
            if (nc >= ncols) continue;
            float *o = out + ((int64_t)r * ncols + nc) * kk + kc;
            const float hi = to_tf32(a[q]);
            o[0] = hi;
            if (split == 3) {
                o[kpad] = to_tf32(a[q] - hi);   // segments hi | lo | hi
                o[2 * kpad] = hi;
            }
        }
    }
}

typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

std::mutex g_tf_mu;
EncodeFn g_tf_encode = nullptr;

cudaError_t map3d_f32(CUtensorMap *m, void *ptr, int64_t kpad, int64_t rows, int64_t planes, int box_rows) {
    {
        std::lock_guard<std::mutex> g(g_tf_mu);
        if (!g_tf_encode) {
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                             cudaEnableDefault, &q);
            if (e != cudaSuccess) return e;
            if (!fn || q != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
            g_tf_encode = (EncodeFn)fn;
        }
    }
    cuuint64_t gdim[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t gstr[2] = {(cuuint64_t)kpad * 4, (cuuint64_t)(kpad * rows * 4)};
    cuuint32_t box[3] = {(cuuint32_t)TB_K, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_tf_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ptr, gdim, gstr, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int sm_count() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

size_t tf32_workspace(int64_t leaves, int64_t m, int64_t k, int64_t n, int split) {
    const int64_t kk = (k + TB_K - 1) / TB_K * TB_K * split;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    return al(size_t(leaves) * m * kk * 4) + al(size_t(leaves) * n * kk * 4);
}

cudaError_t tf32_prepare() {
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && !configured[dev]) {
        if ((e = cudaFuncSetAttribute(tf32_gemm<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tf_smem<256>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(tf32_gemm<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tf_smem<128>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(tf32_gemm<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tf_smem<128>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(tf32_gemm<256, false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tf_smem<256>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(tf32_gemm<128, false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tf_smem<128>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(tf32_gemm<128, true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tf_smem<128>())) != cudaSuccess)
            return e;
        configured[dev] = true;
    }
    int *err = nullptr;
    return cudaGetSymbolAddress((void **)&err, g_tf32_error);
}

cudaError_t read_tf32_error(int *flag, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_tf32_error, sizeof(int));
    if (e != cudaSuccess) return e;
    if (clear && *flag) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_tf32_error, &zero, sizeof(int));
    }
    return e;
}

// The TF32 GEMM over operand planes already in the leaves' layout: fa
// (leaves x m x split kpad), fb (leaves x n x split kpad), both 256-byte
// aligned; Out[leaf] (m x n, ldo, leaf stride os) (+)= fa fb^T, stored as OT
// (double, or float for the fused one-level path).
template <typename OT>
static cudaError_t tf32_gemm_planes(float *fa, float *fb, OT *Out, int64_t ldo, int64_t os, int64_t leaves,
                                    int64_t m, int64_t n, int64_t kpad, int accumulate, cudaStream_t s,
                                    int *launches, int split, int tile) {
    cudaError_t e;
    int *err = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&err, g_tf32_error)) != cudaSuccess) return e;
    const int64_t kk = kpad * split;
    CUtensorMap ta, tb;
    // the chunked sums (FP32-accurate products) keep 64 running sums per drain
    // thread: 128-wide tiles with 8 drain warps fit them in registers
    const bool chunked = split == 3;
    const bool wide = n >= 256 && !chunked && tile != FMM_TILE_128x128;
    const int bn = wide ? 256 : 128;
    if ((e = map3d_f32(&ta, fa, kk, m, leaves, TB_M)) != cudaSuccess) return e;
    if ((e = map3d_f32(&tb, fb, kk, n, leaves, bn)) != cudaSuccess) return e;
    const int64_t tm = (m + TB_M - 1) / TB_M, tn = (n + bn - 1) / bn;
    const int64_t tiles = tm * tn * leaves;
    // FP32-accurate products: chunks of 512 k (1536 tripled) summed on the CUDA
    // cores; one TF32 product: the whole k in TMEM
    const int kblocks = int(kk / TB_K), chunk_kb = chunked ? 3 * 512 / TB_K : kblocks;
    const unsigned ctas = (unsigned)std::min<int64_t>(tiles, sm_count());
    cudaEvent_t t0 = timing_mark(s);
#define FMM_TF32_GEMM(BN_, CH_)                                                                                \
    tf32_gemm<BN_, CH_, OT><<<ctas, tf_threads<BN_, CH_>(), tf_smem<BN_>(), s>>>(ta, tb, Out, m, n, kblocks, chunk_kb, \
                                                                          int(tm), int(tn), tiles, ldo, os,    \
                                                                          accumulate, err, wait_limit_ns(), 0)
    if (chunked) FMM_TF32_GEMM(128, true);
    else if (wide) FMM_TF32_GEMM(256, false);
    else FMM_TF32_GEMM(128, false);
#undef FMM_TF32_GEMM
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (t0 && !timing_mark(s)) timing_unmark();
    return cudaSuccess;
}

static size_t tf_al(size_t x) { return (x + 255) & ~size_t(255); }

// Out[leaf] (m x n, ldo, leaf stride os) (+)= tf32(S[leaf]) tf32(T[leaf]);
// split 3: the FP32-accurate sum of the three TF32 pair products.
cudaError_t tf32_products(const double *S, int64_t lds, int64_t ss, const double *T, int64_t ldt,
                          int64_t ts, double *Out, int64_t ldo, int64_t os, int64_t leaves, int64_t m,
                          int64_t k, int64_t n, int accumulate, void *ws, cudaStream_t s, int *launches,
                          int split, int tile) {
    if (split != 1 && split != 3) return cudaErrorInvalidValue;
    cudaError_t e = tf32_prepare();
    if (e != cudaSuccess) return e;
    const int64_t kpad = (k + TB_K - 1) / TB_K * TB_K, kk = kpad * split;
    float *fa = (float *)ws;
    float *fb = (float *)((char *)ws + tf_al(size_t(leaves) * m * kk * 4));
    {
        const int64_t total = leaves * m * kk;
        const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
        tf32_rows<<<blocks, 256, 0, s>>>(S, lds, ss, m, k, kpad, leaves, split, fa);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        if (leaves > 65535) return cudaErrorInvalidValue;
        dim3 grid((unsigned)((kpad + 31) / 32), (unsigned)((n + 31) / 32), (unsigned)leaves);
        tf32_cols_t<<<grid, dim3(32, 8), 0, s>>>(T, ldt, ts, k, n, kpad, split, fb);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return tf32_gemm_planes(fa, fb, Out, ldo, os, leaves, m, n, kpad, accumulate, s, launches, split, tile);
}

// One recursive level fused with the conversion: A (ld lda) as an gM x gK
// grid of mL x kL blocks and B (ld ldb) as gK x gN blocks of kL x nL; the
// level's term lists (u: S side, v: T side); the R leaf products into Out in
// FP32 (mL x nL each, ldo, leaf stride os; their W combination is
// tf32_w_level).  ws: the same operand planes as tf32_products for R leaves
// of mL x kL x nL.
cudaError_t tf32_first_level_products(const double *A, int64_t lda, const double *B, int64_t ldb, int64_t mL,
                                      int64_t kL, int64_t nL, int gM, int gK, int gN, int R, const int *u_ptr,
                                      const int *u_code, const double *u_coef, const int *v_ptr,
                                      const int *v_code, const double *v_coef, float *Out, int64_t ldo,
                                      int64_t os, void *ws, cudaStream_t s, int *launches, int split, int tile) {
    if (split != 1 && split != 3) return cudaErrorInvalidValue;
    if (R > TF_MAX_R || R > 65535) return cudaErrorInvalidValue;
    cudaError_t e = tf32_prepare();
    if (e != cudaSuccess) return e;
    const int64_t kpad = (kL + TB_K - 1) / TB_K * TB_K, kk = kpad * split;
    float *fa = (float *)ws;
    float *fb = (float *)((char *)ws + tf_al(size_t(R) * mL * kk * 4));
    const int nbA = gM * gK, nbB = gK * gN;
    {
        const int64_t threads = mL * (kpad / 4);
        const unsigned blocks = (unsigned)((threads + 255) / 256);
#define FMM_TFR(NB) tf32_form_rows<NB><<<blocks, 256, 0, s>>>(A, lda, mL, kL, gK, R, u_ptr, u_code, u_coef, kpad, split, fa)
        switch (nbA) {
            case 4: FMM_TFR(4); break;
            case 6: FMM_TFR(6); break;
            case 8: FMM_TFR(8); break;
            case 9: FMM_TFR(9); break;
            default: return cudaErrorNotSupported;
        }
#undef FMM_TFR
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        const dim3 grid((unsigned)((kpad + 31) / 32), (unsigned)((nL + 31) / 32));
#define FMM_TFC(NB) tf32_form_cols_t<NB><<<grid, dim3(32, 8), 0, s>>>(B, ldb, kL, nL, gN, R, v_ptr, v_code, v_coef, kpad, split, fb)
        switch (nbB) {
            case 4: FMM_TFC(4); break;
            case 6: FMM_TFC(6); break;
            case 8: FMM_TFC(8); break;
            case 9: FMM_TFC(9); break;
            default: return cudaErrorNotSupported;
        }
#undef FMM_TFC
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return tf32_gemm_planes(fa, fb, Out, ldo, os, R, mL, nL, kpad, 0, s, launches, split, tile);
}

// The W combination of one level from FP32 leaf products (TF32-family leaves,
// the fused path above): C block q = (a, c) of the gM x gN grid,
// C_q (+)= sum_t w_t P[r_t], the sum in FP32 (a few units of 2^-24 relative,
// below the products' own 2^-11 or 2^-22) and stored in FP64.  Thread: four
// consecutive columns of one row of one block.
__global__ void __launch_bounds__(256) tf32_w_kernel(const float *P, int64_t mL, int64_t nL, int gN, int MN,
                                                     const int *w_ptr, const int *w_r, const double *w_coef,
                                                     double *C, int64_t ldc, int accumulate) {
    const int64_t groups = (nL + 3) / 4;
    const int64_t pos = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (pos >= (int64_t)MN * mL * groups) return;
    const int64_t j0 = (pos % groups) * 4;
    const int64_t rest = pos / groups;
    const int64_t i = rest % mL;
    const int q = int(rest / mL);
    float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int t = __ldg(w_ptr + q); t < __ldg(w_ptr + q + 1); ++t) {
        const float w = (float)__ldg(w_coef + t);
        const float *src = P + ((int64_t)__ldg(w_r + t) * mL + i) * nL + j0;
        if (j0 + 4 <= nL && ((uintptr_t)src & 15) == 0) {
            const float4 v = *reinterpret_cast<const float4 *>(src);
            a[0] = fmaf(w, v.x, a[0]); a[1] = fmaf(w, v.y, a[1]); a[2] = fmaf(w, v.z, a[2]); a[3] = fmaf(w, v.w, a[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (j0 + e < nL) a[e] = fmaf(w, src[e], a[e]);
        }
    }
    double *out = C + ((int64_t)(q / gN) * mL + i) * ldc + (int64_t)(q % gN) * nL + j0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (j0 + e < nL) out[e] = accumulate ? out[e] + (double)a[e] : (double)a[e];
}

cudaError_t tf32_w_level(const float *P, int64_t mL, int64_t nL, int gM, int gN, const int *w_ptr, const int *w_r,
                         const double *w_coef, double *C, int64_t ldc, int accumulate, cudaStream_t s,
                         int *launches) {
    const int MN = gM * gN;
    const int64_t threads = (int64_t)MN * mL * ((nL + 3) / 4);
    if (threads <= 0) return cudaSuccess;
    tf32_w_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(P, mL, nL, gN, MN, w_ptr, w_r, w_coef, C, ldc,
                                                                    accumulate);
    ++*launches;
    return cudaGetLastError();
}

// The timeout path of the TF32 GEMM (see residue_gemm_timeout_probe): one
// dry CTA, the drain warps' first wait runs out with nothing outstanding.
cudaError_t tf32_gemm_timeout_probe(unsigned long long limit_ns, cudaStream_t s) {
    cudaError_t e = tf32_prepare();
    if (e != cudaSuccess) return e;
    int *err = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&err, g_tf32_error)) != cudaSuccess) return e;
    void *buf = nullptr;
    const size_t a_bytes = 128 * 32 * 4, b_bytes = 256 * 32 * 4, o_bytes = 128 * 256 * 8;
    if ((e = cudaMalloc(&buf, a_bytes + b_bytes + o_bytes)) != cudaSuccess) return e;
    char *c = (char *)buf;
    CUtensorMap ta, tb;
    if ((e = map3d_f32(&ta, (float *)c, 32, 128, 1, TB_M)) == cudaSuccess &&
        (e = map3d_f32(&tb, (float *)(c + a_bytes), 32, 256, 1, 256)) == cudaSuccess) {
        tf32_gemm<256, false><<<1, tf_threads<256, false>(), tf_smem<256>(), s>>>(
            ta, tb, (double *)(c + a_bytes + b_bytes), 128, 256, 1, 1, 1, 1, 1, 256, 0, 0, err, limit_ns, 1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    const cudaError_t f = cudaFree(buf);
    return e != cudaSuccess ? e : f;
}

}  // namespace fmm
