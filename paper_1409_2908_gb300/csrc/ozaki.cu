// Emulated-FP64 products on the tensor cores (precision variant
// FMM_PREC_OZAKI_BF16).  For a product S T (FP64):
//
//   1. split   scale row i of S by 2^s_i and column j of T by 2^t_j and round
//              the entries to integers of at most beta bits (ties away from
//              zero), then write their balanced residues modulo each of N
//              pairwise coprime moduli p <= 256 as bfloat16 (|r| <= 128:
//              exact), K-major;
//   2. gemm    Z_p = S'_p T'_p mod p on tcgen05 (kind::f16, FP32 accumulator in
//              TMEM).  Products are < 2^14, so a k-chunk of 512 sums exactly in
//              FP32; each chunk is drained into int32 registers through
//              rotating TMEM buffers while the next chunk is multiplied;
//   3. crt     Z from its N residues as a weighted sum of 16-bit limbs
//              (X = sum_q r_q c_q mod P), brought to [-P/2, P/2), rounded once
//              to FP64 from its integer bits and scaled by 2^-(s_i + t_j).
//
// With integer base coefficients the recursion itself runs on the residues
// (ozaki_fast below): the scaling and the first level share one pass, the
// levels are modular combinations, and the top W level shares the CRT pass.
// Operand tiles reach shared memory by TMA (128-byte swizzle) through an
// mbarrier ring; one thread issues the MMAs, one thread the loads, four or
// eight warps drain TMEM.  Every mbarrier wait is bounded: on timeout the CTA
// records an error, stops issuing work and frees its TMEM.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "fmm_internal.h"
#include "tcgen05.cuh"

namespace fmm {

const int kOzakiModuli[20] = {256, 255, 253, 251, 247, 241, 239, 233, 229, 227,
                              223, 217, 211, 199, 197, 193, 191, 181, 179, 173};

__device__ int g_device_error = 0;   // set when a bounded wait gives up

// Time limit of every bounded device wait in the tensor-core kernels.
static std::atomic<unsigned long long> g_wait_ns{2000000000ull};
unsigned long long wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }
void set_wait_limit_ns(unsigned long long ns) { g_wait_ns.store(ns, std::memory_order_relaxed); }

namespace {

constexpr int OZ_BM = 128, OZ_BK = 64;
constexpr int OZ_CHUNK_KB = 8;          // 8 x 64 = 512 k per exact FP32 chunk
constexpr int OZ_A_BYTES = OZ_BM * OZ_BK * 2;
constexpr int OZ_MAX_MOD = 20;

__constant__ int c_mod[OZ_MAX_MOD];                       // moduli
__constant__ int c_wmod[OZ_MAX_MOD][OZ_MAX_MOD];          // (prod_{l<i} p_l) mod p_j
__constant__ int c_winv[OZ_MAX_MOD];                      // inverse of (prod_{l<j} p_l) mod p_j
__constant__ unsigned c_magic[OZ_MAX_MOD];                // floor(2^32 / p)
__constant__ unsigned c_r32[OZ_MAX_MOD];                  // 2^32 mod p
__constant__ unsigned c_r21[OZ_MAX_MOD], c_r42[OZ_MAX_MOD];  // 2^21 and 2^42 mod p
__constant__ float c_modf[OZ_MAX_MOD], c_invp[OZ_MAX_MOD];  // p and 1/p as floats
__constant__ float c_klimb[2][OZ_MAX_MOD][5];              // 2^(13 i), 2^(14 i) mod p as floats
__constant__ float c_klimbw[OZ_MAX_MOD][3];                // 2^0, 2^22, 2^37 mod p, balanced (|w| <= p/2)
constexpr int OZ_MAX_TERMS = 512, OZ_MAX_R = 64;           // limits of the staged term lists
// CRT by a weighted sum: X = sum_q r_q c_q (mod P), c_q = (P/p_q) ((P/p_q)^-1 mod p_q)
// mod P, held as eight 16-bit limbs so every limb sum fits an int32.
// Tables for every moduli count n <= 16 (P = product of the first n moduli),
// so plans with different counts can run concurrently.
constexpr int OZ_CRT_MAX = 16;
__constant__ int c_crt16[OZ_CRT_MAX + 1][OZ_CRT_MAX][8];
__constant__ int c_P16[OZ_CRT_MAX + 1][8];                  // 16-bit limbs of P
__constant__ float c_fw[OZ_CRT_MAX + 1][8];                 // 2^(16 l) / P (0 where negligible)
__constant__ unsigned long long c_P[OZ_CRT_MAX + 1][2];     // P (lo, hi)
__constant__ unsigned long long c_Phalf[OZ_CRT_MAX + 1][2]; // P div 2
__constant__ unsigned long long c_Plow[OZ_CRT_MAX + 1][2];  // P div 2 - P

// x mod p for any 32-bit x: quotient estimate from floor(2^32/p) is at most
// one short, so one conditional subtraction finishes it.
__device__ __forceinline__ unsigned mod_u32(unsigned x, int q) {
    const unsigned p = (unsigned)c_mod[q];
    unsigned r = x - __umulhi(x, c_magic[q]) * p;
    return r >= p ? r - p : r;
}

using namespace tc;

// Balanced residue modulo moduli[q] of |x| < 2^20 (combinations of a few
// residues): shift positive by p * 2^13, then one Barrett reduction.
__device__ __forceinline__ int bal_mod_q(int x, int q) {
    const int p = c_mod[q];
    const int r = (int)mod_u32((unsigned)(x + (p << 13)), q);
    return r >= (p + 1) / 2 ? r - p : r;
}

#include "residue_gemm.cuh"
#include "residue_gemm_fa.cuh"

// Exponent e with 2^e <= |x| < 2^(e+1) for normal x; subnormals go through
// frexp.
__device__ __forceinline__ int ilog2_abs(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int be = int((b >> 52) & 0x7ff);
    if (be != 0) return be - 1023;
    int e;
    frexp(x, &e);
    return e - 1;
}

// High word of |x| (sign cleared).  For normal x the largest of these has
// the exponent field of max |x|, so exponent maxima run on the integer pipe
// (FP64 max and abs would run on the FP64 pipe, 1/64 of the FP32 rate).
// Below 2^20 (exponent field 0) every entry seen was zero or subnormal.
__device__ __forceinline__ unsigned abs_hi(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }
constexpr unsigned OZ_NORMAL_HI = 0x00100000u;

// x * 2^s rounded to the nearest integer (ties away from zero), by shifting
// the significand (no FP64 ops).  With s = beta - 1 - floor(log2 max|x|) the
// result is at most 2^beta in magnitude.
__device__ __forceinline__ long long scaled_round(double x, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int be = int((b >> 52) & 0x7ff);
    const unsigned long long frac = b & ((1ull << 52) - 1);
    if (be == 0 && frac == 0) return 0;
    // a subnormal is frac 2^-1074: exponent field 1 without the implicit bit
    // (it matters where a whole row or column is subnormal)
    const unsigned long long mant = be ? (frac | (1ull << 52)) : frac;
    const int sh = 52 - ((be ? be : 1) - 1023) - s;   // value = mant * 2^-sh
    long long v;
    if (sh >= 54) v = 0;                       // mant < 2^53: value < 1/2
    else if (sh >= 1) v = (long long)((mant + (1ull << (sh - 1))) >> sh);
    else v = (long long)(mant << (-sh));       // an integer already (beta > 53 with short k)
    return (b >> 63) ? -v : v;
}

// Balanced residue of a beta-bit integer v modulo moduli[q], from its 32-bit
// halves: v = hi 2^32 + lo, so v mod p = (hi mod p)(2^32 mod p) + lo mod p.
__device__ __forceinline__ float residue_bf16(long long v, int q) {
    const unsigned long long u = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const int p = c_mod[q];
    int r = (int)mod_u32(mod_u32(hi, q) * c_r32[q] + mod_u32(lo, q), q);
    if (v < 0 && r != 0) r = p - r;
    return (float)(r >= (p + 1) / 2 ? r - p : r);
}

// Row exponents and residue planes of X (rows x cols per leaf), K-major.
// One warp per (leaf, row).  out[(leaf*nmod + q) * rows + row][0..kpad).
__global__ void split_rows_kernel(const double *X, int64_t ldx, int64_t leaf_stride, int64_t rows,
                                  int64_t cols, int64_t kpad, int64_t leaves, int beta, int nmod,
                                  __nv_bfloat16 *out, int *exps) {
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (gw >= leaves * rows) return;
    const int64_t leaf = gw / rows, row = gw % rows;
    const double *x = X + leaf * leaf_stride + row * ldx;
    double mx = 0.0;
    for (int64_t j = lane; j < cols; j += 32) mx = fmax(mx, fabs(x[j]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int s = (mx == 0.0) ? 0 : beta - 1 - ilog2_abs(mx);
    if (lane == 0) exps[leaf * rows + row] = s;
    for (int64_t j = lane; j < kpad; j += 32) {
        const long long v = j < cols ? scaled_round(x[j], s) : 0;
        for (int q = 0; q < nmod; ++q)
            out[((leaf * nmod + q) * rows + row) * kpad + j] = __float2bfloat16_rn(residue_bf16(v, q));
    }
}

// Residue planes of Y^T (cols x kpad per plane) through a 32x32 tile
// transpose in shared memory.  grid: (ceil(kpad/32), ceil(cols/32), leaves).
__global__ void split_cols_kernel(const double *Y, int64_t ldy, int64_t leaf_stride, int64_t rows,
                                  int64_t cols, int64_t kpad, int nmod, const int *exps,
                                  __nv_bfloat16 *out) {
    __shared__ long long tile[32][33];
    const int64_t leaf = blockIdx.z;
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const double *y = Y + leaf * leaf_stride;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + r, j = j0 + tx;
        long long v = 0;
        if (i < rows && j < cols) v = scaled_round(y[i * ldy + j], exps[leaf * cols + j]);
        tile[r][tx] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t j = j0 + r, i = i0 + tx;       // output row j (a column of Y), col i
        if (j >= cols || i >= kpad) continue;
        const long long v = tile[tx][r];
        for (int q = 0; q < nmod; ++q)
            out[((leaf * nmod + q) * cols + j) * kpad + i] = __float2bfloat16_rn(residue_bf16(v, q));
    }
}

// fl(X) 2^-e for an integer X = (hi, lo) (two's complement, |X| < 2^127):
// X rounded once to FP64 (round to nearest even, from its integer bits), then
// scaled exactly; only a result outside the normal range goes through ldexp
// (which then rounds once more, as ldexp of the rounded value does).
__device__ __forceinline__ double round_scale(long long hi_s, unsigned long long lo, int e) {
    const bool neg = hi_s < 0;
    unsigned long long uh = (unsigned long long)hi_s, ul = lo;
    if (neg) {
        ul = ~ul + 1ull;
        uh = ~uh + (ul == 0ull ? 1ull : 0ull);
    }
    if ((uh | ul) == 0ull) return 0.0;
    int nb;
    unsigned long long top;
    bool sticky;
    if (uh != 0ull) {
        const int lz = __clzll((long long)uh);
        nb = 128 - lz;
        top = lz ? (uh << lz) | (ul >> (64 - lz)) : uh;
        sticky = lz ? (ul << lz) != 0ull : ul != 0ull;   // the bits of ul below the window: its low 64 - lz
    } else {
        const int lz = __clzll((long long)ul);
        nb = 64 - lz;
        top = ul << lz;
        sticky = false;
    }
    // top: leading one at bit 63; 53 significant bits and 11 rounding bits
    unsigned long long m = top >> 11;
    const unsigned rb = (unsigned)(top & 0x7ffull);
    if (rb > 0x400u || (rb == 0x400u && (sticky || (m & 1ull)))) ++m;
    int E = nb - 1;
    if (m >> 53) { m >>= 1; ++E; }
    const unsigned long long frac = m & ((1ull << 52) - 1);
    const int be = E - e + 1023;
    if (be >= 1 && be <= 2046)   // sign, exponent and fraction assembled as bits (no FP64 op)
        return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)be << 52) | frac));
    const double d = ldexp(__longlong_as_double((long long)(((unsigned long long)(E + 1023) << 52) | frac)), -e);
    return neg ? -d : d;
}

// 16-bit limbs needed for P of n moduli (ceil(bits(P) / 16)); 8 for n = 0
// (a count known only at run time).
__host__ __device__ constexpr int crt_limbs(int n) { return n <= 0 ? 8 : (n <= 2 ? 1 : (n + 1) / 2); }

// Add residue r (|r| < 2^8, any representative) of modulus q of n to the limb
// sums (NL limbs: limbs of c_q above those of P are zero).
template <int NL>
__device__ __forceinline__ void crt_add(int (&L)[NL], int r, int q, int n) {
#pragma unroll
    for (int l = 0; l < NL; ++l) L[l] += r * c_crt16[n][q][l];
}

// The integer X in [P div 2 - P, P div 2) congruent to the residues summed in
// L, rounded once to FP64 and scaled by 2^-e.  S = sum_l L_l 2^(16 l); the
// quotient t = round(S / P) comes from a float estimate (off by at most one
// near a half-integer), X = S - t P exactly in limbs, then one correction.
// NL: limbs held; TIGHT: NL is exactly the limb count of P (n known at compile
// time), so only the top three limbs matter for the quotient (the others
// weigh below 2^-40 and their sums stay below 2^31); otherwise all are used.
template <int NL, bool TIGHT>
__device__ __forceinline__ double crt_finish(const int (&L)[NL], int e, int n) {
    float sf = 0.f;
#pragma unroll
    for (int l = (TIGHT && NL > 3 ? NL - 3 : 0); l < NL; ++l) sf = fmaf((float)L[l], c_fw[n][l], sf);
    // t = rint(sf) (|sf| < 2^22); xf estimates X / P to within 2^-10
    const float sm = sf + 12582912.0f;
    const int t = __float_as_int(sm) - 0x4B400000;
    const float xf = sf - (sm - 12582912.0f);
    // X = S - t P in NL limbs; carries leave limbs 0..NL-2 in [0, 2^16) and
    // the sign in the top limb, which then sign-extends into (hi, lo)
    int x[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) x[l] = L[l] - t * c_P16[n][l];
#pragma unroll
    for (int l = 0; l < NL - 1; ++l) {
        const int carry = x[l] >> 16;
        x[l] -= carry * 65536;
        x[l + 1] += carry;
    }
    unsigned long long lo = 0ull;
    long long hi;
    if constexpr (NL <= 4) {
#pragma unroll
        for (int l = 0; l < NL - 1; ++l) lo |= (unsigned long long)(unsigned)x[l] << (16 * l);
        const long long top = (long long)x[NL - 1] * (1ll << (16 * (NL - 1)));
        lo = (unsigned long long)((long long)lo + top);
        hi = (long long)lo >> 63;
    } else {
#pragma unroll
        for (int l = 0; l < 4; ++l) lo |= (unsigned long long)(unsigned)x[l] << (16 * l);
        unsigned long long h = 0ull;
#pragma unroll
        for (int l = 4; l < NL - 1; ++l) h |= (unsigned long long)(unsigned)x[l] << (16 * (l - 4));
        hi = (long long)h + (long long)x[NL - 1] * (1ll << (16 * (NL - 5)));
    }
    if (fabsf(xf) > 0.49f) {
        // near +-P/2 the estimate may have picked the neighbouring multiple of P
        __int128 X = (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
        const __int128 P = (__int128)(((unsigned __int128)c_P[n][1] << 64) | c_P[n][0]);
        const __int128 Ph = (__int128)(((unsigned __int128)c_Phalf[n][1] << 64) | c_Phalf[n][0]);
        const __int128 Pl = (__int128)(((unsigned __int128)c_Plow[n][1] << 64) | c_Plow[n][0]);
        if (X >= Ph) X -= P;
        else if (X < Pl) X += P;
        lo = (unsigned long long)X;
        hi = (long long)((unsigned __int128)X >> 64);
    }
    return round_scale(hi, lo, e);
}

// C[leaf][i][j] (+)= (Z from its residues) * 2^-(sa_i + sb_j), the leaf
// products of the per-leaf emulation.  V consecutive columns per thread.
template <int V>
__global__ void crt_kernel(const int8_t *Z, int64_t m, int64_t n, int64_t ldz, int64_t leaves, int nmod,
                           const int *sa, const int *sb, double *C, int64_t ldc, int64_t leaf_stride,
                           int accumulate) {
    const int64_t plane = m * ldz;
    const int64_t total = leaves * m * n / V;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = g * V;
        const int64_t leaf = e0 / (m * n), rem0 = e0 % (m * n), i = rem0 / n, j = rem0 % n;
        const int64_t rem = i * ldz + j;
        int L[V][8];
#pragma unroll
        for (int e = 0; e < V; ++e)
#pragma unroll
            for (int l = 0; l < 8; ++l) L[e][l] = 0;
        const int8_t *z = Z + leaf * nmod * plane + rem;
        for (int q = 0; q < nmod; ++q) {
            int r[V];
            if (V == 4) {
                const int raw = *reinterpret_cast<const int *>(z + (int64_t)q * plane);
#pragma unroll
                for (int e = 0; e < V; ++e) r[e] = (int)(int8_t)(raw >> (8 * e));
            } else {
                r[0] = z[(int64_t)q * plane];
            }
#pragma unroll
            for (int e = 0; e < V; ++e) crt_add(L[e], r[e], q, nmod);
        }
        double *out = C + leaf * leaf_stride + i * ldc + j;
        const int ei = sa[leaf * m + i];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const double val = crt_finish<8, false>(L[e], ei + sb[leaf * n + j + e], nmod);
            out[e] = accumulate ? out[e] + val : val;
        }
    }
}

// ---------------------------------------------------------------------
// Residue-space recursion: with integer coefficients the bilinear algorithm
// is exact over Z/pZ, so S/T formation, the leaf products and the W
// combination all run on residues of the once-scaled A' and B'; one CRT
// rebuilds C' = A'B' (the same integer the classical emulation computes).
// Buffers are laid out [matrix][modulus][rows][cols], int8 balanced.

// int8 residues of X (rows x cols, ld) scaled by per-row exponents (found
// here, one warp per row) -> out[q][row][col].
__global__ void split_rows_i8(const double *X, int64_t ldx, int64_t rows, int64_t cols, int beta,
                              int nmod, int8_t *out, int *exps) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (row >= rows) return;
    const double *x = X + row * ldx;
    double mx = 0.0;
    for (int64_t j = lane; j < cols; j += 32) mx = fmax(mx, fabs(x[j]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int s = (mx == 0.0) ? 0 : beta - 1 - ilog2_abs(mx);
    if (lane == 0) exps[row] = s;
    for (int64_t j = lane; j < cols; j += 32) {
        const long long v = scaled_round(x[j], s);
        for (int q = 0; q < nmod; ++q)
            out[((int64_t)q * rows + row) * cols + j] = (int8_t)residue_bf16(v, q);
    }
}

// int8 residues of Y^T: Y (rows x cols, ld) scaled by per-column exponents,
// written out[q][col][row] through a 32x32 tile.  grid (ceil(rows/32),
// ceil(cols/32)), block (32, 8).
__global__ void split_cols_t_i8(const double *Y, int64_t ldy, int64_t rows, int64_t cols, int nmod,
                                const int *exps, int8_t *out) {
    __shared__ long long tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + r, j = j0 + tx;
        tile[r][tx] = (i < rows && j < cols) ? scaled_round(Y[i * ldy + j], exps[j]) : 0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t j = j0 + r, i = i0 + tx;
        if (j >= cols || i >= rows) continue;
        const long long v = tile[tx][r];
        for (int q = 0; q < nmod; ++q) out[((int64_t)q * cols + j) * rows + i] = (int8_t)residue_bf16(v, q);
    }
}

// Column exponents with many threads per column: blockDim.x columns x 8 row
// groups, reduced through shared memory.
// grid (ceil(cols/32), leaves); leaf l reads Y + l * leaf_stride.
constexpr int COL_EXP_ROWS = 32;
__global__ void __launch_bounds__(32 * COL_EXP_ROWS) col_exp_wide(const double *Y, int64_t ldy, int64_t leaf_stride, int64_t rows,
                             int64_t cols, int beta, int *exps) {
    // blockDim (32, COL_EXP_ROWS): one column per lane, the rows strided over the warps
    __shared__ unsigned parth[COL_EXP_ROWS][32], partl[COL_EXP_ROWS][32];
    __shared__ double partd[COL_EXP_ROWS][32];
    const int64_t leaf = blockIdx.y;
    const int64_t col = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const double *y = Y + leaf * leaf_stride;
    unsigned mh = 0u, lo = 0u;   // max of the high words of |y|, OR of the low words
    if (col < cols) {
#pragma unroll 4
        for (int64_t i = threadIdx.y; i < rows; i += COL_EXP_ROWS) {
            const double v = y[i * ldy + col];
            mh = max(mh, abs_hi(v));
            lo |= (unsigned)__double2loint(v);
        }
    }
    parth[threadIdx.y][threadIdx.x] = mh;
    partl[threadIdx.y][threadIdx.x] = lo;
    __syncthreads();
    if (threadIdx.y == 0)
        for (int r = 1; r < COL_EXP_ROWS; ++r) {
            mh = max(mh, parth[r][threadIdx.x]);
            lo |= partl[r][threadIdx.x];
        }
    // a column whose largest entry is subnormal: its exact maximum in FP64 (rare)
    const bool sub = threadIdx.y == 0 && col < cols && mh < OZ_NORMAL_HI && (mh | lo) != 0u;
    if (__syncthreads_or(sub)) {
        double mx = 0.0;
        if (col < cols)
            for (int64_t i = threadIdx.y; i < rows; i += COL_EXP_ROWS) mx = fmax(mx, fabs(y[i * ldy + col]));
        partd[threadIdx.y][threadIdx.x] = mx;
        __syncthreads();
        if (sub) {
            for (int r = 1; r < COL_EXP_ROWS; ++r) mx = fmax(mx, partd[r][threadIdx.x]);
            exps[leaf * cols + col] = (mx == 0.0) ? 0 : beta - 1 - ilog2_abs(mx);
        }
    }
    if (threadIdx.y == 0 && col < cols && !sub)
        exps[leaf * cols + col] = (mh | lo) == 0u ? 0 : beta - 1 - (int(mh >> 20) - 1023);
}

// One recursive level in residue space: child o = s*R + r, modulus q:
// sum_t c_t (parent s, block t) mod p.  FINAL writes bfloat16 rows padded to
// out_ld (K-major operand of the residue GEMM), otherwise int8 rows.  VEC:
// eight consecutive columns per thread with 8-byte loads (cols, pc and out_ld
// multiples of 8).
template <bool FINAL, bool VEC>
__global__ void res_form_kernel(const int8_t *parent, int64_t pr, int64_t pc, int64_t rows,
                                int64_t cols, int R, int nmod, int64_t o_base, const int *ptr,
                                const int *code, const int *icoef, void *out, int64_t out_ld) {
    const int64_t o = o_base + blockIdx.y;
    const int64_t sp = o / R;
    const int r = int(o % R);
    const int q = blockIdx.z;
    const int8_t *P = parent + (sp * nmod + q) * pr * pc;
    const int t0 = ptr[r], t1 = ptr[r + 1];
    const int64_t plane = (o * nmod + q) * rows * out_ld;
    constexpr int W = VEC ? 8 : 1;
    for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
        for (int64_t j = (int64_t)threadIdx.x * W; j < out_ld; j += (int64_t)blockDim.x * W) {
            int v[W];
#pragma unroll
            for (int e = 0; e < W; ++e) v[e] = 0;
            if (j < cols) {
                for (int t = t0; t < t1; ++t) {
                    const int cd = code[t];
                    const int c = icoef[t];
                    const int8_t *src = P + ((int64_t)(cd >> 16) * rows + i) * pc + (int64_t)(cd & 0xffff) * cols + j;
                    if (VEC) {
                        const uint2 raw = *reinterpret_cast<const uint2 *>(src);
                        const int8_t *bytes = reinterpret_cast<const int8_t *>(&raw);
#pragma unroll
                        for (int e = 0; e < W; ++e) v[e] += c * (int)bytes[e];
                    } else {
                        v[0] += c * (int)src[0];
                    }
                }
            }
            if (FINAL) {
                __nv_bfloat16 *dst = (__nv_bfloat16 *)out + plane + i * out_ld + j;
                if (VEC) {
                    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) h[e] = __float2bfloat16_rn((float)bal_mod_q(v[e], q));
                    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(h);
                } else {
                    dst[0] = __float2bfloat16_rn((float)bal_mod_q(v[0], q));
                }
            } else {
                int8_t *dst = (int8_t *)out + plane + i * out_ld + j;
                if (VEC) {
                    __align__(8) int8_t h[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) h[e] = (int8_t)bal_mod_q(v[e], q);
                    *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(h);
                } else {
                    dst[0] = (int8_t)bal_mod_q(v[0], q);
                }
            }
        }
    }
}

// One level of the W combination in residue space: parent s, block qb of
// its M x N grid, modulus q = sum_t w_t child_{s*R + r_t} mod p.  VEC: eight
// columns per thread (cols a multiple of 8).
template <bool VEC>
__global__ void res_w_kernel(const int8_t *child, int64_t rows, int64_t cols, int64_t cld, int R, int gridN,
                             int MN, int nmod, int8_t *parent, int64_t o_base, const int *w_ptr,
                             const int *w_r, const int *w_icoef) {
    const int64_t o = o_base + blockIdx.y;
    const int64_t sp = o / MN;
    const int qb = int(o % MN);
    const int a = qb / gridN, c = qb % gridN;
    const int q = blockIdx.z;
    const int64_t prow = rows * (MN / gridN), pcol = cols * gridN;
    int8_t *Pout = parent + (sp * nmod + q) * prow * pcol + (int64_t)a * rows * pcol + (int64_t)c * cols;
    const int t0 = w_ptr[qb], t1 = w_ptr[qb + 1];
    constexpr int W = VEC ? 8 : 1;
    for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
        for (int64_t j = (int64_t)threadIdx.x * W; j < cols; j += (int64_t)blockDim.x * W) {
            int v[W];
#pragma unroll
            for (int e = 0; e < W; ++e) v[e] = 0;
            for (int t = t0; t < t1; ++t) {
                const int wc = w_icoef[t];
                const int8_t *src = child + (((sp * R + w_r[t]) * nmod + q) * rows + i) * cld + j;
                if (VEC) {
                    const uint2 raw = *reinterpret_cast<const uint2 *>(src);
                    const int8_t *bytes = reinterpret_cast<const int8_t *>(&raw);
#pragma unroll
                    for (int e = 0; e < W; ++e) v[e] += wc * (int)bytes[e];
                } else {
                    v[0] += wc * (int)src[0];
                }
            }
            if (VEC) {
                __align__(8) int8_t h[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) h[e] = (int8_t)bal_mod_q(v[e], q);
                *reinterpret_cast<uint2 *>(Pout + i * pcol + j) = *reinterpret_cast<const uint2 *>(h);
            } else {
                Pout[i * pcol + j] = (int8_t)bal_mod_q(v[0], q);
            }
        }
    }
}

// ---------------------------------------------------------------------
// Fused first level: the scaling of A (or B), the residues and the first
// recursive level's combinations in one pass over the FP64 operand, so the
// level-0 residue planes never reach HBM.  With L = 0 the "first level" is the
// identity (one block, one child, coefficient 1) and the pass writes the GEMM
// operand planes directly.

// Balanced residue of a small combination |x| < 2^29.
__device__ __forceinline__ int bal_small(int x, int q) {
    const int p = c_mod[q];
    const int r = (int)mod_u32((unsigned)(x + (p << 22)), q);
    return r >= (p + 1) / 2 ? r - p : r;
}

// Integer-valued floats: x = float(1.5 2^23 + x) - 1.5 2^23 exactly for |x| < 2^22.
constexpr float OZ_FMAGIC = 12582912.0f;
constexpr int OZ_IMAGIC = 0x4B400000;

// One child of the first level: S' = sum_t c_t X'_t over the thread's NB
// block values (int64 in shared memory, [b][e][thread], 4 consecutive
// entries e), exact in int64 (host-checked: 2^beta sum |c_t| < 2^63); then
// per modulus q the residue from 13-bit limbs of |S'|,
//   x = sum_i d_i (2^(13 i) mod p)   (|x| < 2^23.3, exact in float),
// reduced to its nearest representative (|r| <= p/2 + 1) and written to
// dst + q qstep as bfloat16 (FINAL, the GEMM operand; |r| <= 129 is exact and
// keeps the GEMM's 512-long FP32 chunks exact) or int8 (a later level's input;
// representatives that wrap stay in the same class: only p = 256 reaches 128).
template <bool FINAL, int LB, int NLB, bool F16 = false, int LB0 = LB>
__device__ __forceinline__ void emit_child(const long long *sv, const int2 *sterm, int t0, int t1, int nmod,
                                           char *dst, int64_t qstep, int valid) {
    // Uniform layouts: NLB limbs of LB bits (|S'| < 2^(LB NLB), host-checked),
    // weights 2^(LB i) mod p in [0, p): the weighted sum stays below
    // NLB 2^LB 2^8 <= 2^24, exact in float.  The wide layout (LB0 = 22):
    // limbs of 22, 15 and 15 bits (|S'| < 2^52) with balanced weights
    // (|w| <= 128), so |x| < 2^22 + 2 2^15 2^7 = 1.5 2^23, exact too, with one
    // multiply-add fewer per residue than four 14-bit limbs.
    static_assert((LB0 == LB && (LB == 13 || LB == 14)) || (LB0 == 22 && LB == 15 && NLB == 3), "limb layout");
    long long S[4] = {0, 0, 0, 0};
    for (int t = t0; t < t1; ++t) {
        const int2 tm = sterm[t];
        const long long *src = sv + tm.x * 4 * 256 + threadIdx.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) S[e] += (long long)tm.y * src[e * 256];
    }
    float d[4][NLB];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const bool neg = S[e] < 0;
        const unsigned long long u = neg ? (unsigned long long)(-S[e]) : (unsigned long long)S[e];
#pragma unroll
        for (int i = 0; i < NLB; ++i) {
            const int sh = i == 0 ? 0 : LB0 + LB * (i - 1), wd = i == 0 ? LB0 : LB;
            const float f = __int_as_float(OZ_IMAGIC + (int)((u >> sh) & ((1ull << wd) - 1))) - OZ_FMAGIC;
            d[e][i] = neg ? -f : f;
        }
    }
#pragma unroll
    for (int q = 0; q < OZ_CRT_MAX; ++q) {
        if (q >= nmod) break;
        float r[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float x = d[e][0];
#pragma unroll
            for (int i = 1; i < NLB; ++i)
                x = fmaf(d[e][i], LB0 == LB ? c_klimb[LB - 13 < 0 ? 0 : (LB - 13 > 1 ? 1 : LB - 13)][q][i]
                                            : c_klimbw[q][i < 3 ? i : 2], x);
            const float tq = fmaf(x, c_invp[q], OZ_FMAGIC) - OZ_FMAGIC;
            r[e] = fmaf(-tq, c_modf[q], x);
        }
        char *out = dst + q * qstep;
        if (FINAL) {
            // small integers: bfloat16 is the top half of their FP32 bits; half
            // precision by conversion (exact below 2^11)
            uint2 pk;
            if (F16) {
                const __half2 h01 = __floats2half2_rn(r[0], r[1]), h23 = __floats2half2_rn(r[2], r[3]);
                pk.x = *reinterpret_cast<const unsigned *>(&h01);
                pk.y = *reinterpret_cast<const unsigned *>(&h23);
            } else {
                pk.x = __byte_perm(__float_as_uint(r[0]), __float_as_uint(r[1]), 0x7632);
                pk.y = __byte_perm(__float_as_uint(r[2]), __float_as_uint(r[3]), 0x7632);
            }
            if (valid == 4) {
                *reinterpret_cast<uint2 *>(out) = pk;
            } else {
                const unsigned short *h = reinterpret_cast<const unsigned short *>(&pk);
                for (int e = 0; e < valid; ++e) reinterpret_cast<unsigned short *>(out)[e] = h[e];
            }
        } else {
            unsigned word = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                word |= ((unsigned)(__float_as_int(r[e] + OZ_FMAGIC) - OZ_IMAGIC) & 0xffu) << (8 * e);
            if (valid == 4 && ((uintptr_t)out & 3) == 0) {
                *reinterpret_cast<unsigned *>(out) = word;
            } else {
                for (int e = 0; e < valid; ++e) reinterpret_cast<int8_t *>(out)[e] = (int8_t)(word >> (8 * e));
            }
        }
    }
}

// Stage one level's term lists in shared memory: sterm[t] = (block index,
// integer coefficient), sptr[o] = CSR over the children.
__device__ __forceinline__ void stage_terms(int R, int gridC, const int *ptr, const int *code, const int *icoef,
                                            int2 *sterm, int *sptr) {
    const int nterms = __ldg(ptr + R);
    for (int t = threadIdx.x; t < nterms; t += blockDim.x) {
        const int cd = __ldg(code + t);
        sterm[t] = make_int2((cd >> 16) * gridC + (cd & 0xffff), __ldg(icoef + t));
    }
    for (int o = threadIdx.x; o <= R; o += blockDim.x) sptr[o] = __ldg(ptr + o);
}

// S side: A (peeled core, ld lda) as a grid of M x K blocks of rows x cols;
// A' = round(A_ij 2^ea_i).  Thread: one row of the child blocks and 4
// consecutive columns of out_ld (columns >= cols are the zero padding of the
// GEMM operand).  256 threads; dynamic shared memory NB x 4 x 256 int64.
// Limb layouts of the combined integers: LC 0 = 3 x 14 bits, 1 = 4 x 14, 2 = 5 x 13,
// 3 = 22 + 15 + 15 (balanced weights).
template <int LC> struct LimbCfg;
template <> struct LimbCfg<0> { static constexpr int LB = 14, N = 3, LB0 = 14; };
template <> struct LimbCfg<1> { static constexpr int LB = 14, N = 4, LB0 = 14; };
template <> struct LimbCfg<2> { static constexpr int LB = 13, N = 5, LB0 = 13; };
template <> struct LimbCfg<3> { static constexpr int LB = 15, N = 3, LB0 = 22; };   // 22 + 15 + 15 bits

template <int NB, bool FINAL, int LC>
__global__ void __launch_bounds__(256) split_form_rows(const double *A, int64_t lda, const int *ea, int64_t rows,
                                                       int64_t cols, int gridK, int R, int nmod, const int *ptr,
                                                       const int *code, const int *icoef, void *out,
                                                       int64_t out_ld, int64_t r0, int64_t nr) {
    extern __shared__ long long sv[];   // [NB][4][256]
    __shared__ int2 sterm[OZ_MAX_TERMS];
    __shared__ int sptr[OZ_MAX_R + 1];
    stage_terms(R, gridK, ptr, code, icoef, sterm, sptr);
    __syncthreads();
    // the child rows [r0, r0 + nr) (all of them: r0 = 0, nr = rows)
    const int64_t groups = (out_ld + 3) / 4;
    const int64_t pos = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (pos >= nr * groups) return;
    const int64_t i = r0 + pos / groups, j0 = (pos % groups) * 4;
    const int valid = (int)min((int64_t)4, out_ld - j0);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int64_t row = (int64_t)(b / gridK) * rows + i;
        const int s = ea[row];
        const double *x = A + row * lda + (int64_t)(b % gridK) * cols + j0;
        if (j0 + 4 <= cols && ((uintptr_t)x & 15) == 0) {
            const double2 v0 = reinterpret_cast<const double2 *>(x)[0], v1 = reinterpret_cast<const double2 *>(x)[1];
            sv[(b * 4 + 0) * 256 + threadIdx.x] = scaled_round(v0.x, s);
            sv[(b * 4 + 1) * 256 + threadIdx.x] = scaled_round(v0.y, s);
            sv[(b * 4 + 2) * 256 + threadIdx.x] = scaled_round(v1.x, s);
            sv[(b * 4 + 3) * 256 + threadIdx.x] = scaled_round(v1.y, s);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) sv[(b * 4 + e) * 256 + threadIdx.x] = (j0 + e < cols) ? scaled_round(x[e], s) : 0;
        }
    }
    constexpr int ES = FINAL ? 2 : 1;   // bytes per output entry
    const int64_t plane = rows * out_ld;
    char *dst = (char *)out + (i * out_ld + j0) * ES;
    const int64_t qstep = plane * ES, ostep = (int64_t)nmod * plane * ES;
    for (int o = 0; o < R; ++o, dst += ostep)
        emit_child<FINAL, LimbCfg<LC>::LB, LimbCfg<LC>::N, false, LimbCfg<LC>::LB0>(sv, sterm, sptr[o], sptr[o + 1],
                                                                                  nmod, dst, qstep, valid);
}

// T side, transposed: B (peeled core, ld ldb) as a grid of K x N blocks of
// krows x ncols; B' = round(B_ij 2^eb_j).  Output rows are columns of B
// (T^T, K-major for the GEMM).  CTA: 32 k x 32 n positions of the child
// blocks through shared memory (dynamic: NB x 32 x 33 int64, then reused as
// [NB][4][256]); thread: one n and 4 consecutive k.  grid (ceil(out_ld / 32),
// ceil(ncols / 32)), 256 threads.
template <int NB, bool FINAL, int LC, bool F16 = false>
__global__ void __launch_bounds__(256) split_form_cols_t(const double *B, int64_t ldb, const int *eb, int64_t krows,
                                                         int64_t ncols, int gridN, int R, int nmod, const int *ptr,
                                                         const int *code, const int *icoef, void *out,
                                                         int64_t out_ld) {
    extern __shared__ long long sv[];
    __shared__ int2 sterm[OZ_MAX_TERMS];
    __shared__ int sptr[OZ_MAX_R + 1];
    stage_terms(R, gridN, ptr, code, icoef, sterm, sptr);
    const int64_t k0 = (int64_t)blockIdx.x * 32, n0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int64_t bk = b / gridN, bn = b % gridN;
        const int64_t n = n0 + tx;
        const int s = n < ncols ? eb[bn * ncols + n] : 0;
        for (int r = ty; r < 32; r += 8) {
            const int64_t k = k0 + r;
            sv[(b * 32 + r) * 33 + tx] =
                (k < krows && n < ncols) ? scaled_round(B[(bk * krows + k) * ldb + bn * ncols + n], s) : 0;
        }
    }
    __syncthreads();
    const int nn = threadIdx.x / 8, kk = (threadIdx.x % 8) * 4;
    long long v[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int e = 0; e < 4; ++e) v[b][e] = sv[(b * 32 + kk + e) * 33 + nn];
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int e = 0; e < 4; ++e) sv[(b * 4 + e) * 256 + threadIdx.x] = v[b][e];
    const int64_t n = n0 + nn, k = k0 + kk;
    if (n >= ncols || k >= out_ld) return;
    const int valid = FINAL ? 4 : (int)min((int64_t)4, krows - k);
    constexpr int ES = FINAL ? 2 : 1;
    const int64_t plane = ncols * out_ld;
    char *dst = (char *)out + (n * out_ld + k) * ES;
    const int64_t qstep = plane * ES, ostep = (int64_t)nmod * plane * ES;
    for (int o = 0; o < R; ++o, dst += ostep)
        emit_child<FINAL, LimbCfg<LC>::LB, LimbCfg<LC>::N, F16, LimbCfg<LC>::LB0>(sv, sterm, sptr[o], sptr[o + 1], nmod, dst, qstep,
                                                                valid);
}

// ---------------------------------------------------------------------
// Streaming levels (levels >= 2 of S and T, int8 residues in HBM): each
// parent element is read once and every child that uses it is written from
// the same thread (Section 3.2's streaming additions, one level at a time).

// 8 signed bytes of w (little-endian), e-th.
__device__ __forceinline__ int sbyte8(uint2 w, int e) {
    return (int)(int8_t)((e < 4 ? w.x : w.y) >> (8 * (e & 3)));
}

// Nearest representative modulo moduli[q] of a small integer |x| < 2^22.
__device__ __forceinline__ float near_mod_i(int x, int q) {
    const float f = __int_as_float(OZ_IMAGIC + x) - OZ_FMAGIC;
    const float t = fmaf(f, c_invp[q], OZ_FMAGIC) - OZ_FMAGIC;
    return fmaf(-t, c_modf[q], f);
}

// One level of S (or T^T): parent planes P[s][q] (prow x pcol int8) as a grid
// of gridR x gridC blocks of rows x cols; child o = s R + r, modulus q:
// sum_t c_t block(t) mod p, written to out[(o nmod + q)][rows][out_ld] as
// bfloat16 (FINAL) or int8.  Thread: (s, q, row i, 8 columns); 256 threads.
template <int NB, bool FINAL, bool ALIGNED>
__global__ void __launch_bounds__(256) res_stream_form(const int8_t *P, int64_t prow, int64_t pcol, int64_t rows,
                                                       int64_t cols, int gridC, int R, int nmod, int64_t parents,
                                                       const int *ptr, const int *code, const int *icoef, void *out,
                                                       int64_t out_ld) {
    __shared__ uint2 sres[NB * 256];
    __shared__ int2 sterm[OZ_MAX_TERMS];
    __shared__ int sptr[OZ_MAX_R + 1];
    stage_terms(R, gridC, ptr, code, icoef, sterm, sptr);
    __syncthreads();
    const int64_t groups = (out_ld + 7) / 8;
    const int64_t pos = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (pos >= parents * nmod * rows * groups) return;
    const int64_t jg = pos % groups;
    int64_t rest = pos / groups;
    const int64_t i = rest % rows;
    rest /= rows;
    const int q = (int)(rest % nmod);
    const int64_t sp = rest / nmod;
    const int64_t j0 = jg * 8;
    const int8_t *base = P + (sp * nmod + q) * prow * pcol;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int8_t *src = base + ((int64_t)(b / gridC) * rows + i) * pcol + (int64_t)(b % gridC) * cols + j0;
        uint2 w;
        if (ALIGNED && j0 + 8 <= cols) {
            w = *reinterpret_cast<const uint2 *>(src);
        } else {
            unsigned lo = 0, hi = 0;
            for (int e = 0; e < 8; ++e) {
                const unsigned v = (j0 + e < cols) ? (unsigned)(uint8_t)src[e] : 0u;
                if (e < 4) lo |= v << (8 * e); else hi |= v << (8 * (e - 4));
            }
            w = make_uint2(lo, hi);
        }
        sres[b * 256 + threadIdx.x] = w;
    }
    const int valid = (int)min((int64_t)8, out_ld - j0);
    constexpr int ES = FINAL ? 2 : 1;
    char *dst = (char *)out + ((((sp * R) * nmod + q) * rows + i) * out_ld + j0) * ES;
    const int64_t ostep = (int64_t)nmod * rows * out_ld * ES;
    for (int r = 0; r < R; ++r, dst += ostep) {
        int acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const int t1 = sptr[r + 1];
        for (int t = sptr[r]; t < t1; ++t) {
            const int2 tm = sterm[t];
            const uint2 w = sres[tm.x * 256 + threadIdx.x];
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[e] += tm.y * sbyte8(w, e);
        }
        float rr[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) rr[e] = near_mod_i(acc[e], q);
        if (FINAL) {
            uint4 pk;
            pk.x = __byte_perm(__float_as_uint(rr[0]), __float_as_uint(rr[1]), 0x7632);
            pk.y = __byte_perm(__float_as_uint(rr[2]), __float_as_uint(rr[3]), 0x7632);
            pk.z = __byte_perm(__float_as_uint(rr[4]), __float_as_uint(rr[5]), 0x7632);
            pk.w = __byte_perm(__float_as_uint(rr[6]), __float_as_uint(rr[7]), 0x7632);
            if (valid == 8) {
                *reinterpret_cast<uint4 *>(dst) = pk;
            } else {
                const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&pk);
                for (int e = 0; e < valid; ++e) reinterpret_cast<__nv_bfloat16 *>(dst)[e] = h[e];
            }
        } else {
            unsigned lo = 0, hi = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const unsigned v = (unsigned)(__float_as_int(rr[e] + OZ_FMAGIC) - OZ_IMAGIC) & 0xffu;
                if (e < 4) lo |= v << (8 * e); else hi |= v << (8 * (e - 4));
            }
            if (ALIGNED && valid == 8) {
                *reinterpret_cast<uint2 *>(dst) = make_uint2(lo, hi);
            } else {
                for (int e = 0; e < valid; ++e)
                    reinterpret_cast<int8_t *>(dst)[e] = (int8_t)((e < 4 ? lo : hi) >> (8 * (e & 3)));
            }
        }
    }
}

// Top recursion level of the W combination fused with the CRT: output block
// qb = (a, c) of the M x N grid, modulus q: Z_qb = sum_t w_t child(r_t) mod p;
// C'_qb from its residues, times 2^-(ea_i + eb_j), stored (or added) in C.
// With L = 0 the one child is the product itself.  Thread: one row of the
// child blocks, V consecutive columns.  A launch covers the child rows
// [r0, r0 + nr) of every block (rows tall); Z points at the first of them in
// plane 0, and the planes are zr rows apart.
template <int V, bool REDUCE, int NMOD>
__global__ void __launch_bounds__(256, 4) w_crt_kernel(const int8_t *Z, int64_t rows, int64_t cols, int64_t cld,
                                                    int64_t zr, int64_t r0, int64_t nr, int gridN, int MN, int nmod_rt, const int *w_ptr, const int *w_r,
                                                    const int *w_icoef, const int *ea, const int *eb, double *C,
                                                    int64_t ldc, int accumulate) {
    // NMOD > 0: the moduli count is a compile-time constant (loops unrolled,
    // CRT constants as immediate operands, only the limbs P needs)
    const int nmod = NMOD ? NMOD : nmod_rt;
    constexpr int NL = crt_limbs(NMOD);
    __shared__ int2 swt[OZ_MAX_TERMS];   // (child r, coefficient)
    __shared__ int swp[OZ_MAX_R + 1];
    __shared__ int swsum[OZ_MAX_R];      // sum of the coefficients of each block
    {
        const int nterms = __ldg(w_ptr + MN);
        for (int t = threadIdx.x; t < nterms; t += blockDim.x) swt[t] = make_int2(__ldg(w_r + t), __ldg(w_icoef + t));
        for (int o = threadIdx.x; o <= MN; o += blockDim.x) swp[o] = __ldg(w_ptr + o);
        for (int o = threadIdx.x; o < MN; o += blockDim.x) {
            int sum = 0;
            for (int t = __ldg(w_ptr + o); t < __ldg(w_ptr + o + 1); ++t) sum += __ldg(w_icoef + t);
            swsum[o] = sum;
        }
    }
    __syncthreads();
    const int64_t groups = (cols + V - 1) / V;
    const int64_t pos = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (pos >= nr * groups) return;
    const int64_t il = pos / groups, i = r0 + il, j0 = (pos % groups) * V;
    const int valid = (int)min((int64_t)V, cols - j0);
    const int64_t plane = zr * cld;
    const int8_t *zrow = Z + il * cld + j0;
    for (int qb = 0; qb < MN; ++qb) {
        const int a = qb / gridN, c = qb % gridN;
        int L[V][NL];
#pragma unroll
        for (int e = 0; e < V; ++e)
#pragma unroll
            for (int l = 0; l < NL; ++l) L[e][l] = 0;
        const int t0 = swp[qb], t1 = swp[qb + 1];
        if (NMOD > 0 && V == 4) {
            // All moduli of a term loaded together, then combined two columns
            // to a 32-bit word: the bytes b (in [-128, 127]) are read offset
            // as u = b + 128 and paired as u_0 + 2^16 u_1, so one multiply-add
            // does two columns and, the map being linear, the word ends as
            // sum w b_0 + 2^16 sum w b_1 once the offsets (128 sum w per
            // column) are taken off up front.  Both sums lie within 128 sum|w|
            // <= 2^15 (host-checked), so the two halves separate exactly
            // (intermediate wrap-around modulo 2^32 cancels).
            constexpr int NQ = NMOD > 0 ? NMOD : 1;
            const unsigned bias = 0u - 128u * (unsigned)swsum[qb] * 65537u;
            unsigned acc[NQ][2];
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q][0] = acc[q][1] = bias;
            for (int t = t0; t < t1; ++t) {
                const int2 wt = swt[t];
                const int8_t *z = zrow + (int64_t)wt.x * NQ * plane;
                unsigned raw[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) raw[q] = *reinterpret_cast<const unsigned *>(z + q * plane);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const unsigned u = raw[q] ^ 0x80808080u;
                    acc[q][0] += (unsigned)wt.y * __byte_perm(u, 0u, 0x4140);
                    acc[q][1] += (unsigned)wt.y * __byte_perm(u, 0u, 0x4342);
                }
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int lo = (int)(short)acc[q][h];
                    const int hi = ((int)acc[q][h] - lo) >> 16;
                    crt_add(L[2 * h], REDUCE ? bal_small(lo, q) : lo, q, NQ);
                    crt_add(L[2 * h + 1], REDUCE ? bal_small(hi, q) : hi, q, NQ);
                }
        } else {
#pragma unroll 4
            for (int q = 0; q < nmod; ++q) {
                int acc[V];
#pragma unroll
                for (int e = 0; e < V; ++e) acc[e] = 0;
                for (int t = t0; t < t1; ++t) {
                    const int2 wt = swt[t];
                    const int8_t *z = zrow + ((int64_t)wt.x * nmod + q) * plane;
                    if (V == 4) {
                        const unsigned raw = *reinterpret_cast<const unsigned *>(z);
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[e] += wt.y * (int)(int8_t)(raw >> (8 * e));
                    } else {
                        acc[0] += wt.y * (int)z[0];
                    }
                }
                // the limb sums take any representative: the raw combination when it
                // is small enough for them to stay below 2^30 (host-checked bound)
#pragma unroll
                for (int e = 0; e < V; ++e) crt_add(L[e], REDUCE ? bal_small(acc[e], q) : acc[e], q, nmod);
            }
        }
        const int64_t row = (int64_t)a * rows + i;
        const int er = ea[row];
        double *out = C + row * ldc + (int64_t)c * cols + j0;
        const int *ebc = eb + (int64_t)c * cols + j0;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            if (e < valid) {
                const double val = crt_finish<NL, (NMOD > 0)>(L[e], er + ebc[e], nmod);
                out[e] = accumulate ? out[e] + val : val;
            }
        }
    }
}

// Row exponents s_i = beta - 1 - floor(log2 max_j |A_ij|) (0 for a zero row),
// one warp per row.
// rows: the count of rows handled; with a band (band_rows > 0) they are the
// rows [r0, r0 + band_rows) of each block row of block_rows rows.
__global__ void row_exp_kernel(const double *A, int64_t lda, int64_t rows, int64_t cols, int beta, int *exps,
                               int64_t band_rows = 0, int64_t block_rows = 0, int64_t r0 = 0) {
    const int64_t idx = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (idx >= rows) return;
    const int64_t row = band_rows > 0 ? (idx / band_rows) * block_rows + r0 + idx % band_rows : idx;
    const double *x = A + row * lda;
    unsigned mh = 0u, lo = 0u;   // max of the high words of |x|, OR of the low words
    if (((uintptr_t)x & 15) == 0) {
        // 16-byte loads where the row starts 16-byte aligned
        const double2 *x2 = reinterpret_cast<const double2 *>(x);
        const int64_t c2 = cols / 2;
#pragma unroll 4
        for (int64_t j = lane; j < c2; j += 32) {
            const double2 v = x2[j];
            mh = max(mh, max(abs_hi(v.x), abs_hi(v.y)));
            lo |= (unsigned)__double2loint(v.x) | (unsigned)__double2loint(v.y);
        }
        if ((cols & 1) && lane == 0) {
            mh = max(mh, abs_hi(x[cols - 1]));
            lo |= (unsigned)__double2loint(x[cols - 1]);
        }
    } else {
        for (int64_t j = lane; j < cols; j += 32) {
            mh = max(mh, abs_hi(x[j]));
            lo |= (unsigned)__double2loint(x[j]);
        }
    }
    mh = __reduce_max_sync(0xffffffffu, mh);
    lo = __reduce_or_sync(0xffffffffu, lo);
    if (mh >= OZ_NORMAL_HI || (mh | lo) == 0u) {
        if (lane == 0) exps[row] = (mh | lo) == 0u ? 0 : beta - 1 - (int(mh >> 20) - 1023);
        return;
    }
    // the row's largest entry is subnormal: its exact maximum in FP64 (rare)
    double mx = 0.0;
    for (int64_t j = lane; j < cols; j += 32) mx = fmax(mx, fabs(x[j]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) exps[row] = beta - 1 - ilog2_abs(mx);
}

__device__ const int g_ident_ptr[2] = {0, 1};
__device__ const int g_ident_code[1] = {0};
__device__ const int g_ident_coef[1] = {1};

typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

std::mutex g_oz_mu;
EncodeFn g_encode = nullptr;
bool g_tables[64] = {};

cudaError_t encode_fn(EncodeFn *out) {
    std::lock_guard<std::mutex> g(g_oz_mu);
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (!fn || q != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
        g_encode = (EncodeFn)fn;
    }
    *out = g_encode;
    return cudaSuccess;
}

int num_sms() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

template <int BN>
cudaError_t configure_residue_gemm_bn() {
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && !configured[dev]) {
        if ((e = cudaFuncSetAttribute(residue_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      oz_smem<BN>())) != cudaSuccess)
            return e;
        configured[dev] = true;
    }
    return cudaSuccess;
}

cudaError_t configure_residue_gemm() {
    cudaError_t e = configure_residue_gemm_bn<128>();
    return e != cudaSuccess ? e : configure_residue_gemm_bn<256>();
}


long long mod_pow_inv(long long a, long long p) {
    // inverse of a modulo p (a, p coprime) by the extended Euclidean algorithm
    long long t = 0, nt = 1, r = p, nr = a % p;
    while (nr != 0) {
        const long long q = r / nr;
        long long tmp = t - q * nt; t = nt; nt = tmp;
        tmp = r - q * nr; r = nr; nr = tmp;
    }
    return t < 0 ? t + p : t;
}

// The constant tables (moduli, Barrett constants, CRT weights for every
// moduli count) do not depend on the plan: uploaded once per device.
cudaError_t ensure_tables(int nmod) {
    if (nmod < 1 || nmod > OZ_CRT_MAX) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(g_oz_mu);
    if (dev < 64 && g_tables[dev]) return cudaSuccess;
    int mods[OZ_MAX_MOD] = {}, wmod[OZ_MAX_MOD][OZ_MAX_MOD] = {}, winv[OZ_MAX_MOD] = {};
    unsigned magic[OZ_MAX_MOD] = {}, r32[OZ_MAX_MOD] = {}, r21[OZ_MAX_MOD] = {}, r42[OZ_MAX_MOD] = {};
    for (int i = 0; i < OZ_MAX_MOD; ++i) {
        const unsigned long long p = (unsigned long long)kOzakiModuli[i];
        mods[i] = kOzakiModuli[i];
        magic[i] = (unsigned)((1ull << 32) / p);
        r32[i] = (unsigned)((1ull << 32) % p);
        r21[i] = (unsigned)((1ull << 21) % p);
        r42[i] = (unsigned)((1ull << 42) % p);
    }
    for (int j = 0; j < OZ_MAX_MOD; ++j) {
        long long w = 1 % mods[j];
        for (int i = 0; i < j; ++i) {
            wmod[i][j] = int(w);
            w = (w * mods[i]) % mods[j];
        }
        winv[j] = int(mod_pow_inv(w, mods[j]));   // w = (prod_{l<j} p_l) mod p_j
    }
    static int crt16[OZ_CRT_MAX + 1][OZ_CRT_MAX][8];
    static int P16[OZ_CRT_MAX + 1][8];
    static float fw[OZ_CRT_MAX + 1][8];
    static unsigned long long Pw[OZ_CRT_MAX + 1][2], Ph[OZ_CRT_MAX + 1][2], Pl[OZ_CRT_MAX + 1][2];
    std::memset(crt16, 0, sizeof(crt16));
    std::memset(P16, 0, sizeof(P16));
    std::memset(fw, 0, sizeof(fw));
    std::memset(Pw, 0, sizeof(Pw));
    std::memset(Ph, 0, sizeof(Ph));
    std::memset(Pl, 0, sizeof(Pl));
    for (int n = 1; n <= OZ_CRT_MAX; ++n) {
        unsigned __int128 P = 1;
        for (int i = 0; i < n; ++i) P *= (unsigned)mods[i];
        for (int q = 0; q < n; ++q) {
            const unsigned __int128 Mq = P / (unsigned)mods[q];
            const long long y = mod_pow_inv((long long)(Mq % (unsigned)mods[q]), mods[q]);
            const unsigned __int128 c = (Mq * (unsigned __int128)y) % P;   // Mq y < P p / p_q
            for (int l = 0; l < 8; ++l) crt16[n][q][l] = int((c >> (16 * l)) & 0xffff);
        }
        for (int l = 0; l < 8; ++l) {
            P16[n][l] = int((P >> (16 * l)) & 0xffff);
            const long double wl = ldexpl(1.0L, 16 * l) / (long double)P;
            fw[n][l] = wl < ldexpl(1.0L, -60) ? 0.f : (float)wl;
        }
        const unsigned __int128 half = P / 2;
        const __int128 low = (__int128)half - (__int128)P;
        Pw[n][0] = (unsigned long long)P; Pw[n][1] = (unsigned long long)(P >> 64);
        Ph[n][0] = (unsigned long long)half; Ph[n][1] = (unsigned long long)(half >> 64);
        Pl[n][0] = (unsigned long long)(unsigned __int128)low;
        Pl[n][1] = (unsigned long long)((unsigned __int128)low >> 64);
    }
    if ((e = cudaMemcpyToSymbol(c_mod, mods, sizeof(mods))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_wmod, wmod, sizeof(wmod))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_winv, winv, sizeof(winv))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_magic, magic, sizeof(magic))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_r32, r32, sizeof(r32))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_r21, r21, sizeof(r21))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_r42, r42, sizeof(r42))) != cudaSuccess) return e;
    {
        float modf[OZ_MAX_MOD], invp[OZ_MAX_MOD];
        for (int i = 0; i < OZ_MAX_MOD; ++i) {
            modf[i] = (float)mods[i];
            invp[i] = 1.0f / (float)mods[i];
        }
        if ((e = cudaMemcpyToSymbol(c_modf, modf, sizeof(modf))) != cudaSuccess) return e;
        if ((e = cudaMemcpyToSymbol(c_invp, invp, sizeof(invp))) != cudaSuccess) return e;
        float klimb[2][OZ_MAX_MOD][5];
        for (int wdt = 0; wdt < 2; ++wdt)
            for (int i = 0; i < OZ_MAX_MOD; ++i)
                for (int l = 0; l < 5; ++l) {
                    unsigned long long w = 1;
                    for (int t = 0; t < (13 + wdt) * l; ++t) w = (w * 2) % (unsigned long long)mods[i];
                    klimb[wdt][i][l] = (float)w;
                }
        if ((e = cudaMemcpyToSymbol(c_klimb, klimb, sizeof(klimb))) != cudaSuccess) return e;
        float klimbw[OZ_MAX_MOD][3];
        for (int i = 0; i < OZ_MAX_MOD; ++i) {
            const int shifts[3] = {0, 22, 37};
            for (int l = 0; l < 3; ++l) {
                long long w = 1;
                for (int t = 0; t < shifts[l]; ++t) w = (w * 2) % mods[i];
                if (2 * w > mods[i]) w -= mods[i];   // balanced: |w| <= p / 2
                klimbw[i][l] = (float)w;
            }
        }
        if ((e = cudaMemcpyToSymbol(c_klimbw, klimbw, sizeof(klimbw))) != cudaSuccess) return e;
    }
    if ((e = cudaMemcpyToSymbol(c_crt16, crt16, sizeof(crt16))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_P16, P16, sizeof(P16))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_fw, fw, sizeof(fw))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_P, Pw, sizeof(Pw))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_Phalf, Ph, sizeof(Ph))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_Plow, Pl, sizeof(Pl))) != cudaSuccess) return e;
    if (dev < 64) g_tables[dev] = true;
    return cudaSuccess;
}

cudaError_t make_map3d(CUtensorMap *m, void *ptr, int64_t kpad, int64_t rows, int64_t planes,
                       int box_rows, int64_t plane_rows) {
    EncodeFn enc;
    cudaError_t e = encode_fn(&enc);
    if (e != cudaSuccess) return e;
    cuuint64_t gdim[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t gstr[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)(kpad * plane_rows * 2)};
    cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ptr, gdim, gstr, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// A 3-D tiled map of any 1- or 2-byte element type (x innermost, in
// elements), with the given swizzle and box.
cudaError_t make_map3d_typed(CUtensorMap *m, CUtensorMapDataType dt, int esize, void *ptr, int64_t x,
                             int64_t y, int64_t z, int box_x, int box_y, CUtensorMapSwizzle sw) {
    EncodeFn enc;
    cudaError_t e = encode_fn(&enc);
    if (e != cudaSuccess) return e;
    cuuint64_t gdim[3] = {(cuuint64_t)x, (cuuint64_t)y, (cuuint64_t)z};
    cuuint64_t gstr[2] = {(cuuint64_t)(x * esize), (cuuint64_t)(x * y * esize)};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, dt, 3, ptr, gdim, gstr, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Row pitch of the product residues Z: n rounded up to 16 bytes, so the drain
// always stores whole 16-byte chunks.
int64_t z_pitch(int64_t n) { return (n + 15) / 16 * 16; }

// One product's residue GEMM (a group of one).  A band: the rows [r0, r0 + m)
// of planes of plane_m rows (S: plane_m x kpad per plane); the band's
// products go to Z as planes of m rows (the caller points Z at the band's own
// region).
cudaError_t launch_residue_gemm(const void *ra, const void *rb, int8_t *Z, int64_t m, int64_t n,
                                int64_t kpad, int64_t planes, int nmod, int *err, cudaStream_t s,
                                int *launches, int64_t r0 = 0, int64_t plane_m = -1, bool narrow = false) {
    RgDesc d{ra, rb, Z, m, n, kpad, planes, nmod, r0, plane_m < 0 ? m : plane_m};
    return launch_residue_gemm_group(&d, 1, err, s, launches, narrow);
}

// The residue GEMM with S' formed on chip (residue_gemm_fa): ra8 holds the
// int8 residues of A' ([q][m'][k']), rb the fp16 T'^T planes (leaves x nmod
// planes of nL x kpad); the leaves' terms come from the host copy of U.
cudaError_t launch_residue_gemm_fa(const ResPlan &rp, const int8_t *ra8, int64_t mp, int64_t kp, const void *rb,
                                   int8_t *Z, int64_t mL, int64_t kL, int64_t nL, int64_t kpad, int nmod, int *err,
                                   cudaStream_t s, int *launches) {
    cudaError_t e;
    static bool configured[64] = {};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev < 64 && !configured[dev]) {
        if ((e = cudaFuncSetAttribute(residue_gemm_fa, cudaFuncAttributeMaxDynamicSharedMemorySize, fa_smem())) !=
            cudaSuccess)
            return e;
        configured[dev] = true;
    }
    FaParams P;   // built on the host, passed to the kernel by value
    std::memset(&P, 0, sizeof(P));
    const int R = rp.L ? rp.R : 1, MK = rp.L ? rp.M * rp.K : 1, gK = rp.L ? rp.K : 1;
    for (int r = 0; r < R; ++r) {
        int nt = 0, a[2] = {0, 0}, b[2] = {0, 0};
        double c[2] = {1.0, 0.0};
        for (int i = 0; i < MK; ++i) {
            const double cf = rp.L ? rp.hU[(size_t)i * R + r] : 1.0;
            if (cf == 0.0) continue;
            if (nt >= FA_TMAX) return cudaErrorInvalidValue;
            a[nt] = i / gK;
            b[nt] = i % gK;
            c[nt] = cf;
            ++nt;
        }
        int kind;
        if (nt == 1) {
            kind = c[0] == 1.0 ? FA_P : c[0] == -1.0 ? FA_N : c[0] == 2.0 ? FA_P2 : c[0] == -2.0 ? FA_N2 : -1;
        } else if (nt == 2) {
            if (c[0] == -1.0 && c[1] == 1.0) {   // b - a: the positive term first
                std::swap(a[0], a[1]);
                std::swap(b[0], b[1]);
                std::swap(c[0], c[1]);
            }
            kind = (c[0] == 1.0 && c[1] == 1.0) ? FA_PP : (c[0] == 1.0 && c[1] == -1.0) ? FA_PN
                   : (c[0] == -1.0 && c[1] == -1.0) ? FA_NN : -1;
        } else {
            kind = -1;
        }
        if (kind < 0) return cudaErrorInvalidValue;
        P.t.n[r] = nt;
        P.t.kind[r] = kind;
        for (int t = 0; t < nt; ++t) {
            P.t.a[r][t] = a[t];
            P.t.b[r][t] = b[t];
        }
    }
    const int64_t planes = int64_t(R) * nmod;
    if ((e = make_map3d_typed(&P.tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, (void *)ra8, kp, mp, nmod, FA_BK, FA_BM,
                              CU_TENSOR_MAP_SWIZZLE_64B)) != cudaSuccess)
        return e;
    if ((e = make_map3d_typed(&P.tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void *)rb, kpad, nL, planes, FA_BK,
                              FA_BN, CU_TENSOR_MAP_SWIZZLE_128B)) != cudaSuccess)
        return e;
    P.Z = Z;
    P.m = mL;
    P.ldz = z_pitch(nL);
    P.mL = mL;
    P.kL = kL;
    P.kblocks = int(kpad / FA_BK);
    P.nmod = nmod;
    P.tiles_m = int((mL + FA_BM - 1) / FA_BM);
    P.tiles_n = int((nL + FA_BN - 1) / FA_BN);
    P.tiles_total = (int64_t)P.tiles_m * P.tiles_n * planes;
    const unsigned ctas = (unsigned)std::min<int64_t>(P.tiles_total, num_sms());
    cudaEvent_t t0 = timing_mark(s);
    residue_gemm_fa<<<ctas, FA_THREADS, fa_smem(), s>>>(P, err, wait_limit_ns());
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (t0 && !timing_mark(s)) timing_unmark();
    return cudaSuccess;
}

}  // namespace

// One persistent launch over all tiles of all planes of every problem of a
// group; N = 256 tiles when every problem's planes are at least 256 wide (and
// narrow tiles were not asked for).
cudaError_t launch_residue_gemm_group(const RgDesc *d, int count, int *err, cudaStream_t s, int *launches,
                                      bool narrow) {
    cudaError_t e;
    if (count < 1 || count > RG_MAX) return cudaErrorInvalidValue;
    if ((e = configure_residue_gemm()) != cudaSuccess) return e;
    bool wide = !narrow;
    for (int i = 0; i < count; ++i) wide = wide && d[i].n >= 256;
    const int bn = wide ? 256 : 128;
    RgGroup g;
    std::memset(&g, 0, sizeof(g));
    int64_t tiles = 0;
    for (int i = 0; i < count; ++i) {
        const RgDesc &q = d[i];
        // kpad is a multiple of 64, so the band's first row starts 16-byte aligned
        if ((e = make_map3d(&g.tmA[i], (void *)((const char *)q.ra + q.r0 * q.kpad * 2), q.kpad, q.m, q.planes,
                            OZ_BM, q.plane_m)) != cudaSuccess)
            return e;
        if ((e = make_map3d(&g.tmB[i], (void *)q.rb, q.kpad, q.n, q.planes, bn, q.n)) != cudaSuccess) return e;
        RgProblem &P = g.pr[i];
        P.Z = q.Z;
        P.m = q.m;
        P.ldz = z_pitch(q.n);
        P.kblocks = int(q.kpad / OZ_BK);
        P.nmod = q.nmod;
        P.tiles_m = int((q.m + OZ_BM - 1) / OZ_BM);
        P.tiles_n = int((q.n + bn - 1) / bn);
        P.tile_base = tiles;
        tiles += (int64_t)P.tiles_m * P.tiles_n * q.planes;
    }
    g.count = count;
    g.tiles_total = tiles;
    if (tiles == 0) return cudaSuccess;
    const unsigned ctas = (unsigned)std::min<int64_t>(tiles, num_sms());
    cudaEvent_t t0 = timing_mark(s);
    const unsigned long long wns = wait_limit_ns();
    if (wide)
        residue_gemm<256><<<ctas, oz_threads<256>(), oz_smem<256>(), s>>>(g, err, wns, 0);
    else
        residue_gemm<128><<<ctas, oz_threads<128>(), oz_smem<128>(), s>>>(g, err, wns, 0);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (t0 && !timing_mark(s)) timing_unmark();
    return cudaSuccess;
}

cudaError_t device_error_flag(int **out) { return cudaGetSymbolAddress((void **)out, g_device_error); }

cudaError_t read_device_error(int *flag, bool clear) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyFromSymbol(flag, g_device_error, sizeof(int))) != cudaSuccess) return e;
    if (clear && *flag) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_device_error, &zero, sizeof(int));
    }
    return e;
}

// The timeout path of the residue GEMM: one CTA over a 128 x 256 tile whose
// load and MMA threads issue nothing (dry), so the drain warps' first wait
// runs out after limit_ns with no copy or MMA outstanding; the CTA then sets
// the error flag and exits.  Small private buffers back the tensor maps.
cudaError_t residue_gemm_timeout_probe(unsigned long long limit_ns, cudaStream_t s) {
    cudaError_t e;
    if ((e = configure_residue_gemm()) != cudaSuccess) return e;
    int *err = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&err, g_device_error)) != cudaSuccess) return e;
    void *buf = nullptr;
    const size_t a_bytes = 128 * 64 * 2, b_bytes = 256 * 64 * 2, z_bytes = 128 * 256;
    if ((e = cudaMalloc(&buf, a_bytes + b_bytes + z_bytes)) != cudaSuccess) return e;
    char *c = (char *)buf;
    RgGroup g;
    std::memset(&g, 0, sizeof(g));
    if ((e = make_map3d(&g.tmA[0], c, 64, 128, 1, OZ_BM, 128)) == cudaSuccess &&
        (e = make_map3d(&g.tmB[0], c + a_bytes, 64, 256, 1, 256, 256)) == cudaSuccess) {
        g.pr[0] = RgProblem{(int8_t *)(c + a_bytes + b_bytes), 128, 256, 0, 1, 1, 1, 1};
        g.count = 1;
        g.tiles_total = 1;
        residue_gemm<256><<<1, oz_threads<256>(), oz_smem<256>(), s>>>(g, err, limit_ns, 1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    const cudaError_t f = cudaFree(buf);
    return e != cudaSuccess ? e : f;
}

// Largest beta <= 62 with k 2^(2 beta + 1) < P (P = product of the moduli,
// < 2^127 for N <= 16), so that |S'T'| < P/2 and the CRT is unambiguous.
static cudaError_t configure_split_form();

cudaError_t ozaki_prepare(int nmod) {
    cudaError_t e = ensure_tables(nmod);
    if (e != cudaSuccess) return e;
    if ((e = configure_split_form()) != cudaSuccess) return e;
    EncodeFn enc;
    if ((e = encode_fn(&enc)) != cudaSuccess) return e;
    int *err = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&err, g_device_error)) != cudaSuccess) return e;
    return configure_residue_gemm();
}

int ozaki_beta(int nmod, int64_t k) {
    unsigned __int128 P = 1;
    for (int i = 0; i < nmod; ++i) P *= (unsigned)kOzakiModuli[i];
    for (int beta = 62; beta > 0; --beta) {
        const int sh = 2 * beta + 1;
        // k 2^sh < P  <=>  k 2^sh <= P - 1  <=>  k <= floor((P - 1) / 2^sh)
        if (sh < 128 && (unsigned __int128)k <= ((P - 1) >> sh)) return beta;
    }
    return 0;
}

size_t ozaki_workspace(int64_t leaves, int nmod, int64_t m, int64_t k, int64_t n) {
    const int64_t kpad = (k + OZ_BK - 1) / OZ_BK * OZ_BK;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    return al(size_t(leaves) * nmod * m * kpad * 2) + al(size_t(leaves) * nmod * n * kpad * 2) +
           al(size_t(leaves) * m * 4) + al(size_t(leaves) * n * 4) + al(size_t(leaves) * nmod * m * z_pitch(n));
}

struct ResLayout {
    size_t ra0 = 0, rb0 = 0, ea = 0, eb = 0, zres = 0, total = 0;
    std::vector<size_t> la, lb, lw;   // per level l = 1..L (lw: l = 1..L-1); L = 0: la/lb = GEMM operands
};

// Block counts of the fused first-level kernels with a compiled instance.
static bool fused_nb(int nb) { return nb == 1 || nb == 4 || nb == 6 || nb == 8 || nb == 9; }

// The fused first level combines the scaled integers (|X'| < 2^beta) in
// int64: 2^beta sum_t |c_t| must stay below 2^62.
static bool first_level_fused(const ResPlan &rp, int nmod, int64_t kp) {
    const int beta = ozaki_beta(nmod, kp);
    const int cmax = rp.L ? std::max(rp.u_absmax, rp.v_absmax) : 1;
    int lg = 0;
    while ((1 << lg) < cmax) ++lg;
    if (beta + lg > 62) return false;
    return rp.L == 0 || (fused_nb(rp.M * rp.K) && fused_nb(rp.K * rp.N));
}

// The S side formed inside the residue GEMM (residue_gemm_fa): at most one
// level, integer coefficients with at most two terms and sum |c| <= 2 per
// leaf (|S'| <= 256), k blocks aligned for TMA (16 bytes) and at most 32768
// long, and the plan asked for it.  Then the workspace holds the int8 residues of A' instead of the S'
// operand planes, and T'^T planes in fp16.
static bool fused_a(const ResPlan &rp, int64_t mp, int64_t kp, int nmod) {
    if (!rp.fused_s || rp.L > 1 || !rp.hU || mp <= 0) return false;
    const int MK = rp.L ? rp.M * rp.K : 1, R = rp.L ? rp.R : 1;
    if (R > FA_MAX_LEAVES) return false;
    const int64_t kL = kp / (rp.L ? rp.K : 1);
    if (kL % 16 || kp % 16 || kp > (int64_t(1) << 31) - 64 || mp > (int64_t(1) << 31) - 256) return false;
    // |S'| <= p - 1 and |T'| <= p / 2: the int32 drain sum k_L p^2 / 2 stays
    // below the p 2^22 shift of the final reduction for k_L <= 2^23 / 256
    if (kL > 32768) return false;
    if (!first_level_fused(rp, nmod, kp)) return false;
    for (int r = 0; r < R && rp.L; ++r) {
        int nt = 0;
        double sum = 0;
        for (int i = 0; i < MK; ++i) {
            const double c = rp.hU[(size_t)i * R + r];
            if (c == 0.0) continue;
            ++nt;
            sum += std::fabs(c);
        }
        if (nt < 1 || nt > FA_TMAX || sum > 2.0) return false;
    }
    return true;
}

static ResLayout res_layout(const ResPlan &rp, int64_t mp, int64_t kp, int64_t np, int nmod) {
    ResLayout w;
    if (fused_a(rp, mp, kp, nmod)) {
        // exponents, int8 residues of A' ([q][m'][k']), T'^T fp16 planes, products
        auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
        size_t off = 0;
        auto take = [&](size_t bytes) { size_t o = off; off = al(off + bytes); return o; };
        const int64_t R = rp.L ? rp.R : 1, ml = mp / (rp.L ? rp.M : 1), kl = kp / (rp.L ? rp.K : 1),
                      nl = np / (rp.L ? rp.N : 1);
        const int64_t kpad = (kl + OZ_BK - 1) / OZ_BK * OZ_BK;
        w.ea = take(size_t(mp) * 4);
        w.eb = take(size_t(np) * 4);
        w.la.push_back(take(size_t(nmod) * mp * kp));
        w.lb.push_back(take(size_t(R) * nmod * nl * kpad * 2));
        w.zres = take(size_t(R) * nmod * ml * z_pitch(nl));
        w.total = off;
        return w;
    }
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = al(off + bytes); return o; };
    if (!first_level_fused(rp, nmod, kp)) {
        w.ra0 = take(size_t(nmod) * mp * kp);
        w.rb0 = take(size_t(nmod) * kp * np);
    }
    w.ea = take(size_t(mp) * 4);
    w.eb = take(size_t(np) * 4);
    int64_t cnt = 1, ml = mp, kl = kp, nl = np;
    if (rp.L == 0) {
        const int64_t kpad = (kp + OZ_BK - 1) / OZ_BK * OZ_BK;
        w.la.push_back(take(size_t(nmod) * mp * kpad * 2));
        w.lb.push_back(take(size_t(nmod) * np * kpad * 2));
        w.zres = take(size_t(nmod) * mp * z_pitch(np));
    }
    for (int l = 1; l <= rp.L; ++l) {
        cnt *= rp.R;
        ml /= rp.M; kl /= rp.K; nl /= rp.N;
        const int64_t kpad = (kl + OZ_BK - 1) / OZ_BK * OZ_BK;
        if (l < rp.L) {
            w.la.push_back(take(size_t(cnt) * nmod * ml * kl));
            w.lb.push_back(take(size_t(cnt) * nmod * nl * kl));
            w.lw.push_back(take(size_t(cnt) * nmod * ml * nl));
        } else {
            w.la.push_back(take(size_t(cnt) * nmod * ml * kpad * 2));
            w.lb.push_back(take(size_t(cnt) * nmod * nl * kpad * 2));
            w.zres = take(size_t(cnt) * nmod * ml * z_pitch(nl));
        }
    }
    w.total = off;
    return w;
}

size_t ozaki_fast_workspace(const ResPlan &rp, int64_t mp, int64_t kp, int64_t np, int nmod) {
    return res_layout(rp, mp, kp, np, nmod).total;
}

template <bool FINAL, int LC>
static cudaError_t launch_split_form_rows(int nb, const double *A, int64_t lda, const int *ea, int64_t rows,
                                          int64_t cols, int gridK, int R, int nmod, const int *ptr, const int *code,
                                          const int *icoef, void *out, int64_t out_ld, cudaStream_t s,
                                          int64_t r0 = 0, int64_t nr = -1) {
    if (nr < 0) nr = rows;
    if (nr == 0) return cudaSuccess;
    const int64_t threads = nr * ((out_ld + 3) / 4);
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    const size_t smem = size_t(nb) * 4 * 256 * 8;
#define FMM_SFR(NB) split_form_rows<NB, FINAL, LC><<<blocks, 256, smem, s>>>(A, lda, ea, rows, cols, gridK, R, nmod, ptr, code, icoef, out, out_ld, r0, nr)
    switch (nb) {
        case 1: FMM_SFR(1); break;
        case 4: FMM_SFR(4); break;
        case 6: FMM_SFR(6); break;
        case 8: FMM_SFR(8); break;
        case 9: FMM_SFR(9); break;
        default: return cudaErrorNotSupported;
    }
#undef FMM_SFR
    return cudaGetLastError();
}

template <bool FINAL, int LC, bool F16 = false>
static cudaError_t launch_split_form_cols_t(int nb, const double *B, int64_t ldb, const int *eb, int64_t krows,
                                            int64_t ncols, int gridN, int R, int nmod, const int *ptr,
                                            const int *code, const int *icoef, void *out, int64_t out_ld,
                                            cudaStream_t s) {
    const dim3 grid((unsigned)((out_ld + 31) / 32), (unsigned)((ncols + 31) / 32));
    const size_t smem = size_t(nb) * 32 * 33 * 8;   // >= nb * 4 * 256 * 8 (reused after the transpose)
#define FMM_SFC(NB) split_form_cols_t<NB, FINAL, LC, F16><<<grid, 256, smem, s>>>(B, ldb, eb, krows, ncols, gridN, R, nmod, ptr, code, icoef, out, out_ld)
    switch (nb) {
        case 1: FMM_SFC(1); break;
        case 4: FMM_SFC(4); break;
        case 6: FMM_SFC(6); break;
        case 8: FMM_SFC(8); break;
        case 9: FMM_SFC(9); break;
        default: return cudaErrorNotSupported;
    }
#undef FMM_SFC
    return cudaGetLastError();
}

// Shared-memory limits of the transposing split (NB x 8448 bytes); once per device.
static cudaError_t configure_split_form() {
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || configured[dev]) return cudaSuccess;
#define FMM_CFG1(NB, F, LC)                                                                                  \
    if ((e = cudaFuncSetAttribute(split_form_cols_t<NB, F, LC>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                  NB * 32 * 33 * 8)) != cudaSuccess)                                           \
        return e;                                                                                              \
    if ((e = cudaFuncSetAttribute(split_form_rows<NB, F, LC>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                  NB * 4 * 256 * 8)) != cudaSuccess)                                           \
        return e;
#define FMM_CFG16(NB, LC)                                                                                    \
    if ((e = cudaFuncSetAttribute(split_form_cols_t<NB, true, LC, true>,                                     \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, NB * 32 * 33 * 8)) != cudaSuccess) \
        return e;
#define FMM_CFG(NB) FMM_CFG1(NB, true, 0) FMM_CFG1(NB, false, 0) FMM_CFG1(NB, true, 1) FMM_CFG1(NB, false, 1) \
                    FMM_CFG1(NB, true, 2) FMM_CFG1(NB, false, 2) FMM_CFG1(NB, true, 3) FMM_CFG1(NB, false, 3) \
                    FMM_CFG16(NB, 0) FMM_CFG16(NB, 1) FMM_CFG16(NB, 2) FMM_CFG16(NB, 3)
    FMM_CFG(1) FMM_CFG(4) FMM_CFG(6) FMM_CFG(8) FMM_CFG(9)
#undef FMM_CFG16
#undef FMM_CFG1
#undef FMM_CFG
    configured[dev] = true;
    return cudaSuccess;
}

// C[:mp,:np] (+)= the fast algorithm run entirely in residue space on the
// once-scaled A' and B' (L = 0: the classical product), rebuilt by the CRT
// fused into the top level of the W combination.
cudaError_t ozaki_fast(const ResPlan &rp, const double *A, int64_t lda, const double *B, int64_t ldb,
                       double *C, int64_t ldc, int64_t mp, int64_t kp, int64_t np, int nmod,
                       int accumulate, void *ws, cudaStream_t s, int *launches, const HostPipe *pipe,
                       GemmDefer *defer) {
    // defer (grouped products): phase 0 enqueues everything before the
    // residue GEMM and describes that GEMM in defer->gemm; phase 1 enqueues
    // everything after it
    if (defer && (pipe || defer->phase < 0 || defer->phase > 1)) return cudaErrorInvalidValue;
    const bool pre = !defer || defer->phase == 0;
    cudaError_t e = ensure_tables(nmod);
    if (e != cudaSuccess) return e;
    if ((e = configure_split_form()) != cudaSuccess) return e;
    int *err = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&err, g_device_error)) != cudaSuccess) return e;
    const int *id_ptr = nullptr, *id_code = nullptr, *id_coef = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&id_ptr, g_ident_ptr)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&id_code, g_ident_code)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&id_coef, g_ident_coef)) != cudaSuccess) return e;
    const ResLayout w = res_layout(rp, mp, kp, np, nmod);
    const bool fused = first_level_fused(rp, nmod, kp);
    // S' formed inside the GEMM (not with grouped launches: those take the
    // ordinary operand planes)
    const bool fa = !defer && fused_a(rp, mp, kp, nmod);
    char *b = (char *)ws;
    int *ea = (int *)(b + w.ea), *eb = (int *)(b + w.eb);
    const int beta = ozaki_beta(nmod, kp);
    auto check = [&]() { ++*launches; return cudaGetLastError(); };

    auto form = [&](const int8_t *par, int64_t parents, int64_t prr, int64_t pcc, int64_t rows, int64_t cols,
                    const int *uptr, const int *ucode, const int *ucoef, void *out, bool last,
                    int64_t out_ld) -> cudaError_t {
        const int nbl = int((prr / rows) * (pcc / cols));
        if (nbl == 4 || nbl == 6 || nbl == 8 || nbl == 9) {
            // streaming: every parent element read once
            const bool al = (cols % 8 == 0) && (pcc % 8 == 0) && (out_ld % 8 == 0);
            const int gC = int(pcc / cols);
            const int64_t total = parents * nmod * rows * ((out_ld + 7) / 8);
            const unsigned blocks = (unsigned)((total + 255) / 256);
#define FMM_RSF(NB, F, AL) res_stream_form<NB, F, AL><<<blocks, 256, 0, s>>>(par, prr, pcc, rows, cols, gC, rp.R, nmod, parents, uptr, ucode, ucoef, out, out_ld)
#define FMM_RSF_NB(F, AL)                                                             \
    switch (nbl) {                                                                    \
        case 4: FMM_RSF(4, F, AL); break;                                             \
        case 6: FMM_RSF(6, F, AL); break;                                             \
        case 8: FMM_RSF(8, F, AL); break;                                             \
        default: FMM_RSF(9, F, AL); break;                                            \
    }
            if (last) {
                if (al) { FMM_RSF_NB(true, true) } else { FMM_RSF_NB(true, false) }
            } else {
                if (al) { FMM_RSF_NB(false, true) } else { FMM_RSF_NB(false, false) }
            }
#undef FMM_RSF_NB
#undef FMM_RSF
            return check();
        }
        const int64_t outs = parents * rp.R;
        const bool vec = (cols % 8 == 0) && (pcc % 8 == 0) && (out_ld % 8 == 0);
        const unsigned threads = 128;
        for (int64_t ob = 0; ob < outs; ob += 65535) {
            const unsigned cnt = (unsigned)std::min<int64_t>(65535, outs - ob);
            dim3 grid((unsigned)std::min<int64_t>(rows, 1024), cnt, (unsigned)nmod);
            if (last && vec)
                res_form_kernel<true, true><<<grid, threads, 0, s>>>(par, prr, pcc, rows, cols, rp.R, nmod, ob, uptr, ucode, ucoef, out, out_ld);
            else if (last)
                res_form_kernel<true, false><<<grid, threads, 0, s>>>(par, prr, pcc, rows, cols, rp.R, nmod, ob, uptr, ucode, ucoef, out, out_ld);
            else if (vec)
                res_form_kernel<false, true><<<grid, threads, 0, s>>>(par, prr, pcc, rows, cols, rp.R, nmod, ob, uptr, ucode, ucoef, out, out_ld);
            else
                res_form_kernel<false, false><<<grid, threads, 0, s>>>(par, prr, pcc, rows, cols, rp.R, nmod, ob, uptr, ucode, ucoef, out, out_ld);
            cudaError_t ce = check();
            if (ce != cudaSuccess) return ce;
        }
        return cudaSuccess;
    };

    // level 1 (or the GEMM operands when L = 0) straight from A and B; B is
    // kept transposed from here on, so every T_r is formed directly in the
    // K-major layout the residue GEMM reads.  Everything that reads A is
    // issued before anything that reads B, so that B may still be arriving
    // (pipe->b_ready) while the A side runs.
    const int64_t ml1 = mp / (rp.L ? rp.M : 1), kl1 = kp / (rp.L ? rp.K : 1), nl1 = np / (rp.L ? rp.N : 1);
    const int64_t kpad1 = (kl1 + OZ_BK - 1) / OZ_BK * OZ_BK;
    const bool last1 = rp.L <= 1;
    const int64_t out_ld1 = last1 ? kpad1 : kl1;
    const int R1 = rp.L ? rp.R : 1;
    const int gK = rp.L ? rp.K : 1, gN = rp.L ? rp.N : 1, nbA = rp.L ? rp.M * rp.K : 1, nbB = rp.L ? rp.K * rp.N : 1;
    const int *up = rp.L ? rp.u_ptr : id_ptr, *uc = rp.L ? rp.u_code : id_code, *ui = rp.L ? rp.u_icoef : id_coef;
    const int *vp = rp.L ? rp.v_ptr : id_ptr, *vc = rp.L ? rp.v_code : id_code, *vi = rp.L ? rp.v_icoef : id_coef;
    // limbs of |S'| < 2^(beta + ceil(log2 max sum|c|)): 3 x 14, 22 + 15 + 15, 4 x 14 or 5 x 13 bits
    int lc = 0;
    {
        const int cmax = rp.L ? std::max(rp.u_absmax, rp.v_absmax) : 1;
        // |A'| <= 2^beta (rounded), so |S'| <= cmax 2^beta < 2^(beta + floor(log2 cmax) + 1)
        int bits = beta + 1;
        while ((2 << (bits - beta - 1)) <= cmax) ++bits;
        lc = bits <= 42 ? 0 : bits <= 52 ? 3 : (bits <= 56 ? 1 : 2);
    }
#define FMM_SPLIT(WHICH, F, LC)                                                                                     \
    (WHICH ? launch_split_form_cols_t<F, LC>(nbB, B, ldb, eb, kl1, nl1, gN, R1, nmod, vp, vc, vi, b + w.lb[0],      \
                                             out_ld1, s)                                                           \
           : launch_split_form_rows<F, LC>(nbA, A, lda, ea, ml1, kl1, gK, R1, nmod, up, uc, ui, b + w.la[0],       \
                                           out_ld1, s, ar0, anr))
    // which 0: the A side, child rows [ar0, ar0 + anr); 1: the B side
    int64_t ar0 = 0, anr = ml1;
    // with S' formed in the GEMM: the A side is the int8 residues of A' itself
    // (the identity "level", one launch per first-level block row of the
    // band), the B side the first level in fp16
    int lc_id = 0;
    {
        const int bits = beta + 1;   // |A'| <= 2^beta
        lc_id = bits <= 42 ? 0 : bits <= 52 ? 3 : (bits <= 56 ? 1 : 2);
    }
    auto fa_split = [&](int which) -> cudaError_t {
        cudaError_t se = cudaSuccess;
        if (which) {
#define FMM_SFC16(LC) launch_split_form_cols_t<true, LC, true>(nbB, B, ldb, eb, kl1, nl1, gN, R1, nmod, vp, vc, vi, \
                                                                 b + w.lb[0], out_ld1, s)
            se = lc == 0 ? FMM_SFC16(0) : lc == 3 ? FMM_SFC16(3) : lc == 1 ? FMM_SFC16(1) : FMM_SFC16(2);
#undef FMM_SFC16
            ++*launches;
            return se;
        }
        const int gM1 = rp.L ? rp.M : 1;
        for (int a = 0; a < gM1 && se == cudaSuccess; ++a) {
            const int64_t r0 = a * ml1 + ar0;
#define FMM_SFR8(LC) launch_split_form_rows<false, LC>(1, A, lda, ea, mp, kp, 1, 1, nmod, id_ptr, id_code, id_coef, \
                                                         b + w.la[0], kp, s, r0, anr)
            se = lc_id == 0 ? FMM_SFR8(0) : lc_id == 3 ? FMM_SFR8(3) : lc_id == 1 ? FMM_SFR8(1) : FMM_SFR8(2);
#undef FMM_SFR8
            ++*launches;
        }
        return se;
    };
    auto fused_split = [&](int which) -> cudaError_t {
        if (fa) return fa_split(which);
        cudaError_t se;
        if (last1)
            se = lc == 0 ? FMM_SPLIT(which, true, 0) : lc == 3 ? FMM_SPLIT(which, true, 3)
                 : lc == 1 ? FMM_SPLIT(which, true, 1) : FMM_SPLIT(which, true, 2);
        else
            se = lc == 0 ? FMM_SPLIT(which, false, 0) : lc == 3 ? FMM_SPLIT(which, false, 3)
                 : lc == 1 ? FMM_SPLIT(which, false, 1) : FMM_SPLIT(which, false, 2);
        ++*launches;
        return se;
    };
#undef FMM_SPLIT
    // a base case without a fused first-level instance: level-0 residues, then level 1
    int8_t *ra0 = (int8_t *)(b + w.ra0), *rb0 = (int8_t *)(b + w.rb0);

    auto a_side = [&]() -> cudaError_t {
        cudaError_t ae;
        row_exp_kernel<<<(unsigned)((mp + 7) / 8), 256, 0, s>>>(A, lda, mp, kp, beta, ea);
        if ((ae = check()) != cudaSuccess) return ae;
        if (fused) return fused_split(0);
        split_rows_i8<<<(unsigned)((mp + 7) / 8), 256, 0, s>>>(A, lda, mp, kp, beta, nmod, ra0, ea);
        if ((ae = check()) != cudaSuccess) return ae;
        return form(ra0, 1, mp, kp, ml1, kl1, rp.u_ptr, rp.u_code, rp.u_icoef, b + w.la[0], last1, out_ld1);
    };
    auto b_side = [&]() -> cudaError_t {
        cudaError_t be;
        if (pipe && pipe->b_ready && (be = cudaStreamWaitEvent(s, pipe->b_ready, 0)) != cudaSuccess) return be;
        col_exp_wide<<<dim3((unsigned)((np + 31) / 32), 1), dim3(32, COL_EXP_ROWS), 0, s>>>(B, ldb, 0, kp, np, beta, eb);
        if ((be = check()) != cudaSuccess) return be;
        if (fused) return fused_split(1);
        split_cols_t_i8<<<dim3((unsigned)((kp + 31) / 32), (unsigned)((np + 31) / 32)), dim3(32, 8), 0, s>>>(
            B, ldb, kp, np, nmod, eb, rb0);
        if ((be = check()) != cudaSuccess) return be;
        return form(rb0, 1, np, kp, nl1, kl1, rp.v_ptr, rp.vt_code, rp.v_icoef, b + w.lb[0], last1, out_ld1);
    };
    // band j of A as the host copies it in: child rows [ml1 j / a_bands,
    // ml1 (j + 1) / a_bands) of every block row, exponents and the fused split
    auto a_band = [&](int j) -> cudaError_t {
        cudaError_t ae;
        if ((ae = cudaStreamWaitEvent(s, pipe->a_ready[j], 0)) != cudaSuccess) return ae;
        ar0 = ml1 * j / pipe->a_bands;
        anr = ml1 * (j + 1) / pipe->a_bands - ar0;
        if (anr > 0) {
            const int64_t rows = anr * (rp.L ? rp.M : 1);
            row_exp_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(A, lda, rows, kp, beta, ea, anr, ml1, ar0);
            if ((ae = check()) != cudaSuccess) return ae;
            ae = fused_split(0);
        }
        ar0 = 0;
        anr = ml1;
        return ae;
    };
    // With the products made in row bands, each A band is formed just before
    // the first product band that reads its rows (below), so the products
    // start once the first band of A is in rather than all of it.
    const int gb_pipe = (pipe && pipe->band_done && rp.L <= 1 && !fa)
                            ? (int)std::max<int64_t>(1, std::min<int64_t>(std::min(pipe->gemm_bands,
                                                                                   std::max(1, pipe->bands)), ml1))
                            : 1;
    const bool a_deferred = pre && pipe && pipe->a_bands > 0 && fused && !fa && !defer && gb_pipe > 1;
    int a_next = 0;   // the next A band still to be formed (a_deferred)
    if (!pre) {
        // phase 1: the operands were formed in phase 0
    } else if (pipe && pipe->a_bands > 0) {
        // the host copies B first, then A in bands, each with an event: the B
        // side runs while A arrives, and each A band is formed once it is in
        if ((e = b_side()) != cudaSuccess) return e;
        if (!fused) {
            if ((e = cudaStreamWaitEvent(s, pipe->a_ready[pipe->a_bands - 1], 0)) != cudaSuccess) return e;
            if ((e = a_side()) != cudaSuccess) return e;
        } else if (!a_deferred) {
            for (int j = 0; j < pipe->a_bands; ++j)
                if ((e = a_band(j)) != cudaSuccess) return e;
        }
    } else {
        if ((e = a_side()) != cudaSuccess) return e;
        if ((e = b_side()) != cudaSuccess) return e;
    }
    // levels 2..L: S and T^T level by level
    int64_t parents = rp.L ? rp.R : 1;
    int64_t pm = mp / (rp.L ? rp.M : 1), pk = kp / (rp.L ? rp.K : 1), pn = np / (rp.L ? rp.N : 1);
    for (int l = 2; l <= rp.L; ++l) {
        const int64_t ml = pm / rp.M, kl = pk / rp.K, nl = pn / rp.N;
        const int64_t kpad = (kl + OZ_BK - 1) / OZ_BK * OZ_BK;
        const bool last = l == rp.L;
        if (pre && (e = form((const int8_t *)(b + w.la[l - 2]), parents, pm, pk, ml, kl, rp.u_ptr, rp.u_code,
                             rp.u_icoef, b + w.la[l - 1], last, last ? kpad : kl)) != cudaSuccess)
            return e;
        // B^T: parent n x k, child nl x kl, block codes with rows and columns swapped
        if (pre && (e = form((const int8_t *)(b + w.lb[l - 2]), parents, pn, pk, nl, kl, rp.v_ptr, rp.vt_code,
                             rp.v_icoef, b + w.lb[l - 1], last, last ? kpad : kl)) != cudaSuccess)
            return e;
        parents *= rp.R;
        pm = ml; pk = kl; pn = nl;
    }
    // the leaf products, all leaves and moduli in one launch
    const int64_t mL = pm, kL = pk, nL = pn, leaves = parents;
    const int64_t kpadL = (kL + OZ_BK - 1) / OZ_BK * OZ_BK;
    const int64_t planes = leaves * nmod;
    int8_t *Z = (int8_t *)(b + w.zres);
    if (defer && defer->phase == 0) {
        defer->gemm = RgDesc{b + w.la.back(), b + w.lb.back(), Z, mL, nL, kpadL, planes, nmod, 0, mL};
        defer->narrow = rp.tile == FMM_TILE_128x128;
        return cudaSuccess;
    }

    // top level of W fused with the CRT, straight into C: the child rows
    // [r0, r0 + nr) of every block, from z (the first of them in plane 0,
    // planes zr rows apart)
    const int MN = rp.L ? rp.M * rp.N : 1, gM = rp.L ? rp.M : 1;   // gN: the block columns, as above
    const int *wp = rp.L ? rp.w_ptr : id_ptr, *wr = rp.L ? rp.w_r : id_code, *wc = rp.L ? rp.w_icoef : id_coef;
    // |limb sum| <= (sum_t |w_t|) 128 (2^16 - 1) nmod
    const bool reduce = double(rp.L ? rp.w_absmax : 1) * 128.0 * 65535.0 * nmod >= 1073741824.0;
    // the compiled moduli counts combine two columns per word: |sum w b| <= 128 sum|w| < 2^15
    const bool packed = (rp.L ? rp.w_absmax : 1) <= 255;
    auto w_crt = [&](const int8_t *z, int64_t zr, int64_t r0, int64_t nr, int64_t cm, int64_t cn,
                     int64_t cld) -> cudaError_t {
        const bool v4 = cld % 4 == 0;
        const int64_t threads = v4 ? nr * ((cn + 3) / 4) : nr * cn;
        const unsigned blocks = (unsigned)((threads + 255) / 256);
#define FMM_WCRT(V, RED, NM) w_crt_kernel<V, RED, NM><<<blocks, 256, 0, s>>>(z, cm, cn, cld, zr, r0, nr, gN, MN, nmod, wp, wr, wc, ea, eb, C, ldc, accumulate)
#define FMM_WCRT_N(V, RED)                                        \
    switch (nmod) {                                               \
        case 12: FMM_WCRT(V, RED, 12); break;                     \
        case 13: FMM_WCRT(V, RED, 13); break;                     \
        case 14: FMM_WCRT(V, RED, 14); break;                     \
        case 15: FMM_WCRT(V, RED, 15); break;                     \
        case 16: FMM_WCRT(V, RED, 16); break;                     \
        default: FMM_WCRT(V, RED, 0); break;                      \
    }
        if (v4 && packed) {
            if (reduce) { FMM_WCRT_N(4, true) } else { FMM_WCRT_N(4, false) }
        } else if (v4) {
            if (reduce) { FMM_WCRT(4, true, 0); } else { FMM_WCRT(4, false, 0); }
        } else {
            if (reduce) { FMM_WCRT(1, true, 0); } else { FMM_WCRT(1, false, 0); }
        }
#undef FMM_WCRT_N
#undef FMM_WCRT
        cudaError_t ce = check();
        if (ce == cudaSuccess && pipe && pipe->band_done) ce = pipe->band_done(pipe->ctx, r0, r0 + nr, cm, gM);
        return ce;
    };
    // the host's copy-out bands: each pass hands its rows over as soon as
    // they are written
    const int bands = (pipe && pipe->band_done) ? std::max(1, pipe->bands) : 1;

    // with one recursive level at most, the products themselves may be made
    // in row bands (each band of S against all of T; the band's products form
    // a region of their own in Z), each combined and handed over while the
    // next band is multiplied
    const int gb = (pipe && pipe->band_done && rp.L <= 1 && !fa)
                       ? (int)std::max<int64_t>(1, std::min<int64_t>(std::min(pipe->gemm_bands, bands), mL))
                       : 1;
    if (a_deferred && gb != gb_pipe) return cudaErrorInvalidValue;   // the two counts are the same rule
    if (gb > 1) {
        const int64_t cld = z_pitch(nL);
        const int sub = std::max(1, bands / gb);
        for (int g = 0; g < gb; ++g) {
            const int64_t R0 = mL * g / gb, NR = mL * (g + 1) / gb - R0;
            // every A band with rows below R0 + NR formed first (their S' rows
            // and row exponents are this band's inputs)
            while (a_deferred && a_next < pipe->a_bands && ml1 * a_next / pipe->a_bands < R0 + NR)
                if ((e = a_band(a_next++)) != cudaSuccess) return e;
            int8_t *Zb = Z + planes * R0 * cld;
            if ((e = launch_residue_gemm(b + w.la.back(), b + w.lb.back(), Zb, NR, nL, kpadL, planes, nmod, err,
                                         s, launches, R0, mL, rp.tile == FMM_TILE_128x128)) != cudaSuccess)
                return e;
            const int ns = (int)std::max<int64_t>(1, std::min<int64_t>(sub, NR));
            for (int t = 0; t < ns; ++t) {
                const int64_t r0 = R0 + NR * t / ns, nr = R0 + NR * (t + 1) / ns - r0;
                if ((e = w_crt(Zb + (r0 - R0) * cld, NR, r0, nr, mL, nL, cld)) != cudaSuccess) return e;
            }
        }
        while (a_deferred && a_next < pipe->a_bands)   // (none left: the bands cover all rows)
            if ((e = a_band(a_next++)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    while (a_deferred && a_next < pipe->a_bands)
        if ((e = a_band(a_next++)) != cudaSuccess) return e;

    if (fa) {
        if ((e = launch_residue_gemm_fa(rp, (const int8_t *)(b + w.la[0]), mp, kp, b + w.lb[0], Z, mL, kL, nL, kpadL,
                                        nmod, err, s, launches)) != cudaSuccess)
            return e;
    } else if (!defer && (e = launch_residue_gemm(b + w.la.back(), b + w.lb.back(), Z, mL, nL, kpadL, planes, nmod,
                                                  err, s, launches, 0, -1, rp.tile == FMM_TILE_128x128)) !=
               cudaSuccess) {
        return e;
    }
    // W levels L..2 on residues, down to the level-1 products
    int64_t cm = mL, cn = nL, cld = z_pitch(nL);
    const int8_t *child = Z;
    int64_t lp = leaves / (rp.L ? rp.R : 1);
    for (int l = rp.L; l >= 2; --l) {
        int8_t *parent = (int8_t *)(b + w.lw[l - 2]);
        const int64_t outs = lp * rp.M * rp.N;
        const bool vec = cn % 8 == 0;
        for (int64_t ob = 0; ob < outs; ob += 65535) {
            const unsigned cnt = (unsigned)std::min<int64_t>(65535, outs - ob);
            dim3 grid((unsigned)std::min<int64_t>(cm, 1024), cnt, (unsigned)nmod);
            if (vec)
                res_w_kernel<true><<<grid, 128, 0, s>>>(child, cm, cn, cld, rp.R, rp.N, rp.M * rp.N, nmod, parent,
                                                        ob, rp.w_ptr, rp.w_r, rp.w_icoef);
            else
                res_w_kernel<false><<<grid, 128, 0, s>>>(child, cm, cn, cld, rp.R, rp.N, rp.M * rp.N, nmod, parent,
                                                         ob, rp.w_ptr, rp.w_r, rp.w_icoef);
            if ((e = check()) != cudaSuccess) return e;
        }
        child = parent;
        cm *= rp.M;
        cn *= rp.N;
        cld = cn;
        lp /= rp.R;
    }
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(bands, cm));
    for (int band = 0; band < nb; ++band) {
        const int64_t r0 = cm * band / nb, nr = cm * (band + 1) / nb - r0;
        if ((e = w_crt(child + r0 * cld, cm, r0, nr, cm, cn, cld)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Leaf products Out[leaf] (m x n, ld ldo, leaf stride) = S[leaf] T[leaf]
// emulated in FP64 with nmod moduli.  S: m x k (lds, stride ss); T: k x n
// (ldt, stride ts).  ws: ozaki_workspace() bytes, 256-aligned.
cudaError_t ozaki_products(const double *S, int64_t lds, int64_t ss, const double *T, int64_t ldt,
                           int64_t ts, double *Out, int64_t ldo, int64_t os, int64_t leaves,
                           int64_t m, int64_t k, int64_t n, int nmod, void *ws,
                           cudaStream_t s, int *launches, int tile) {
    int *err = nullptr;
    cudaError_t e0 = cudaGetSymbolAddress((void **)&err, g_device_error);
    if (e0 != cudaSuccess) return e0;
    cudaError_t e = ensure_tables(nmod);
    if (e != cudaSuccess) return e;
    const int64_t kpad = (k + OZ_BK - 1) / OZ_BK * OZ_BK;
    const int beta = ozaki_beta(nmod, k);
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    char *w = (char *)ws;
    __nv_bfloat16 *ra = (__nv_bfloat16 *)w;
    w += al(size_t(leaves) * nmod * m * kpad * 2);
    __nv_bfloat16 *rb = (__nv_bfloat16 *)w;
    w += al(size_t(leaves) * nmod * n * kpad * 2);
    int *ea = (int *)w;
    w += al(size_t(leaves) * m * 4);
    int *eb = (int *)w;
    w += al(size_t(leaves) * n * 4);
    int8_t *Z = (int8_t *)w;

    {
        const int64_t warps = leaves * m;
        const unsigned blocks = (unsigned)((warps + 7) / 8);
        split_rows_kernel<<<blocks, 256, 0, s>>>(S, lds, ss, m, k, kpad, leaves, beta, nmod, ra, ea);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        if (leaves > 65535) return cudaErrorInvalidValue;
        col_exp_wide<<<dim3((unsigned)((n + 31) / 32), (unsigned)leaves), dim3(32, COL_EXP_ROWS), 0, s>>>(
            T, ldt, ts, k, n, beta, eb);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        dim3 grid((unsigned)((kpad + 31) / 32), (unsigned)((n + 31) / 32), (unsigned)leaves);
        split_cols_kernel<<<grid, dim3(32, 8), 0, s>>>(T, ldt, ts, k, n, kpad, nmod, eb, rb);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = launch_residue_gemm(ra, rb, Z, m, n, kpad, leaves * nmod, nmod, err, s, launches, 0, -1,
                                 tile == FMM_TILE_128x128)) != cudaSuccess)
        return e;
    {
        const int64_t total = leaves * m * n;
        const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
        if (n % 4 == 0)
            crt_kernel<4><<<blocks, 256, 0, s>>>(Z, m, n, z_pitch(n), leaves, nmod, ea, eb, Out, ldo, os, 0);
        else
            crt_kernel<1><<<blocks, 256, 0, s>>>(Z, m, n, z_pitch(n), leaves, nmod, ea, eb, Out, ldo, os, 0);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fmm
