// The residue GEMM with the S side formed on chip (emulated FP64, residue
// space, at most one recursive level): for every plane z = leaf * nmod + q,
// Z_z = S'_z T'_z mod p_q where S'_z = sum_t c_t A'_q(block t) is built in
// the kernel from the int8 residues of the once-scaled A' (never written to
// HBM as an operand plane), and T'^T comes from fp16 planes as usual.
//
// tcgen05 reads its A operand from tensor memory: four converter warps read
// the int8 term tiles that TMA brought into shared memory, combine them with
// the leaf's coefficients, convert to fp16 (exact: |S'| <= 256) and store the
// 128 x 64 k-block into one of two TMEM stages; the MMA thread multiplies it
// with the fp16 T'^T tile from shared memory.  Products are < 2^15, so a
// k-chunk of 512 sums exactly in FP32, drained to int32 as in residue_gemm.
// 128 x 192 tiles: two FP32 accumulators of 192 columns and the two A stages
// (32 columns each) fit the 512 TMEM columns.  Every wait is bounded.
// Included by ozaki.cu after residue_gemm.cuh.
#pragma once

constexpr int FA_BM = 128, FA_BN = 192, FA_BK = 64;
constexpr int FA_STAGES = 4, FA_ASTAGES = 2, FA_TBUF = 2, FA_TMAX = 2;
constexpr int FA_CONV_WARPS = 4, FA_DRAIN_WARPS = 8;
constexpr int FA_THREADS = (FA_CONV_WARPS + FA_DRAIN_WARPS + 2) * 32;
constexpr int FA_B_BYTES = FA_BN * FA_BK * 2;               // fp16 T'^T tile, 128-byte rows
constexpr int FA_A_BYTES = FA_BM * FA_BK;                   // int8 term tile, 64-byte rows
constexpr int FA_STAGE_BYTES = FA_B_BYTES + FA_TMAX * FA_A_BYTES;
constexpr int FA_A_COL0 = FA_TBUF * FA_BN;                  // TMEM columns of the A stages
constexpr int FA_TMEM_COLS = 512;
constexpr int FA_MAX_LEAVES = 64;
constexpr int fa_smem() { return FA_STAGES * FA_STAGE_BYTES + 1024 + 256; }

// The terms of each leaf's S': block (a, b) of the M x K grid and the
// coefficient kind (see fa_combine); at most FA_TMAX terms, sum |c| <= 2.
struct FaTerms {
    int n[FA_MAX_LEAVES];
    int kind[FA_MAX_LEAVES];
    int a[FA_MAX_LEAVES][FA_TMAX], b[FA_MAX_LEAVES][FA_TMAX];
};
// kind of a leaf's combination: value of S' from the biased bytes ua, ub
// (u = r + 128, r the balanced residue):
//   0: +a      1: -a      2: a + b    3: a - b    4: -a - b    5: +2a    6: -2a
enum { FA_P = 0, FA_N = 1, FA_PP = 2, FA_PN = 3, FA_NN = 4, FA_P2 = 5, FA_N2 = 6 };

struct FaParams {
    CUtensorMap tmA;     // int8 residues of A': (k', m', nmod), box (64, 128, 1), 64-byte swizzle
    CUtensorMap tmB;     // fp16 T'^T planes: (kpad, nL, planes), box (64, 192, 1), 128-byte swizzle
    int8_t *Z;           // product residues: planes of m x ldz
    int64_t m, ldz;      // rows of a plane (m_L), Z row pitch
    int64_t mL, kL;      // block size: row offset of block row a is a mL, of block column b is b kL
    int kblocks, nmod, tiles_m, tiles_n;
    int64_t tiles_total;
    FaTerms t;
};

__device__ __forceinline__ void mma_f16_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t bd, uint32_t idesc,
                                               uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
                 ::"r"(d_tmem), "r"(a_tmem), "l"(bd), "r"(idesc), "r"(acc) : "memory");
}

// Two fp16 values of S' (k-elements e, e+1) from the biased bytes of the two
// terms held in the 16-bit lanes of la / lb (lane value = byte): the integer
// L = combination + bias lies in [0, 1023], so 0x6400 + L is the fp16 1024 + L
// and one half2 subtraction leaves the exact value.
template <int KIND>
__device__ __forceinline__ unsigned fa_combine(unsigned la, unsigned lb) {
    // bias of L and sign of the result for each kind
    constexpr unsigned short B = KIND == FA_P || KIND == FA_N ? 0x6480 : KIND == FA_PN ? 0x64ff : 0x6500;
    constexpr bool NEG = KIND == FA_N || KIND == FA_NN || KIND == FA_N2;
    unsigned w;
    if constexpr (KIND == FA_P || KIND == FA_N) w = la;                          // L = a + 128
    else if constexpr (KIND == FA_PP || KIND == FA_NN) w = la + lb;              // L = a + b + 256
    else if constexpr (KIND == FA_PN) w = la + 0x00ff00ffu - lb;                 // L = a - b + 255
    else w = la + la;                                                            // L = 2a + 256
    w += 0x64006400u;
    const __half2 x = *reinterpret_cast<const __half2 *>(&w);
    const __half2 base = __halves2half2(__ushort_as_half(B), __ushort_as_half(B));
    const __half2 r = NEG ? __hsub2(base, x) : __hsub2(x, base);
    return *reinterpret_cast<const unsigned *>(&r);
}

// The converter warps' work on one tile: for every k-block, wait for its
// term tiles and for the tensor-memory stage to be free, form the 128 x 64
// block of S' (this thread: one row, 64 k-elements) and store it.  KIND and
// the term count are compile-time, so the loop is straight-line code.
template <int KIND>
__device__ __forceinline__ bool fa_convert_tile(const unsigned char *smem, uint64_t *full, uint64_t *afull,
                                                uint64_t *aempty, uint32_t tmem, int warp, int row, int kblocks,
                                                int64_t kL, int64_t &gk, unsigned long long wait_ns) {
    constexpr bool TWO = KIND == FA_PP || KIND == FA_PN || KIND == FA_NN;
    for (int kb = 0; kb < kblocks; ++kb, ++gk) {
        const int s = int(gk % FA_STAGES), j = int(gk % FA_ASTAGES);
        if (!mbar_wait(&full[s], uint32_t((gk / FA_STAGES) & 1), wait_ns) ||
            (gk >= FA_ASTAGES && !mbar_wait(&aempty[j], uint32_t(((gk / FA_ASTAGES) - 1) & 1), wait_ns)))
            return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned char *ta = smem + s * FA_STAGE_BYTES + FA_B_BYTES + row * 64;
        uint32_t v[32];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            // 16-byte chunk c of the row, 64-byte swizzle: chunk c ^ ((row / 2) % 4)
            const int off = 16 * (c ^ ((row >> 1) & 3));
            const uint4 x = *reinterpret_cast<const uint4 *>(ta + off);
            uint4 y = x;
            if constexpr (TWO) y = *reinterpret_cast<const uint4 *>(ta + FA_A_BYTES + off);
            const unsigned xa[4] = {x.x ^ 0x80808080u, x.y ^ 0x80808080u, x.z ^ 0x80808080u, x.w ^ 0x80808080u};
            const unsigned ya[4] = {y.x ^ 0x80808080u, y.y ^ 0x80808080u, y.z ^ 0x80808080u, y.w ^ 0x80808080u};
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                v[8 * c + 2 * w] = fa_combine<KIND>(__byte_perm(xa[w], 0u, 0x4140), __byte_perm(ya[w], 0u, 0x4140));
                v[8 * c + 2 * w + 1] =
                    fa_combine<KIND>(__byte_perm(xa[w], 0u, 0x4342), __byte_perm(ya[w], 0u, 0x4342));
            }
        }
        const int kvalid = (int)min((int64_t)FA_BK, kL - (int64_t)kb * FA_BK);
        if (kvalid < FA_BK) {
            // past the block's k range: zero (the tile reaches into the next block)
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if (2 * e >= kvalid) v[e] = 0u;
                else if (2 * e + 1 >= kvalid) v[e] &= 0xffffu;
            }
        }
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(FA_A_COL0 + j * 32);
        asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                     "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                     ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                       "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
                       "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]),
                       "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]),
                       "r"(v[31])
                     : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&afull[j]);
    }
    return true;
}

__global__ void __launch_bounds__(FA_THREADS, 1)
residue_gemm_fa(const __grid_constant__ FaParams P, int *err, unsigned long long wait_ns) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + FA_STAGES * FA_STAGE_BYTES);
    uint64_t *empty = full + FA_STAGES;
    uint64_t *afull = empty + FA_STAGES;
    uint64_t *aempty = afull + FA_ASTAGES;
    uint64_t *tfull = aempty + FA_ASTAGES;
    uint64_t *tempty = tfull + FA_TBUF;
    uint64_t *mdone = tempty + FA_TBUF;
    uint32_t *tmem_slot = (uint32_t *)(mdone + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t per_plane = (int64_t)P.tiles_m * P.tiles_n;
    const int nchunks = (P.kblocks + OZ_CHUNK_KB - 1) / OZ_CHUNK_KB;
    constexpr int DRAIN0 = FA_CONV_WARPS, TMAW = DRAIN0 + FA_DRAIN_WARPS, MMAW = TMAW + 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < FA_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int j = 0; j < FA_ASTAGES; ++j) { mbar_init(&afull[j], FA_CONV_WARPS * 32); mbar_init(&aempty[j], 1); }
        for (int b = 0; b < FA_TBUF; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], FA_DRAIN_WARPS * 32); }
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(tmem_slot)), "r"(FA_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == TMAW) {
        if (lane == 0) {
            int64_t gk = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < P.tiles_total && ok; tile += gridDim.x) {
                int z, tm, tn;
                tile_coords(tile, per_plane, P.tiles_m, P.tiles_n, z, tm, tn);
                const int leaf = z / P.nmod, q = z % P.nmod, nt = P.t.n[leaf];
                for (int kb = 0; kb < P.kblocks; ++kb, ++gk) {
                    const int s = int(gk % FA_STAGES);
                    if (gk >= FA_STAGES &&
                        !mbar_wait(&empty[s], uint32_t(((gk / FA_STAGES) - 1) & 1), wait_ns)) {
                        atomicExch(err, 1);
                        ok = false;
                        break;
                    }
                    unsigned char *sb = smem + s * FA_STAGE_BYTES, *sa = sb + FA_B_BYTES;
                    mbar_expect_tx(&full[s], FA_B_BYTES + nt * FA_A_BYTES);
                    tma_load_3d(sb, &P.tmB, kb * FA_BK, tn * FA_BN, z, &full[s]);
                    for (int t = 0; t < nt; ++t)
                        tma_load_3d(sa + t * FA_A_BYTES, &P.tmA, int(P.t.b[leaf][t] * P.kL) + kb * FA_BK,
                                    int(P.t.a[leaf][t] * P.mL) + tm * FA_BM, q, &full[s]);
                }
            }
            // no bulk copy of this CTA may still be in flight when it exits
            for (int64_t j = gk > FA_STAGES ? gk - FA_STAGES : 0; j < gk; ++j)
                if (!mbar_wait(&full[j % FA_STAGES], uint32_t((j / FA_STAGES) & 1), wait_ns)) atomicExch(err, 1);
        }
    } else if (warp == MMAW) {
        if (lane == 0) {
            // FP32 accumulator, fp16 A (tensor memory) and B (shared memory, K-major)
            const uint32_t idesc = (1u << 4) | ((uint32_t)(FA_BN >> 3) << 17) | ((uint32_t)(FA_BM >> 4) << 24);
            bool ok = true;
            int64_t gk = 0, cg = 0;
            for (int64_t tile = blockIdx.x; tile < P.tiles_total && ok; tile += gridDim.x) {
                int kb = 0;
                for (int c = 0; c < nchunks && ok; ++c, ++cg) {
                    const int b = int(cg % FA_TBUF);
                    if (cg >= FA_TBUF && !mbar_wait(&tempty[b], uint32_t(((cg / FA_TBUF) - 1) & 1), wait_ns)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t acc = tmem + (uint32_t)(b * FA_BN);
                    const int kend = min(P.kblocks, (c + 1) * OZ_CHUNK_KB);
                    for (int first = 1; kb < kend; ++kb, ++gk, first = 0) {
                        const int s = int(gk % FA_STAGES), j = int(gk % FA_ASTAGES);
                        if (!mbar_wait(&full[s], uint32_t((gk / FA_STAGES) & 1), wait_ns) ||
                            !mbar_wait(&afull[j], uint32_t((gk / FA_ASTAGES) & 1), wait_ns)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t b0 = su32(smem + s * FA_STAGE_BYTES);
                        const uint32_t a0 = tmem + (uint32_t)(FA_A_COL0 + j * 32);
#pragma unroll
                        for (int kk = 0; kk < FA_BK / 16; ++kk)
                            mma_f16_tmem_a(acc, a0 + kk * 8, smem_desc(b0 + kk * 32), idesc,
                                           (first && kk == 0) ? 0u : 1u);
                        mma_commit(&empty[s]);
                        mma_commit(&aempty[j]);
                    }
                    mma_commit(&tfull[b]);
                }
            }
            // every MMA issued here completes before TMEM is freed
            mma_commit(mdone);
            if (!mbar_wait(mdone, 0u, wait_ns)) ok = false;
            if (!ok) atomicExch(err, 1);
        }
    } else if (warp < DRAIN0) {
        // converter warps: warp w owns TMEM lanes (tile rows) 32 w .. 32 w + 31
        const int row = 32 * warp + lane;
        bool ok = true;
        int64_t gk = 0;
        for (int64_t tile = blockIdx.x; tile < P.tiles_total && ok; tile += gridDim.x) {
            int z, tm, tn;
            tile_coords(tile, per_plane, P.tiles_m, P.tiles_n, z, tm, tn);
            const int leaf = z / P.nmod;
#define FA_CONV(K) ok = fa_convert_tile<K>(smem, full, afull, aempty, tmem, warp, row, P.kblocks, P.kL, gk, wait_ns)
            switch (P.t.kind[leaf]) {
                case FA_P: FA_CONV(FA_P); break;
                case FA_N: FA_CONV(FA_N); break;
                case FA_PP: FA_CONV(FA_PP); break;
                case FA_PN: FA_CONV(FA_PN); break;
                case FA_NN: FA_CONV(FA_NN); break;
                case FA_P2: FA_CONV(FA_P2); break;
                default: FA_CONV(FA_N2); break;
            }
#undef FA_CONV
        }
        if (!ok && lane == 0) atomicExch(err, 1);
    } else {
        // drain warps: warp w reads TMEM lanes 32 (w % 4) .. + 31 and the
        // 96-column half (w - DRAIN0) / 4 of the accumulator
        const int lg = warp % 4, ch = (warp - DRAIN0) / 4;
        bool ok = true;
        int64_t cg = 0;
        for (int64_t tile = blockIdx.x; tile < P.tiles_total && ok; tile += gridDim.x) {
            int z, tm, tn;
            tile_coords(tile, per_plane, P.tiles_m, P.tiles_n, z, tm, tn);
            const int q = z % P.nmod;
            const int p = c_mod[q];
            int acc[96];
#pragma unroll
            for (int j = 0; j < 96; ++j) acc[j] = 0;
            for (int c = 0; c < nchunks; ++c, ++cg) {
                const int b = int(cg % FA_TBUF);
                if (!mbar_wait(&tfull[b], uint32_t((cg / FA_TBUF) & 1), wait_ns)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * FA_BN + ch * 96);
#pragma unroll
                for (int c0 = 0; c0 < 96; c0 += 16) {
                    uint32_t r[16];
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                                 : "r"(base + (uint32_t)c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[c0 + j] += __float2int_rn(__uint_as_float(r[j]));
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&tempty[b]);
            }
            if (!ok) break;
            const int64_t orow = (int64_t)tm * FA_BM + lg * 32 + lane;
            if (orow < P.m) {
                const int64_t col0 = (int64_t)tn * FA_BN + ch * 96;
                int8_t *out = P.Z + ((int64_t)z * P.m + orow) * P.ldz + col0;
                const int64_t cols = min((int64_t)96, P.ldz - col0);
                // |acc| < 2^28: shift positive by p 2^22 (< 2^31) for one Barrett step
#pragma unroll
                for (int j0 = 0; j0 < 96; j0 += 16) {
                    if (j0 < cols) {
                        __align__(16) int8_t h[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int rr = (int)mod_u32((unsigned)(acc[j0 + e] + (p << 22)), q);
                            h[e] = (int8_t)(rr >= (p + 1) / 2 ? rr - p : rr);
                        }
                        *reinterpret_cast<uint4 *>(out + j0) = *reinterpret_cast<const uint4 *>(h);
                    }
                }
            }
        }
        if (!ok && lane == 0) atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FA_TMEM_COLS) : "memory");
}
