// The residue GEMM of the emulated-FP64 variant: for every plane z (leaf
// times modulus), Z_z = S'_z T'_z mod p on tcgen05 (kind::f16, bfloat16
// residues, FP32 accumulation in TMEM drained to int32 every 512 k), stored
// as balanced int8 residues.  Included by ozaki.cu after the moduli tables
// (c_mod, c_magic) and mod_u32; kept in its own file so its measured DRAM
// traffic can be tied to this exact source.
#pragma once

// Z[z][row][col] (int8 balanced residues), z = leaf * nmod + modulus index,
// for each problem of the launch.
// Persistent: CTA c handles tiles c, c + gridDim.x, ...; the load, MMA and
// drain roles walk the same tile sequence, so stage and TMEM-buffer phases
// continue across tiles and the tensor core never waits for a tile's final
// reduction.  Every wait gives up after wait_ns nanoseconds (err set); before
// the CTA exits, the load thread waits for the copies it issued to land and
// the MMA thread for its MMAs to complete, so nothing asynchronous of the CTA
// outlives it (unless those waits run out too).  dry != 0 (tests of the
// timeout path only): the load and MMA threads issue nothing, so the drain
// warps' first wait runs out with no copy or MMA outstanding.
// Tile t of the persistent sequence -> (plane z, tile row tm, tile column tn).
// Within a plane, tiles go in groups of OZ_GROUP tile rows, column by column,
// so the CTAs of one wave share a few A row panels and B column panels in L2
// (a plane of 8192 x 8192 bf16 residues, 128 MB per operand, does not fit).
constexpr int OZ_GROUP = 16;
__device__ __forceinline__ void tile_coords(int64_t tile, int64_t per_plane, int tiles_m, int tiles_n, int &z,
                                            int &tm, int &tn) {
    z = int(tile / per_plane);
    const int rem = int(tile % per_plane);
    const int g = rem / (OZ_GROUP * tiles_n);
    const int tm0 = g * OZ_GROUP;
    const int gsz = min(OZ_GROUP, tiles_m - tm0);
    const int within = rem - g * OZ_GROUP * tiles_n;
    tn = within / gsz;
    tm = tm0 + within % gsz;
}

// A launch covers a group of up to RG_MAX independent problems (one for an
// ordinary product): each has its own operand tensor maps, product planes and
// sizes; the persistent tile sequence runs through problem 0's tiles, then
// problem 1's, and so on (tile_base: the first tile of each).
constexpr int RG_MAX = RG_MAX_PROBLEMS;
struct RgProblem {
    int8_t *Z;                 // product residues, planes of m x ldz
    int64_t m, ldz;
    int64_t tile_base;         // first tile of this problem in the launch
    int kblocks, nmod, tiles_m, tiles_n;
};
struct RgGroup {
    CUtensorMap tmA[RG_MAX];   // S' planes (K-major, bf16)
    CUtensorMap tmB[RG_MAX];   // T'^T planes
    RgProblem pr[RG_MAX];
    int64_t tiles_total;
    int count;
};

// Problem of a tile of the launch (the problems' tile ranges are consecutive).
__device__ __forceinline__ int rg_problem(const RgGroup &g, int64_t tile) {
    int p = 0;
#pragma unroll 1
    while (p + 1 < g.count && tile >= g.pr[p + 1].tile_base) ++p;
    return p;
}

template <int BN>
struct OzCfg;
template <>
struct OzCfg<128> {   // 4 drain warps, 4 TMEM accumulators, 6 stages of 32 KB
    static constexpr int TBUF = 4, DRAIN_WARPS = 4, STAGES = 6;
};
template <>
struct OzCfg<256> {   // 8 drain warps (two column halves), 2 accumulators, 4 stages of 48 KB
    static constexpr int TBUF = 2, DRAIN_WARPS = 8, STAGES = 4;
};
template <int BN>
constexpr int oz_threads() { return (OzCfg<BN>::DRAIN_WARPS + 2) * 32; }
template <int BN>
constexpr int oz_smem() { return OzCfg<BN>::STAGES * (OZ_A_BYTES + BN * OZ_BK * 2) + 1024 + 256; }

template <int BN>
__global__ void __launch_bounds__(oz_threads<BN>(), 1)
residue_gemm(const __grid_constant__ RgGroup g, int *err, unsigned long long wait_ns, int dry) {
    constexpr int OZ_TBUF = OzCfg<BN>::TBUF, OZ_STAGES = OzCfg<BN>::STAGES;
    constexpr int DW = OzCfg<BN>::DRAIN_WARPS;
    constexpr int OZ_BN = BN, OZ_B_BYTES = BN * OZ_BK * 2, OZ_STAGE_BYTES = OZ_A_BYTES + OZ_B_BYTES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + OZ_STAGES * OZ_STAGE_BYTES);
    uint64_t *empty = full + OZ_STAGES;
    uint64_t *tfull = empty + OZ_STAGES;
    uint64_t *tempty = tfull + OZ_TBUF;
    uint64_t *mdone = tempty + OZ_TBUF;   // the MMA thread's last commit
    uint32_t *tmem_slot = (uint32_t *)(mdone + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t tiles_total = g.tiles_total;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZ_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < OZ_TBUF; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], DW * 32); }
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(tmem_slot)), "r"(OZ_TBUF * OZ_BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == DW) {
        if (lane == 0 && !dry) {
            int64_t gk = 0;   // global k-block counter: stage and phase
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < tiles_total && ok; tile += gridDim.x) {
                const int p = rg_problem(g, tile);
                const RgProblem &P = g.pr[p];
                int z, tm, tn;
                tile_coords(tile - P.tile_base, (int64_t)P.tiles_m * P.tiles_n, P.tiles_m, P.tiles_n, z, tm, tn);
                for (int kb = 0; kb < P.kblocks; ++kb, ++gk) {
                    const int s = int(gk % OZ_STAGES);
                    if (gk >= OZ_STAGES && !mbar_wait(&empty[s], uint32_t(((gk / OZ_STAGES) - 1) & 1), wait_ns)) {
                        atomicExch(err, 1);
                        ok = false;
                        break;
                    }
                    unsigned char *sa = smem + s * OZ_STAGE_BYTES, *sb = sa + OZ_A_BYTES;
                    mbar_expect_tx(&full[s], OZ_STAGE_BYTES);
                    tma_load_3d(sa, &g.tmA[p], kb * OZ_BK, tm * OZ_BM, z, &full[s]);
                    tma_load_3d(sb, &g.tmB[p], kb * OZ_BK, tn * OZ_BN, z, &full[s]);
                }
            }
            // no bulk copy of this CTA may still be in flight when it exits:
            // wait for the last (at most OZ_STAGES) k-blocks issued to land
            // (normally consumed long ago; after a timeout elsewhere, bounded)
            for (int64_t j = gk > OZ_STAGES ? gk - OZ_STAGES : 0; j < gk; ++j)
                if (!mbar_wait(&full[j % OZ_STAGES], uint32_t((j / OZ_STAGES) & 1), wait_ns)) atomicExch(err, 1);
        }
    } else if (warp == DW + 1) {
        if (lane == 0 && !dry) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                   ((uint32_t)(OZ_BN >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
            bool ok = true;
            int64_t gk = 0, cg = 0;   // global k-block and chunk counters
            for (int64_t tile = blockIdx.x; tile < tiles_total && ok; tile += gridDim.x) {
                const int kblocks = g.pr[rg_problem(g, tile)].kblocks;
                const int nchunks = (kblocks + OZ_CHUNK_KB - 1) / OZ_CHUNK_KB;
                int kb = 0;
                for (int c = 0; c < nchunks && ok; ++c, ++cg) {
                    const int b = int(cg % OZ_TBUF);
                    if (cg >= OZ_TBUF && !mbar_wait(&tempty[b], uint32_t(((cg / OZ_TBUF) - 1) & 1), wait_ns)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t acc_tmem = tmem + (uint32_t)(b * OZ_BN);
                    const int kend = min(kblocks, (c + 1) * OZ_CHUNK_KB);
                    for (int first = 1; kb < kend; ++kb, ++gk, first = 0) {
                        const int s = int(gk % OZ_STAGES);
                        if (!mbar_wait(&full[s], uint32_t((gk / OZ_STAGES) & 1), wait_ns)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t a0 = su32(smem + s * OZ_STAGE_BYTES), b0 = a0 + OZ_A_BYTES;
#pragma unroll
                        for (int kk = 0; kk < OZ_BK / 16; ++kk)
                            mma_bf16(acc_tmem, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32), idesc,
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
        // and the 128-column half w/4 of the accumulator
        const int lg = warp % 4, ch = warp / 4;
        bool ok = true;
        int64_t cg = 0;
        for (int64_t tile = blockIdx.x; tile < tiles_total && ok; tile += gridDim.x) {
            const RgProblem &P = g.pr[rg_problem(g, tile)];
            int z, tm, tn;
            tile_coords(tile - P.tile_base, (int64_t)P.tiles_m * P.tiles_n, P.tiles_m, P.tiles_n, z, tm, tn);
            const int q = z % P.nmod;
            const int p = c_mod[q];
            const int nchunks = (P.kblocks + OZ_CHUNK_KB - 1) / OZ_CHUNK_KB;
            const int64_t m = P.m, ldz = P.ldz;
            int8_t *Z = P.Z;
            int acc[128];
#pragma unroll
            for (int j = 0; j < 128; ++j) acc[j] = 0;
            for (int c = 0; c < nchunks; ++c, ++cg) {
                const int b = int(cg % OZ_TBUF);
                if (!mbar_wait(&tfull[b], uint32_t((cg / OZ_TBUF) & 1), wait_ns)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * OZ_BN + ch * 128);
#pragma unroll
                for (int c0 = 0; c0 < 128; c0 += 16) {
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
            const int64_t row = (int64_t)tm * OZ_BM + lg * 32 + lane;
            if (row < m) {
                const int64_t col0 = (int64_t)tn * OZ_BN + ch * 128;
                // rows of Z are padded to ldz (a multiple of 16); columns past n hold
                // residues of zero (the TMA fills B rows past n with zeros)
                int8_t *out = Z + ((int64_t)z * m + row) * ldz + col0;
                const int64_t cols = min((int64_t)128, ldz - col0);
                // |acc| < 2^28: shift positive by p 2^22 (< 2^31) for one Barrett step
#pragma unroll
                for (int j0 = 0; j0 < 128; j0 += 16) {
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TBUF * OZ_BN) : "memory");
}

