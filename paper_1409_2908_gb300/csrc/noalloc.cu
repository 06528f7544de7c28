// fmm_gemm_noalloc: the deterministic product (leaf products stored, then a
// fixed-order pass forms C) with its only scratch, the leaf products, held in
// a fixed static device array instead of caller-provided or allocated memory.
//
// Some callers cannot allocate device memory at the point where they need a
// product: host runtimes whose device memory is reserved up front by another
// allocator (a framework's caching allocator or a pool sized at start-up, so
// a cudaMalloc there fails or competes with the pool), and code that may not
// call into the CUDA allocator on its hot path at all.  This entry point
// allocates nothing and copies nothing from the host: the unrolled plan lists
// are the plan's own device copy (made by fmm_plan_prepare or an earlier
// fmm_gemm), and the leaf products live in `g_noalloc_scratch`, a file-scope
// array of FMM_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "fmm_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FMM_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array, looked up once per device with that
// device current (a host-side reference to the symbol is not a device address).
std::mutex g_scratch_mu;
void *g_scratch_ptr[64] = {};

fmm_status scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FMM_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return FMM_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return FMM_OK;
}

int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

bool overlap(const void *a, size_t na, const void *b, size_t nb) {
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + nb && y < x + na;
}

size_t span_bytes(int64_t rows, int64_t cols, int64_t ld) { return size_t(((rows - 1) * ld + cols) * 8); }

fmm_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return FMM_OK;
    cudaGetLastError();
    return FMM_ERR_CUDA;
}

}  // namespace

extern "C" fmm_status fmm_gemm_noalloc(fmm_plan_t p, const double *A, int64_t lda,
                                       const double *B, int64_t ldb, double *C, int64_t ldc,
                                       int64_t m, int64_t k, int64_t n, void *stream) {
    using namespace fmm;
    set_last_launch_count(0);
    if (!p || !A || !B || !C) return FMM_ERR_ARG;
    if (m < 1 || k < 1 || n < 1 || lda < k || ldb < n || ldc < n) return FMM_ERR_ARG;
    if (m > (int64_t(1) << 31) || k > (int64_t(1) << 31) || n > (int64_t(1) << 31)) return FMM_ERR_ARG;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 7) return FMM_ERR_ARG;
    if (overlap(C, span_bytes(m, n, ldc), A, span_bytes(m, k, lda)) ||
        overlap(C, span_bytes(m, n, ldc), B, span_bytes(k, n, ldb)))
        return FMM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int launches = 0;

    const int64_t sm = ipow(p->M, p->L), sk = ipow(p->K, p->L), sn = ipow(p->N, p->L);
    const int64_t mp = (m / sm) * sm, kp = (k / sk) * sk, np = (n / sn) * sn;
    const int64_t mL = mp / sm, kL = kp / sk, nL = np / sn;
    if (p->L == 0 || mp == 0 || kp == 0 || np == 0) {
        const fmm_status cs = to_status(launch_classical(A, lda, B, ldb, C, ldc, m, k, n, FMM_TILE_AUTO, s, &launches));
        set_last_launch_count(launches);
        return cs;
    }

    // the plan's lists must already be on this device: uploading them here
    // would allocate
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess) return to_status(cudaGetLastError());
    {
        std::lock_guard<std::mutex> g(p->upload_mu);
        if (!p->uploaded || p->upload_device != dev) return FMM_ERR_ARG;
    }
    const size_t need = size_t(p->leaves) * size_t(mL) * size_t(nL) * 8;
    if (need > size_t(FMM_NOALLOC_SCRATCH_BYTES)) return FMM_ERR_UNSUPPORTED;

    void *base = nullptr;
    fmm_status st = scratch_address(&base);
    if (st != FMM_OK) return st;
    double *wsM = (double *)base;
    cudaError_t e;

    LeafLaunch L{};
    L.A = A; L.lda = lda; L.B = B; L.ldb = ldb; L.C = C; L.ldc = ldc;
    L.mL = mL; L.kL = kL; L.nL = nL; L.leaves = p->leaves;
    L.a_ptr = p->dev.a_ptr; L.a_code = p->dev.a_code; L.a_coef = p->dev.a_coef;
    L.b_ptr = p->dev.b_ptr; L.b_code = p->dev.b_code; L.b_coef = p->dev.b_coef;
    L.wsM = wsM;
    L.epi = EPI_WORKSPACE;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const double extra_a = double(p->a.row.size()) / double(p->leaves) - 1.0;
    const double extra_b = double(p->b.row.size()) / double(p->leaves) - 1.0;
    L.tile = resolve_tile(p->tile, mL, nL, kL, p->leaves, extra_a, extra_b, sms);
    if ((e = launch_leaf_gemm(L, s, &launches)) != cudaSuccess) return to_status(e);
    const bool kfringe = kp < k;
    if (kfringe && (e = launch_classical(A + kp, lda, B + kp * ldb, ldb, C, ldc, mp, k - kp, np,
                                         FMM_TILE_AUTO, s, &launches)) != cudaSuccess)
        return to_status(e);
    if ((e = launch_w_pass(C, ldc, mL, nL, int(sn), sm * sn, p->dev.cq_ptr, p->dev.cq_leaf, p->dev.cq_coef,
                           wsM, kfringe ? 1 : 0, s, &launches)) != cudaSuccess)
        return to_status(e);
    if (mp < m && (e = launch_classical(A + mp * lda, lda, B, ldb, C + mp * ldc, ldc, m - mp, k, n,
                                        FMM_TILE_AUTO, s, &launches)) != cudaSuccess)
        return to_status(e);
    if (np < n && (e = launch_classical(A, lda, B + np, ldb, C + np, ldc, mp, k, n - np,
                                        FMM_TILE_AUTO, s, &launches)) != cudaSuccess)
        return to_status(e);
    set_last_launch_count(launches);
    return FMM_OK;
}
