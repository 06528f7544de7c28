// fmm_gemm_noalloc: the deterministic product (leaf products stored, then a
// fixed-order pass forms C) with its scratch held in a fixed static device
// array instead of caller-provided or allocated memory.
//
// Some callers cannot allocate device memory at the point where they need a
// product: code running while a CUDA graph is being captured, host runtimes
// whose device memory is reserved up front by another allocator, and paths
// that must not pay the implicit synchronisation of cudaMalloc.  This entry
// point never allocates: the unrolled plan lists and the leaf products live
// in `g_noalloc_scratch`, a file-scope array of FMM_NOALLOC_SCRATCH_BYTES that
// every GPU loading this library holds until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

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

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

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

// Host image of the lists the stored-product scheme reads, packed at the
// front of the scratch array; offsets are 256-byte aligned.
struct ListImage {
    std::vector<unsigned char> bytes;
    size_t a_ptr, a_code, a_coef, b_ptr, b_code, b_coef, cq_ptr, cq_leaf, cq_coef;
};

void build_image(const fmm_plan *p, ListImage *img) {
    const int64_t leaves = p->leaves, na = p->a.row.size(), nb = p->b.row.size(),
                  nc = p->c.row.size();
    const int64_t gridN = ipow(p->N, p->L), blocks = ipow(p->M, p->L) * gridN;
    size_t off = 0;
    auto take = [&](size_t n) { size_t o = off; off = al256(off + n); return o; };
    img->a_ptr = take((leaves + 1) * 4); img->a_code = take(na * 4); img->a_coef = take(na * 8);
    img->b_ptr = take((leaves + 1) * 4); img->b_code = take(nb * 4); img->b_coef = take(nb * 8);
    img->cq_ptr = take((blocks + 1) * 4); img->cq_leaf = take(nc * 4); img->cq_coef = take(nc * 8);
    img->bytes.assign(off, 0);
    unsigned char *h = img->bytes.data();
    int *ap = (int *)(h + img->a_ptr), *ac = (int *)(h + img->a_code);
    int *bp = (int *)(h + img->b_ptr), *bc = (int *)(h + img->b_code);
    for (int64_t r = 0; r <= leaves; ++r) { ap[r] = int(p->a.ptr[r]); bp[r] = int(p->b.ptr[r]); }
    for (int64_t t = 0; t < na; ++t) ac[t] = (p->a.row[t] << 16) | p->a.col[t];
    for (int64_t t = 0; t < nb; ++t) bc[t] = (p->b.row[t] << 16) | p->b.col[t];
    if (na) std::memcpy(h + img->a_coef, p->a_norm.data(), na * 8);
    if (nb) std::memcpy(h + img->b_coef, p->b_norm.data(), nb * 8);
    // per C block: its (leaf, scaled W coefficient) pairs in ascending leaf order
    int *qp = (int *)(h + img->cq_ptr), *ql = (int *)(h + img->cq_leaf);
    double *qc = (double *)(h + img->cq_coef);
    for (int64_t t = 0; t < nc; ++t) qp[(int64_t)p->c.row[t] * gridN + p->c.col[t] + 1]++;
    for (int64_t q = 0; q < blocks; ++q) qp[q + 1] += qp[q];
    std::vector<int> fill(qp, qp + blocks);
    for (int64_t r = 0; r < leaves; ++r) {
        const bool live = p->a.ptr[r + 1] > p->a.ptr[r] && p->b.ptr[r + 1] > p->b.ptr[r];
        for (int64_t t = p->c.ptr[r]; t < p->c.ptr[r + 1]; ++t) {
            const int64_t q = (int64_t)p->c.row[t] * gridN + p->c.col[t];
            ql[fill[q]] = int(r);
            qc[fill[q]] = live ? p->c_scaled[t] : 0.0;
            fill[q]++;
        }
    }
}

}  // namespace

extern "C" fmm_status fmm_gemm_noalloc(fmm_plan_t p, const double *A, int64_t lda,
                                       const double *B, int64_t ldb, double *C, int64_t ldc,
                                       int64_t m, int64_t k, int64_t n, void *stream) {
    using namespace fmm;
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
    if (p->L == 0 || mp == 0 || kp == 0 || np == 0)
        return to_status(launch_classical(A, lda, B, ldb, C, ldc, m, k, n, FMM_TILE_AUTO, s, &launches));

    ListImage img;
    try {
        build_image(p, &img);
    } catch (const std::bad_alloc &) {
        return FMM_ERR_NO_MEMORY;
    }
    const size_t prod_off = al256(img.bytes.size());
    const size_t need = prod_off + size_t(p->leaves) * size_t(mL) * size_t(nL) * 8;
    if (need > size_t(FMM_NOALLOC_SCRATCH_BYTES)) return FMM_ERR_UNSUPPORTED;

    void *base = nullptr;
    fmm_status st = scratch_address(&base);
    if (st != FMM_OK) return st;
    unsigned char *d = (unsigned char *)base;
    cudaError_t e = cudaMemcpyAsync(d, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return to_status(e);
    double *wsM = (double *)(d + prod_off);

    LeafLaunch L{};
    L.A = A; L.lda = lda; L.B = B; L.ldb = ldb; L.C = C; L.ldc = ldc;
    L.mL = mL; L.kL = kL; L.nL = nL; L.leaves = p->leaves;
    L.a_ptr = (const int *)(d + img.a_ptr); L.a_code = (const int *)(d + img.a_code);
    L.a_coef = (const double *)(d + img.a_coef);
    L.b_ptr = (const int *)(d + img.b_ptr); L.b_code = (const int *)(d + img.b_code);
    L.b_coef = (const double *)(d + img.b_coef);
    L.wsM = wsM;
    L.epi = EPI_WORKSPACE;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const double extra_a = double(p->a.row.size()) / double(p->leaves) - 1.0;
    const double extra_b = double(p->b.row.size()) / double(p->leaves) - 1.0;
    L.tile = resolve_tile(p->tile, mL, nL, kL, p->leaves, extra_a, extra_b, sms);
    if ((e = launch_leaf_gemm(L, s, &launches)) != cudaSuccess) return to_status(e);
    const bool kfringe = kp < k;
    if (kfringe && (e = launch_classical(A + kp, lda, B + kp * ldb, ldb, C, ldc, mp, k - kp, np,
                                         FMM_TILE_AUTO, s, &launches)) != cudaSuccess)
        return to_status(e);
    if ((e = launch_w_pass(C, ldc, mL, nL, int(sn), sm * sn, (const int *)(d + img.cq_ptr),
                           (const int *)(d + img.cq_leaf), (const double *)(d + img.cq_coef),
                           wsM, kfringe ? 1 : 0, s, &launches)) != cudaSuccess)
        return to_status(e);
    if (mp < m && (e = launch_classical(A + mp * lda, lda, B, ldb, C + mp * ldc, ldc, m - mp, k, n,
                                        FMM_TILE_AUTO, s, &launches)) != cudaSuccess)
        return to_status(e);
    if (np < n && (e = launch_classical(A, lda, B + np, ldb, C + np, ldc, mp, k, n - np,
                                        FMM_TILE_AUTO, s, &launches)) != cudaSuccess)
        return to_status(e);
    return FMM_OK;
}
