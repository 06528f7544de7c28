// Internal declarations shared by the host plan layer (plan.cpp), the kernels
// (fp64_kernels.cu) and the ABI entry points (api.cu).
#pragma once

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fmm.h"

namespace fmm {

// Per-leaf list of blocks with coefficients, in CSR form over the leaves.
struct TermList {
    std::vector<int64_t> ptr;   // leaves + 1
    std::vector<int32_t> row;   // block row in the grid of blocks
    std::vector<int32_t> col;   // block column
    std::vector<double> coef;   // coefficient (product over the L steps)
    int max_terms() const {
        int m = 0;
        for (size_t i = 0; i + 1 < ptr.size(); ++i)
            m = std::max<int>(m, int(ptr[i + 1] - ptr[i]));
        return m;
    }
};

// Device copy of the unrolled plan.  Operand codes: code >= 0 is a block of
// the input matrix, (row << 16) | col; code < 0 is workspace slot (-code - 1)
// holding a pre-formed S_r or T_r (write-once scheme).
struct DevicePlan {
    int *a_ptr = nullptr, *a_code = nullptr;     // fused: all terms
    double *a_coef = nullptr;
    int *b_ptr = nullptr, *b_code = nullptr;
    double *b_coef = nullptr;
    int *c_ptr = nullptr, *c_code = nullptr;     // epilogue terms per leaf
    double *c_coef = nullptr;                    // W coefficient * sA * sB
    // write-once scheme: per leaf one operand code (block or slot)
    int *ua_code = nullptr, *ub_code = nullptr;
    int *ua_ptr = nullptr, *ub_ptr = nullptr;    // CSR with one term per leaf
    double *u_one = nullptr;                     // coefficient 1.0 per leaf
    // slots of the write-once pass: leaf index and CSR into a_* / b_*
    int *sa_leaf = nullptr, *sb_leaf = nullptr;
    // per C block: CSR over (leaf, coefficient) for the write-once W pass
    int *cq_ptr = nullptr, *cq_leaf = nullptr;
    double *cq_coef = nullptr;
    // level-by-level scheme: the base [[U,V,W]] as lists
    int *lu_ptr = nullptr, *lu_code = nullptr;   // per r: A blocks (a<<16|b)
    double *lu_coef = nullptr;
    int *lv_ptr = nullptr, *lv_code = nullptr;   // per r: B blocks
    int *lvt_code = nullptr;                     // the same blocks of B^T (c<<16|b)
    double *lv_coef = nullptr;
    int *lw_ptr = nullptr, *lw_r = nullptr;      // per C block q: (r, W_qr)
    double *lw_coef = nullptr;
    int *lu_icoef = nullptr, *lv_icoef = nullptr, *lw_icoef = nullptr;  // integer base coefficients
    int *leaf_slot = nullptr;                    // code -(r+1) for every leaf
    double *c_coef_raw = nullptr;                // unscaled flattened W
    double *a_coef_raw = nullptr, *b_coef_raw = nullptr;  // unnormalised chains
    void *blob = nullptr;                        // single allocation
};

}  // namespace fmm

struct fmm_plan {
    int M = 0, K = 0, N = 0, R = 0, L = 0;
    unsigned flags = 0;
    int device = 0;
    fmm_tile tile = FMM_TILE_AUTO;
    int64_t leaves = 1;
    fmm::TermList a, b, c;                   // unscaled, as exported
    std::vector<double> U, V, W;             // the base case, row-major
    // normalised lists (first coefficient of each S_r/T_r is 1, the scale
    // folded into the epilogue coefficient)
    std::vector<double> a_norm, b_norm, c_scaled;
    int64_t slots_a = 0, slots_b = 0;        // leaves with > 1 term
    std::vector<int32_t> slot_of_leaf_a, slot_of_leaf_b;
    fmm::DevicePlan dev;                     // uploaded on first use
    std::mutex upload_mu;
    bool uploaded = false;
    int upload_device = -1;                  // device holding `dev` once uploaded
    fmm_precision prec = FMM_PREC_FP64;
    int nmod = 15;                           // moduli of the emulated-FP64 variant
    bool integer_coefs = false;              // every base coefficient an integer in [-127, 127]
};

namespace fmm {

// plan.cpp
fmm_status build_plan(fmm_plan *p, int M, int K, int N, int R, const double *U,
                      const double *V, const double *W, int levels);
fmm_status upload_plan(fmm_plan *p);
void free_plan_device(fmm_plan *p);
bool brent_exact(int M, int K, int N, int R, const double *U, const double *V,
                 const double *W, bool *representable);
fmm_status parse_fmm_file(const char *path, int *M, int *K, int *N, int *R,
                          std::vector<double> *U, std::vector<double> *V,
                          std::vector<double> *W);

// fp64_kernels.cu
struct LeafLaunch {
    const double *A; int64_t lda;
    const double *B; int64_t ldb;
    double *C; int64_t ldc;
    int64_t mL, kL, nL;
    int64_t leaves;
    const int *a_ptr; const int *a_code; const double *a_coef;
    const int *b_ptr; const int *b_code; const double *b_coef;
    const int *c_ptr; const int *c_code; const double *c_coef;
    const double *slotA; int64_t slotA_stride;   // write-once S slots (ld kL)
    const double *slotB; int64_t slotB_stride;   // write-once T slots (ld nL)
    double *wsM;                                 // leaf products (ld nL)
    int epi;                                     // EPI_* below
    int tile;                                    // fmm_tile (resolved)
    // batched products (grid z): device arrays of per-product bases, or null
    const double *const *Ab = nullptr;
    const double *const *Bb = nullptr;
    double *const *Cb = nullptr;
    int64_t batch = 1;
};
enum { EPI_STORE = 0, EPI_ATOMIC = 1, EPI_WORKSPACE = 2 };

cudaError_t launch_leaf_gemm(const LeafLaunch &a, cudaStream_t s, int *launches);
cudaError_t launch_form_slots(const double *X, int64_t ldx, int64_t rows, int64_t cols,
                              int64_t slots, const int *slot_leaf, const int *ptr,
                              const int *code, const double *coef, double *out,
                              int64_t out_stride, cudaStream_t s, int *launches);
cudaError_t launch_w_pass(double *C, int64_t ldc, int64_t mL, int64_t nL, int gridN,
                          int64_t blocks, const int *cq_ptr, const int *cq_leaf,
                          const double *cq_coef, const double *wsM, int accumulate,
                          cudaStream_t s, int *launches);
cudaError_t launch_level_form(const double *parent, int64_t parent_ld, int64_t parent_stride,
                              int64_t parents, int64_t rows, int64_t cols, int R, const int *ptr,
                              const int *code, const double *coef, double *out, cudaStream_t s,
                              int *launches);
cudaError_t launch_level_w(const double *child, int64_t rows, int64_t cols, int R, int gridN,
                           int MN, double *parent, int64_t parent_ld, int64_t parent_stride,
                           int64_t parents, const int *w_ptr, const int *w_r, const double *w_coef,
                           int accumulate, cudaStream_t s, int *launches);
cudaError_t launch_level_stream(const double *parent, int64_t parent_ld, int64_t parent_stride,
                                int64_t parents, int64_t rows, int64_t cols, int gridR, int gridC, int R,
                                const int *ptr, const int *code, const double *coef, double *out,
                                cudaStream_t s, int *launches);
cudaError_t launch_level_w_stream(const double *child, int64_t rows, int64_t cols, int R, int gridN, int MN,
                                  double *parent, int64_t parent_ld, int64_t parent_stride, int64_t parents,
                                  const int *w_ptr, const int *w_r, const double *w_coef, int accumulate,
                                  cudaStream_t s, int *launches);
cudaError_t launch_block_axpy(const double *X, int64_t xld, int64_t xstride, double *Y, int64_t yld,
                              int64_t ystride, int64_t parents, int64_t rows, int64_t cols, double c,
                              int first, cudaStream_t s, int *launches);
cudaError_t launch_classical(const double *A, int64_t lda, const double *B, int64_t ldb,
                             double *C, int64_t ldc, int64_t m, int64_t k, int64_t n,
                             int tile, cudaStream_t s, int *launches);
// api.cu: launch count reported by fmm_last_launch_count (this host thread)
void set_last_launch_count(int n);
// api.cu: CUDA event pairs around the dominant launch (fmm_timing_enable)
cudaEvent_t timing_mark(cudaStream_t s);
void timing_unmark();

// ozaki.cu
extern const int kOzakiModuli[20];
int ozaki_beta(int nmod, int64_t k);
size_t ozaki_workspace(int64_t leaves, int nmod, int64_t m, int64_t k, int64_t n);
cudaError_t ozaki_products(const double *S, int64_t lds, int64_t ss, const double *T, int64_t ldt,
                           int64_t ts, double *Out, int64_t ldo, int64_t os, int64_t leaves,
                           int64_t m, int64_t k, int64_t n, int nmod, void *ws, cudaStream_t s,
                           int *launches, int tile = FMM_TILE_AUTO);
cudaError_t read_device_error(int *flag, bool clear);
// time limit of the tensor-core kernels' bounded waits (fmm_set_wait_limit)
unsigned long long wait_limit_ns();
void set_wait_limit_ns(unsigned long long ns);
// One problem of a grouped residue GEMM launch (launch_residue_gemm_group):
// operand planes ra (S', plane_m x kpad bf16 per plane, rows [r0, r0 + m)
// used) and rb (T'^T, n x kpad), products into Z (planes of m x z_pitch(n)).
constexpr int RG_MAX_PROBLEMS = 8;   // problems per grouped residue GEMM launch
// Device address of the tensor-core kernels' error flag (g_device_error).
cudaError_t device_error_flag(int **out);
struct RgDesc {
    const void *ra, *rb;
    int8_t *Z;
    int64_t m, n, kpad, planes;
    int nmod;
    int64_t r0, plane_m;
};
cudaError_t launch_residue_gemm_group(const RgDesc *d, int count, int *err, cudaStream_t s, int *launches,
                                      bool narrow);
// kernels of the timeout tests: a wait that nothing completes runs out
cudaError_t residue_gemm_timeout_probe(unsigned long long limit_ns, cudaStream_t s);
cudaError_t tf32_gemm_timeout_probe(unsigned long long limit_ns, cudaStream_t s);
cudaError_t ozaki_prepare(int nmod);          // constant tables, kernel attributes
cudaError_t prepare_fp64_kernels();           // kernel attributes of every tile
// tf32.cu
size_t tf32_workspace(int64_t leaves, int64_t m, int64_t k, int64_t n, int split = 1);
cudaError_t tf32_prepare();
cudaError_t read_tf32_error(int *flag, bool clear);
cudaError_t tf32_products(const double *S, int64_t lds, int64_t ss, const double *T, int64_t ldt,
                          int64_t ts, double *Out, int64_t ldo, int64_t os, int64_t leaves, int64_t m,
                          int64_t k, int64_t n, int accumulate, void *ws, cudaStream_t s, int *launches,
                          int split = 1, int tile = FMM_TILE_AUTO);
// One recursive level fused with the TF32 conversion (csrc/tf32.cu): the R
// leaf products of A (gM x gK blocks of mL x kL) and B (gK x gN blocks of
// kL x nL) from the level's term lists, S and T formed in FP32 while each
// operand is read once.  Block grids of 4, 6, 8 or 9; R <= 64.
cudaError_t tf32_first_level_products(const double *A, int64_t lda, const double *B, int64_t ldb, int64_t mL,
                                      int64_t kL, int64_t nL, int gM, int gK, int gN, int R, const int *u_ptr,
                                      const int *u_code, const double *u_coef, const int *v_ptr,
                                      const int *v_code, const double *v_coef, float *Out, int64_t ldo,
                                      int64_t os, void *ws, cudaStream_t s, int *launches, int split, int tile);
// ... and the W combination of that level from its FP32 products, summed in
// FP32, into C (FP64; added when accumulate).
cudaError_t tf32_w_level(const float *P, int64_t mL, int64_t nL, int gM, int gN, const int *w_ptr, const int *w_r,
                         const double *w_coef, double *C, int64_t ldc, int accumulate, cudaStream_t s,
                         int *launches);
// residue-space recursion (integer base coefficients only)
struct ResPlan {
    int M, K, N, R, L;
    const int *u_ptr, *u_code, *u_icoef;
    const int *v_ptr, *v_code, *v_icoef;
    const int *vt_code;                      // B block codes with row and column swapped (B^T)
    const int *w_ptr, *w_r, *w_icoef;
    int w_absmax;                            // max over C blocks of sum_r |W_qr|
    int u_absmax, v_absmax;                  // max over r of sum_i |U_ir|, of sum_j |V_jr|
    int tile;                                // the plan's fmm_tile (128x128: narrow GEMM tiles)
    bool fused_s;                            // form S' inside the residue GEMM where it can
    const double *hU;                        // the base U on the host (MK x R), for that choice
};
size_t ozaki_fast_workspace(const ResPlan &rp, int64_t mp, int64_t kp, int64_t np, int nmod);
// Overlap hooks of the host entry point.  b_ready (or null): an event the
// kernels that read B wait on, so B may still be arriving from the host while
// the kernels that read only A run.  band_done (or null): the final W + CRT
// pass runs in `bands` row bands, and after each band is enqueued band_done is
// called on the host with the band's rows [r0, r1) inside each of the
// `block_rows_count` block rows of C (each `block_rows` tall); it may enqueue
// work on other streams (a copy of the band out of C).  gemm_bands > 1: with
// at most one recursive level, the residue products are made in that many
// row bands too, each combined and handed over before the next is made.
struct HostPipe {
    cudaEvent_t b_ready;
    // a_bands > 0: A arrives after B in that many bands of the first level's
    // child rows ([ml j / a_bands, ml (j + 1) / a_bands) of every block row, ml
    // the rows of a level-1 block, or of A itself with no level), band j
    // complete at a_ready[j]
    int a_bands;
    const cudaEvent_t *a_ready;
    int bands, gemm_bands;
    cudaError_t (*band_done)(void *ctx, int64_t r0, int64_t r1, int64_t block_rows, int block_rows_count);
    void *ctx;
};
// A product split around its residue GEMM, for grouped launches: phase 0
// enqueues what comes before the GEMM and fills `gemm`; phase 1 what comes
// after it (the caller launches the GEMMs of several products in between).
struct GemmDefer {
    int phase;
    RgDesc gemm;
    bool narrow;
};
cudaError_t ozaki_fast(const ResPlan &rp, const double *A, int64_t lda, const double *B, int64_t ldb,
                       double *C, int64_t ldc, int64_t mp, int64_t kp, int64_t np, int nmod,
                       int accumulate, void *ws, cudaStream_t s, int *launches,
                       const HostPipe *pipe = nullptr, GemmDefer *defer = nullptr);

int resolve_tile(int requested, int64_t mL, int64_t nL, int64_t kL, int64_t leaves,
                 double extra_a, double extra_b, int num_sms);
void tile_dims(int tile, int *bm, int *bn);

}  // namespace fmm
