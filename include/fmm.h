/*
 * fmm.h - C ABI of the GB300 recursive fast matrix multiplication library.
 *
 * Method (Benson & Ballard, "A Framework for Practical Parallel Fast Matrix
 * Multiplication"): a base case <M,K,N;R> with factor matrices [[U,V,W]]
 * (Section 2.2, Eq. 2) multiplies an M x K block matrix A by a K x N block
 * matrix B with R block products.  One recursive step forms
 *     S_r = sum_i U_ir A_i,   T_r = sum_j V_jr B_j,          (Section 3.1)
 *     M_r = S_r T_r,          C_q = sum_r W_qr M_r,
 * and L steps are applied recursively before the classical product takes
 * over at the leaves (Section 3.4).  Dimensions that the block sizes do not
 * divide are handled by peeling (Section 3.5).
 *
 * Conventions for every entry point
 *   - Matrices are row-major with a leading dimension (ld >= columns);
 *     A is m x k, B is k x n, C is m x n.  U, V, W are row-major host arrays
 *     of MK x R, KN x R, MN x R whose rows follow the row-order vectorisation
 *     of the A, B and C blocks (Section 2.2.2: block (a,b) of A is row a*K+b).
 *   - C = A B overwrites C (no alpha/beta).  C must not overlap A or B.
 *   - "device pointer" arguments are CUDA global-memory addresses on the
 *     device that was current when the plan was created; the caller owns
 *     them.  Work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 *     default stream) and is asynchronous unless stated otherwise.
 *   - Every argument is validated on the host before any launch; no
 *     exception crosses the ABI.  Non-finite inputs are unsupported (fast
 *     algorithms may turn Inf into NaN through Inf - Inf).
 *   - A plan is immutable after creation and may be used from several host
 *     threads and streams at once.
 */
#ifndef FMM_H_
#define FMM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_plan *fmm_plan_t; /* opaque; owned by the library */

typedef enum {
    FMM_OK = 0,
    FMM_ERR_ARG = -1,               /* bad pointer, size, stride or aliasing  */
    FMM_ERR_INVALID_ALGORITHM = -2, /* [[U,V,W]] fails the Brent equations    */
    FMM_ERR_UNSUPPORTED = -3,       /* valid request the library cannot run   */
    FMM_ERR_NO_MEMORY = -4,         /* host or device allocation failed, or
                                       the workspace passed is too small      */
    FMM_ERR_CUDA = -5,              /* a CUDA call failed                     */
    FMM_ERR_TIMEOUT = -6            /* a bounded device wait gave up          */
} fmm_status;

typedef enum {
    FMM_PREC_FP64 = 0,       /* FP64 leaves (DFMA), FP64 combinations */
    /* Leaf products emulated to FP64 accuracy on the tensor cores: the
       operands are scaled per row (A or S) / column (B or T) by powers of two
       and truncated to beta-bit integers, the integer product is computed
       exactly modulo N pairwise coprime moduli <= 256 with bfloat16 residues
       and FP32 accumulation (tcgen05), and rebuilt by the Chinese remainder
       theorem, rounded once to FP64.  beta is the largest width <= 62 with
       k 2^(2 beta + 1) < P, P the product of the moduli (an exact integer
       search; about 51 bits for N = 15, k = 16384).
       With integer base coefficients (every shipped algorithm) the whole
       recursion runs on residues of the once-scaled A and B: S/T formation
       and the W combination are exact modular arithmetic on the residues, and
       only the scaling and the final CRT rounding touch FP64 values.  With
       other coefficients, or with FMM_FLAG_LEAF_EMULATION, each leaf product
       is emulated on its own and S/T formation and the W combination run in
       FP64.  The fringe (Section 3.5) is a classical FP64 product. */
    FMM_PREC_OZAKI_BF16 = 3,
    /* Leaf products on the tensor cores in TF32 (operands rounded to a
       10-bit significand, FP32 accumulation).  With one recursive level
       (block grids of 4, 6, 8 or 9 blocks, R <= 64) S and T are formed in
       FP32 while each FP64 operand is read once (each block value rounded
       to FP32), the leaf products are kept in FP32 and the W combination is
       summed in FP32 into C (a few units of 2^-24 in all; small integers
       stay exact while every sum stays below 2^24); deeper plans form S/T
       and W in FP64 from FP64 products.  The fringe is FP64.  Relative
       error of order 2^-11 per leaf operand. */
    FMM_PREC_TF32 = 2,
    /* FP32-accurate leaf products on the same TF32 tensor path: each leaf
       operand x (taken in FP32) is split into x_hi = tf32(x) and x_lo =
       tf32(x - x_hi), and one product over three K segments sums
       S_hi T_hi + S_hi T_lo + S_lo T_hi with FP32 accumulation (three times
       the TF32 work; the dropped S_lo T_lo is 2^-22 relative).  S/T
       formation, the products' precision and the W combination as for
       FMM_PREC_TF32 (FP32 with one level, else FP64); the fringe is FP64. */
    FMM_PREC_FP32 = 1
} fmm_precision;

/* Execution-scheme flags (fmm_plan_create / fmm_plan_load `flags`). */
enum {
    /* S_r and T_r are formed inside the leaf kernel's shared-memory operand
       staging (never written to HBM); when clear they are formed by a
       write-once pass into the workspace first (Section 3.2). */
    FMM_FLAG_FUSED_ST = 1u << 0,
    /* W is applied in the leaf kernel's epilogue by FP64 reductions into C
       (summation order across leaves not fixed; exact on integer data); when
       clear the leaf products M_r go to the workspace and a write-once pass
       forms C in a fixed order (bitwise reproducible). */
    FMM_FLAG_FUSED_W = 1u << 1,
    /* With FUSED_ST and/or FUSED_W clear: form the unfused parts one
       recursive level at a time, as the recursion of Section 3.1 does (the
       S_r of level l are combinations of the level l-1 S_r, and C blocks of
       level l-1 are combined from the level-l products), instead of from the
       fully unrolled per-leaf chains.  Needs more workspace, but the addition
       count grows like sum_l R^(l-1) nnz rather than nnz^L. */
    FMM_FLAG_LEVELWISE = 1u << 2,
    /* Emulated-precision plans only: emulate each leaf product separately
       (S/T and W in FP64) instead of running the whole recursion on residues
       of the once-scaled A and B (the default when every base coefficient
       is an integer: the bilinear algorithm is then exact modulo p). */
    FMM_FLAG_LEAF_EMULATION = 1u << 3,
    /* Addition schemes of the level-by-level passes (Section 3.2), for the
       parts FMM_FLAG_LEVELWISE forms outside the leaf kernel (FP64 plans, and
       TF32 plans deeper than one level): by default each child S_r, T_r or C block is written once from
       all its terms ("write-once").  STREAMING reads each parent element
       once and writes it into every child that uses it; PAIRWISE forms each
       child by one pass per term (child = c x, then child += c x).  All three
       do the same additions in the same order and give the same bits.  At
       most one of the two flags; base cases with more than 512 terms in a
       factor matrix, R > 128 or more than 64 blocks fall back to write-once
       for STREAMING. */
    FMM_FLAG_STREAMING = 1u << 4,
    FMM_FLAG_PAIRWISE = 1u << 5,
    /* Emulated-FP64 plans in residue space with at most one recursive level
       (or none): form each leaf's S' inside the tensor-core GEMM from the int8
       residues of A' (converter warps combine the leaf's one or two blocks and
       store the fp16 operand in tensor memory, which tcgen05 reads as its A
       operand), so no S' operand plane is written to HBM; T' comes from fp16
       planes.  Used where every leaf's S' has at most two terms with
       sum |c| <= 2 and the k blocks are multiples of 16; otherwise ignored.
       Same integers, so the same result bit for bit. */
    FMM_FLAG_TC_FUSED_S = 1u << 6,
    FMM_FLAGS_DEFAULT = FMM_FLAG_FUSED_ST | FMM_FLAG_FUSED_W
};

/* Tile shape of the leaf GEMM kernel (fmm_plan_set_tile). */
typedef enum {
    FMM_TILE_AUTO = 0,
    FMM_TILE_128x128 = 1,
    FMM_TILE_96x96 = 2,
    FMM_TILE_64x64 = 3,
    FMM_TILE_32x32 = 4,
    FMM_TILE_128x64 = 5,
    FMM_TILE_64x128 = 6
} fmm_tile;

/*
 * fmm_plan_create - build a plan for `levels` recursive steps of the base
 * case <M,K,N;R> given by U (MK x R), V (KN x R), W (MN x R).
 *
 * The factor matrices are checked exactly against the Brent equations
 * (Eq. 2, with the matmul tensor of Section 2.2.2); FP64 values are exact
 * dyadic rationals, so the check has no rounding.  The L steps are then
 * unrolled into R^L leaf products (Section 3.1 applied recursively), each
 * with its list of A blocks, B blocks and C blocks and their coefficients,
 * and the lists are copied to the current device.
 *
 * levels: 0..6 (0 = classical product).  M, K, N: 1..16; R: 1..1024.
 * out: receives the plan; unchanged on error.
 * Errors: FMM_ERR_ARG (null pointer, sizes out of range, levels out of range,
 * unknown flags, STREAMING with PAIRWISE), FMM_ERR_INVALID_ALGORITHM (Brent
 * check failed),
 * FMM_ERR_UNSUPPORTED (R^L or the unrolled term lists too large, or a
 * coefficient that is not finite), FMM_ERR_NO_MEMORY, FMM_ERR_CUDA.
 */
fmm_status fmm_plan_create(fmm_plan_t *out, int M, int K, int N, int R,
                           const double *U, const double *V, const double *W,
                           int levels, fmm_precision prec, unsigned flags);

/*
 * fmm_plan_load - as fmm_plan_create, reading [[U,V,W]] from a text file:
 * optional '#' comments, a line "M K N R", then lines "U", "V", "W" each
 * followed by MK, KN, MN rows of R rationals written as p or p/q.
 * Denominators must be powers of two (exact in FP64); others give
 * FMM_ERR_UNSUPPORTED.  A file that cannot be read or parsed gives
 * FMM_ERR_ARG.
 */
fmm_status fmm_plan_load(fmm_plan_t *out, const char *fmm_file, int levels,
                         fmm_precision prec, unsigned flags);

/* Release a plan and its device memory.  NULL is a no-op.  The caller must
   make sure no work using the plan is still running. */
void fmm_plan_destroy(fmm_plan_t plan);

/* Number of moduli N (3..16, default 15) of an FMM_PREC_OZAKI_BF16 plan;
   more moduli give more bits (beta grows by about 4 per modulus) and cost
   one more residue GEMM each.  FMM_ERR_ARG outside the range or for an FP64
   plan.  Not thread-safe against concurrent fmm_gemm calls on the plan. */
fmm_status fmm_plan_set_moduli(fmm_plan_t plan, int n_moduli);

/* Synchronise the current device and report whether any bounded device-side
   wait of this library gave up since the last call (FMM_ERR_TIMEOUT; the
   flag is then cleared), FMM_OK otherwise, FMM_ERR_CUDA if the device
   reports an error. */
fmm_status fmm_check_device_error(void);

/* Time limit, in nanoseconds of the GPU's global timer, of every bounded
   device-side wait in the tensor-core kernels (the emulated-FP64 residue
   GEMM and the TF32 GEMM) launched after this call; default 2e9 (2 s).  A
   kernel whose wait runs out stops issuing work, waits (with the same limit)
   for the copies and MMAs it already issued, frees its tensor memory and
   returns; fmm_check_device_error then reports FMM_ERR_TIMEOUT and the
   product's result is undefined.  Process-wide.
   Errors: FMM_ERR_ARG for 0. */
fmm_status fmm_set_wait_limit(uint64_t ns);

/* Self-test of that timeout path: launches one CTA of the chosen kernel
   (0 = residue GEMM, 1 = TF32 GEMM) on small private buffers with its load
   and MMA threads told to issue nothing, so its first wait for a finished
   accumulator runs out after `ns` nanoseconds with no copy or MMA
   outstanding.  Synchronises `stream`, then reads and clears the device
   error flag: FMM_ERR_TIMEOUT is the expected answer (the wait ran out and
   the kernel returned), FMM_OK would mean it did not.  The CUDA context stays
   usable.  Errors: FMM_ERR_ARG (kernel not 0 or 1, ns = 0), FMM_ERR_CUDA,
   FMM_ERR_NO_MEMORY. */
fmm_status fmm_selftest_wait_timeout(int kernel, uint64_t ns, void *stream);

/* Copy the plan to the current device and set up everything its kernels
   need (constant tables, kernel attributes) now, instead of on the first
   fmm_gemm call; afterwards fmm_gemm with this plan performs no allocation or
   synchronous copy, so it can be captured into a CUDA graph.  Errors:
   FMM_ERR_ARG, FMM_ERR_NO_MEMORY, FMM_ERR_CUDA. */
fmm_status fmm_plan_prepare(fmm_plan_t plan);

/* Choose the leaf GEMM tile shape used by later fmm_gemm calls with this
   plan (default FMM_TILE_AUTO).  FP64 plans: the FP64 leaf kernel's CTA tile.
   Tensor-core plans (emulated FP64, TF32, FP32): FMM_TILE_128x128 narrows the
   tensor-core GEMM's tiles from 128 x 256 to 128 x 128 (two TMEM accumulators
   of 128 columns, more CTAs for narrow or few leaves); any other value keeps
   128 x 256 wherever the leaves are at least 256 wide.  Not thread-safe
   against concurrent fmm_gemm calls on the same plan. */
fmm_status fmm_plan_set_tile(fmm_plan_t plan, fmm_tile tile);

/* Description of a plan (fmm_plan_info). */
typedef struct {
    int M, K, N, R, levels;
    unsigned flags;
    int64_t leaves;        /* R^levels                                      */
    int64_t nnz_a_terms;   /* sum over leaves of A blocks in S_r            */
    int64_t nnz_b_terms;   /* ... B blocks in T_r                           */
    int64_t nnz_c_terms;   /* ... C blocks that M_r contributes to          */
    int max_a_terms, max_b_terms, max_c_terms; /* largest per-leaf list     */
} fmm_plan_info_t;

fmm_status fmm_plan_info(fmm_plan_t plan, fmm_plan_info_t *info);

/*
 * fmm_plan_leaf_terms - copy out the unrolled coefficient lists (for
 * verification).  For operand `which` (0 = A/U, 1 = B/V, 2 = C/W):
 *   ptr[leaves+1]   CSR row pointers into the term arrays,
 *   row[nnz], col[nnz]  block coordinates in the M^L x K^L (A), K^L x N^L (B)
 *                   or M^L x N^L (C) grid of blocks,
 *   coef[nnz]       the unscaled coefficient prod_l U[i_l, r_l] (resp. V, W).
 * Any output pointer may be NULL; `capacity` is the length of row/col/coef.
 * Leaf r = sum_l r_l R^(L-l) with r_1 the outermost step.
 * Errors: FMM_ERR_ARG (bad `which`, capacity too small).
 */
fmm_status fmm_plan_leaf_terms(fmm_plan_t plan, int which, int64_t *ptr,
                               int32_t *row, int32_t *col, double *coef,
                               int64_t capacity);

/*
 * fmm_workspace_size - device workspace bytes fmm_gemm needs for an
 * m x k x n product with this plan (0 when the fused scheme needs none).
 */
fmm_status fmm_workspace_size(fmm_plan_t plan, int64_t m, int64_t k, int64_t n,
                              size_t *bytes);

/*
 * fmm_gemm - C = A B with the plan's fast algorithm on the device.
 *
 * A (m x k, lda), B (k x n, ldb), C (m x n, ldc): device pointers, FP64,
 * row-major; 8-byte aligned.  m, k, n >= 1.  lda >= k, ldb >= n, ldc >= n.
 * The core m' x k' x n' (m' the largest multiple of M^L not above m, etc.)
 * runs the fast algorithm; the rest is added by classical products
 * (Section 3.5):  C[:m',:n'] += A[:m',k':] B[k':,:n'],  C[m':,:] = A[m':,:] B,
 * C[:m',n':] = A[:m',:] B[:,n'].
 * workspace: device pointer of at least fmm_workspace_size() bytes, 256-byte
 * aligned (may be NULL when that size is 0).
 * Errors: FMM_ERR_ARG (null plan or pointers, sizes < 1, ld too small,
 * misaligned pointers, C overlapping A or B), FMM_ERR_NO_MEMORY (workspace
 * too small), FMM_ERR_CUDA (launch failure).
 */
fmm_status fmm_gemm(fmm_plan_t plan, const double *A, int64_t lda,
                    const double *B, int64_t ldb, double *C, int64_t ldc,
                    int64_t m, int64_t k, int64_t n, void *workspace,
                    size_t ws_bytes, void *stream);

/*
 * fmm_gemm_batched - `count` independent products C_b = A_b B_b of one shape
 * with one plan, all R^L leaves of all products in ONE grouped leaf launch
 * (S/T formed in the leaf kernel, W applied by FP64 reductions into C,
 * whatever the plan's scheme flags say; FP64 plans only).
 *
 * A, B, C: HOST arrays of `count` device pointers (each as in fmm_gemm,
 * sharing lda, ldb, ldc); count 1..65535.  C_b may not overlap any A or B.
 * workspace: at least fmm_workspace_size_batched() bytes, 256-byte aligned;
 * it receives a device copy of the pointer arrays.  Fringe products of
 * shapes the block sizes do not divide are launched per product.
 * Errors: as fmm_gemm; FMM_ERR_UNSUPPORTED for an emulated-precision plan.
 */
fmm_status fmm_workspace_size_batched(fmm_plan_t plan, int64_t count, int64_t m,
                                      int64_t k, int64_t n, size_t *bytes);
fmm_status fmm_gemm_batched(fmm_plan_t plan, int64_t count,
                            const double *const *A, int64_t lda,
                            const double *const *B, int64_t ldb,
                            double *const *C, int64_t ldc, int64_t m, int64_t k,
                            int64_t n, void *workspace, size_t ws_bytes,
                            void *stream);

/*
 * fmm_gemm_grouped - `count` independent products C_i = A_i B_i of any
 * shapes, each with its own plan, issued together on `stream`.  The residue
 * GEMMs of the emulated-FP64 products whose plans run in residue space with at
 * most one recursive level (or none) go into grouped tensor-core launches of
 * up to 8 products each (one persistent launch over all their tiles, which
 * fills the GPU where a single small product cannot); every other step, and
 * every other product, runs as fmm_gemm would run it.  Each result is the
 * same, bit for bit, as fmm_gemm's for that product alone.
 *
 * plans, A, lda, B, ldb, C, ldc, m, k, n, ws, ws_bytes: HOST arrays of
 * `count` entries, each entry as the matching argument of fmm_gemm (ws[i] of
 * at least fmm_workspace_size(plans[i], m[i], k[i], n[i]) bytes; the C_i
 * may not overlap each other or any operand).  count 1..4096.
 * Errors: as fmm_gemm, checked for every product before anything runs.
 */
fmm_status fmm_gemm_grouped(int64_t count, const fmm_plan_t *plans,
                            const double *const *A, const int64_t *lda,
                            const double *const *B, const int64_t *ldb,
                            double *const *C, const int64_t *ldc,
                            const int64_t *m, const int64_t *k, const int64_t *n,
                            void *const *ws, const size_t *ws_bytes, void *stream);

/*
 * fmm_classical_gemm - C = A B by the library's classical FP64 GEMM (the
 * same kernel the leaves use; the comparator of Section 5).  Same pointer,
 * size and error rules as fmm_gemm; needs no plan and no workspace.
 */
fmm_status fmm_classical_gemm(const double *A, int64_t lda, const double *B,
                              int64_t ldb, double *C, int64_t ldc, int64_t m,
                              int64_t k, int64_t n, void *stream);

/*
 * fmm_host_workspace_size / fmm_gemm_host - end-to-end variant taking HOST
 * matrices: copies A and B to the device, runs fmm_gemm (or the classical
 * GEMM when plan is NULL), copies C back, and returns when C is on the host.
 * Host buffers should be page-locked for full copy speed.  dev_ws is a
 * device buffer of at least fmm_host_workspace_size() bytes, 256-byte
 * aligned, holding the device copies and the plan's workspace.
 * Work is issued on `stream` and on one internal stream per calling thread
 * and device, which copies B in first and then A in row bands.  For the
 * emulated-FP64 residue path without a fringe, the kernels that read B run
 * while A arrives, each band of A is formed once it is in (with the products
 * made in row bands: just before the first product band that reads it), and
 * C is copied out in row bands while the following bands are computed.  On return
 * (success or error) nothing the call issued is still in flight.
 */
fmm_status fmm_host_workspace_size(fmm_plan_t plan, int64_t m, int64_t k,
                                   int64_t n, size_t *bytes);
/*
 * fmm_set_host_pipeline - depth of that overlap for later fmm_gemm_host calls
 * on the calling thread: C leaves in `bands` row bands, and (emulated FP64 at
 * most one recursive level deep, no fringe) the residue products are made in
 * `gemm_bands` row bands, each combined and copied out while the next band
 * is multiplied.  0 for either: chosen from the sizes.  The result does not
 * depend on either count.
 * Errors: FMM_ERR_ARG for a count below 0 or above 64.
 */
fmm_status fmm_set_host_pipeline(int bands, int gemm_bands);
fmm_status fmm_gemm_host(fmm_plan_t plan, const double *A, int64_t lda,
                         const double *B, int64_t ldb, double *C, int64_t ldc,
                         int64_t m, int64_t k, int64_t n, void *dev_ws,
                         size_t ws_bytes, void *stream);

/*
 * fmm_gemm_noalloc - C = A B like fmm_gemm, for callers that cannot allocate
 * device memory when they need a product.  The paper has no counterpart.
 *
 * Who needs it: programs whose device memory is all reserved up front by
 * another allocator (a framework's caching allocator, or a pool sized at
 * start-up), where a cudaMalloc at call time fails or competes with that
 * pool, and code that may not call into the CUDA allocator on its hot path
 * at all.  The call allocates no device or host memory, takes no workspace
 * and copies nothing from the host.  It runs the stored-product scheme (leaf
 * products M_r kept, then C formed in a fixed order, bitwise reproducible)
 * with S_r/T_r formed in the leaf kernel; the plan's own scheme flags are
 * ignored.  Its only scratch, the leaf products, is one file-scope device
 * array of FMM_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU loading this
 * library holds until the process exits.
 *
 * Precondition: the plan's lists are already on the current device
 * (fmm_plan_prepare, or any earlier fmm_gemm with this plan, made with this
 * device current); otherwise FMM_ERR_ARG, since uploading them would
 * allocate.  The first call on a device looks up the scratch array's device
 * address with that device current.
 *
 * Limit: R^L * (m'/M^L) * (n'/N^L) * 8 bytes of leaf products must fit in
 * FMM_NOALLOC_SCRATCH_BYTES; larger problems return FMM_ERR_UNSUPPORTED
 * before anything is enqueued.  Products that take the classical path (no
 * fast core) need no scratch.
 *
 * Every call uses the same array, which keeps whatever the last call left
 * (each call writes all of it that it reads), so calls whose GPU work
 * overlaps - on different streams or host threads - race and must be
 * serialised by the caller.  fmm_last_launch_count reports this call's
 * launches.  Pointer, size and error rules are those of fmm_gemm.
 */
#define FMM_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
fmm_status fmm_gemm_noalloc(fmm_plan_t plan, const double *A, int64_t lda,
                            const double *B, int64_t ldb, double *C, int64_t ldc,
                            int64_t m, int64_t k, int64_t n, void *stream);

/* Number of CUDA kernel launches the last fmm_gemm, fmm_gemm_batched,
   fmm_gemm_noalloc, fmm_gemm_host or fmm_classical_gemm call on this host
   thread enqueued (for launch accounting). */
int fmm_last_launch_count(void);

/*
 * Kernel timing for benchmarks.  While enabled on a host thread, each
 * fmm_gemm / fmm_classical_gemm call made from that thread records a CUDA
 * event pair around its leaf-product launch on the call's stream (up to 1024
 * calls are kept).  fmm_timing_leaf_ms waits for the recorded events and
 * returns the summed milliseconds and the number of calls, then clears the
 * record.  Errors: FMM_ERR_ARG (null output), FMM_ERR_CUDA.
 */
fmm_status fmm_timing_enable(int on);
fmm_status fmm_timing_leaf_ms(double *total_ms, int *count);

/* Static string for a status code. */
const char *fmm_status_string(fmm_status status);

#ifdef __cplusplus
}
#endif

#endif /* FMM_H_ */
