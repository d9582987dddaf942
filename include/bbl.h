/*
 * bbl.h - C ABI of the GB300 bootstrapped block Lanczos eigensolver.
 *
 * Method: Zbikowski & Johnson, "Bootstrapped Block Lanczos for
 * large-dimension eigenvalue problems" (arXiv 2210.15763), Sec. II.
 * The solver finds the nev algebraically smallest eigenpairs of a large,
 * sparse, real symmetric matrix H by block Lanczos with full
 * reorthogonalisation, started from a pivot block that is random or
 * "bootstrapped" from a truncated space.
 *
 * Conventions for every entry point
 *  - Every function returns a bbl_status; nothing throws across the ABI.
 *    On failure bbl_last_error() returns a thread-local message.
 *  - Argument errors are detected on the host before any kernel launch.
 *  - "device pointer" = memory allocated by the caller with cudaMalloc (or by
 *    torch) on the current device; "host pointer" = ordinary host memory.
 *    Pointers documented "host or device" are classified with
 *    cudaPointerGetAttributes.
 *  - Blocks of vectors are n x b ROW-MAJOR (the b values of one row are
 *    contiguous), the layout of the paper's W^T (Sec. II.B, Eqs. 3-5).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    ordered on that stream; functions that return results in host memory
 *    synchronise it before returning.
 *  - The caller owns every pointer it passes; the library owns (and frees in
 *    the matching destroy call) everything it allocates.
 *  - Matrix values are given in FP64 or FP32; the storage precision of the
 *    device copy is chosen at creation (FP64, or FP32 for the mixed-precision
 *    form).  Column indices are int32 (n < 2^31), row pointers int64.
 */
#ifndef BBL_H
#define BBL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BBL_OK = 0,
    BBL_ERR_INVALID_ARG = 1,    /* bad size, pointer, option or CSR structure      */
    BBL_ERR_NOT_SYMMETRIC = 2,  /* symmetry check requested and failed             */
    BBL_ERR_OOM = 3,            /* a device allocation failed                      */
    BBL_ERR_CUDA = 4,           /* a CUDA runtime error (message has the details)  */
    BBL_ERR_NOT_CONVERGED = 5,  /* basis full before the tolerance was met; the
                                   best Ritz pairs so far are still returned       */
    BBL_ERR_NUMERICAL = 6,      /* NaN / Inf or an unrecoverable breakdown         */
    BBL_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up              */
    BBL_ERR_UNSUPPORTED = 8     /* valid request this build does not implement     */
} bbl_status;

typedef enum { BBL_FP64 = 0, BBL_FP32 = 1 } bbl_dtype;
typedef enum { BBL_CSR = 0, BBL_SELL = 1, BBL_KRON = 2, BBL_TILED = 3 } bbl_format;

typedef struct bbl_matrix bbl_matrix;   /* opaque, library-owned device copy of H */

/* Solver options (Sec. II.B; defaults from bbl_options_default). */
typedef struct {
    double tol;                 /* converged when every one of the nev lowest Ritz
                                   pairs has ||H x - theta x||_2 <= tol*||H||_inf
                                   (default 1e-8)                                  */
    int max_vectors;            /* basis capacity; J_max = max_vectors / b blocks
                                   (default 2000)                                  */
    int criterion;              /* 0: residual estimate ||B_j s_i[last b]||_2;
                                   1: rms change of the nev lowest Ritz values
                                   below rms_tol (the paper's Sec. III.A test)     */
    double rms_tol;             /* for criterion 1 (default 1e-6)                  */
    uint64_t seed;              /* random pivot and deflation vectors (splitmix64) */
    double defl_tol;            /* a new column whose orthogonal part is below
                                   defl_tol*||H||_inf is deflated (default 1e-10;
                                   1e-6 is used for FP32 storage if left at 0)     */
    int storage;                /* bbl_dtype of the Lanczos blocks: BBL_FP64, or
                                   BBL_FP32 (mixed precision: FP32 blocks and SpMM,
                                   FP64 coefficients, Gram, T, residual).  Must
                                   match the matrix storage.                       */
    int polish;                 /* FP32 storage only: 1 (default) restarts block
                                   Lanczos from the FP32 Ritz vectors to reach
                                   `tol`, with float-float blocks (pairs of FP32
                                   numbers, ~48-bit significands, products on the
                                   FP32 pipes) and FP64 coefficients, Gram and T;
                                   2: the same restart with FP64 blocks and FP64
                                   arithmetic (on an FP64 copy of the values when
                                   bbl_matrix_create kept one); 0: no polish.
                                   The reported residuals are FP64 products.      */
    double stage1_tol;          /* FP32 stage tolerance when polishing (default 2e-6) */
    int check_every;            /* k > 0: Ritz solve (convergence test) after every
                                   k-th block; 0 (default): adaptive, from the decay
                                   rate of the last two residual estimates the next
                                   test is placed at half the predicted distance to
                                   convergence (at most 8 blocks ahead), so that the
                                   run stops at most a few blocks after the first
                                   block that passes.  The rms-change criterion
                                   always tests every block.                       */
    void* stream;               /* cudaStream_t                                    */
    int ritz_overlap;           /* 1 (default): the Ritz solve of block j runs on a
                                   second stream while block j+1 is formed (one
                                   speculative block at the end); 2: the same, but
                                   block j+1's Gram-Schmidt waits for it (it
                                   overlaps the SpMM only); 0: on `stream`, read
                                   before the next block                           */
    int half_first_pass;        /* FP32 storage with b = 8: 1 (default) the first
                                   Gram-Schmidt pass of the FP32 stage reads an
                                   FP16 copy of the basis (it only has to remove
                                   the bulk; the FP32 second pass removes the
                                   rest and A_j sums both passes' coefficients);
                                   0: both passes read the FP32 basis             */
    int restart_keep;           /* thick restart (Sec. II.A: the remedy for storing
                                   every Lanczos vector).  0 (default): none -- a
                                   stage that fills max_vectors stops with
                                   BBL_ERR_NOT_CONVERGED.  k > 0: when the basis is
                                   full, keep the k lowest Ritz vectors and the
                                   newest block and go on (k a multiple of b,
                                   nev <= k <= 16, k + 2b <= max_vectors; the
                                   polish stage, of block size nev, keeps
                                   k rounded up to a multiple of nev).  The kept
                                   vectors are rotated so that the projected
                                   matrix stays block tridiagonal.              */
    int max_blocks;             /* with restart_keep: cap on the blocks (SpMM
                                   calls) of a stage; 0 (default) = 10000        */
    int fused_update_gram;      /* FP32 blocks with b = 8 and at most 128 stored
                                   blocks: 1 the first pass's update and the
                                   second pass's Gram run as one kernel on the
                                   tensor cores, reading the basis once
                                   (bbl_block_update_gram); 0 (default): two
                                   kernels on the FP32 pipes, which are faster
                                   at n = 2e6 (the fused kernel's 16-row
                                   chunks are latency-bound)                     */
    int narrow_old_updates;      /* with half_first_pass (FP32 blocks, b = 8): 1
                                   (default) both passes' updates read the
                                   blocks older than the two newest from the
                                   FP16 copy (their coefficients are of the
                                   order of the lost orthogonality and of the
                                   first pass's FP16 Gram error, so the FP16
                                   rounding changes W far below its FP32
                                   rounding; bbl_block_update_f16old); 0 reads
                                   every block in FP32.  Off after a thick
                                   restart (restart_keep > 0), whose kept
                                   blocks carry large coefficients.             */
} bbl_options;

typedef struct {
    int iters;                  /* block iterations (SpMM calls) in the main stage,
                                   over all thick restarts                        */
    int vec_equiv_iters;        /* iters * b (Sec. III.A's vector-equivalent count) */
    int polish_iters;           /* FP64 block iterations of the polish stage       */
    int deflations;
    int converged;
    double t_spmm_ms, t_reorth_ms, t_cholqr_ms, t_ritz_ms, t_other_ms, t_total_ms;
    double spmm_bytes;          /* algorithmic bytes of one SpMM of the main stage */
    double spmm_gbs;            /* spmm_bytes * iters / t_spmm                     */
    double ns_per_op;           /* t_spmm / (nnz * b * iters)  (Tables I-II)       */
    double ortho_err;           /* max |V^T V - I| over the final basis (if measured) */
    double spmm_bytes_total;    /* algorithmic bytes of every SpMM of the call     */
    double reorth_bytes_total;  /* algorithmic bytes of every Gram-Schmidt pass:
                                   per pass 2*n*m*s + 3*n*b*s (m basis columns;
                                   an FP16 first-pass Gram counts n*m*s/2 less)    */
    int ritz_solves;            /* Ritz solves (convergence tests) of all stages   */
    int gram_calls;             /* main stage: first-pass Gram products C1 = Q^T W */
    double t_gram_ms;           /* their time (split-K kernel + partial reduction) */
    double gram_bytes_total;    /* their algorithmic bytes: (n*m + n*b)*s each
                                   (n*m*2 + n*b*4 when read from the FP16 copy)    */
    int spmm_calls;             /* main stage SpMM launches (spmm_gbs is over them) */
    int restarts;               /* thick restarts of all stages                   */
    int graph_kernels;          /* batched form: kernels in one captured block
                                   iteration                                      */
} bbl_stats;

void bbl_options_default(bbl_options* opt);
const char* bbl_last_error(void);
const char* bbl_status_string(bbl_status s);
int bbl_version(void);
/* Measured fused multiply-add rate of the current GPU in FLOP/s (2 per
 * FMA) for BBL_FP32 or BBL_FP64 arithmetic: independent FMA chains on every
 * SM, best of three timed launches.  No counterpart in the paper: it backs
 * the precision choices (FP64 arithmetic runs at a small fraction of the
 * FP32 rate on this GPU).  Synchronises `stream`.                         */
bbl_status bbl_probe_fma_rate(bbl_dtype dtype, double* flops_per_s, void* stream);
/* Number of kernels this library has launched in the process so far. */
uint64_t bbl_kernel_launches(void);
/* Workspace cache.  The Lanczos bases (bbl_solve, bbl_pivot_bootstrap,
 * bbl_batch_solve) are device allocations of up to max_vectors * n * s bytes;
 * when a call ends they stay reserved for the next call on the same device
 * instead of being freed (an allocation plus free of 16 GB costs about 10 ms);
 * a later request reuses an idle buffer of at least its size and at most
 * 1/16 more (repeated solves of one size reuse theirs exactly).
 * Reuse is ordered by an event on the stream that last used the memory, so
 * calls on different streams may share the cache.  A call whose allocation
 * fails frees the idle buffers and tries once more before reporting
 * BBL_ERR_OOM; other users of the device get the memory back only through
 * bbl_workspace_release.
 *   bbl_workspace_bytes    bytes held idle for the current device
 *   bbl_workspace_release  waits for and frees every idle buffer of the
 *                          current device; BBL_ERR_CUDA if that fails      */
size_t bbl_workspace_bytes(void);
bbl_status bbl_workspace_release(void);

/* ---------------------------------------------------------------- matrix
 * Copies a CSR matrix (host or device arrays) to the device.
 *   n, nnz      dimension and number of stored entries (nnz >= 0, n >= 1)
 *   row_ptr     int64[n+1], row_ptr[0]=0, non-decreasing, row_ptr[n]=nnz
 *   col         int32[nnz], each row's columns strictly increasing in [0,n)
 *   val         FP64 or FP32 (val_dtype) [nnz]
 *   storage     precision of the device values (BBL_FP32 = mixed form)
 *   fmt         BBL_CSR, or BBL_SELL (SELL-C-sigma with C = 32 rows per
 *               slice, rows sorted by length inside windows of sell_sigma
 *               rows; sell_sigma a multiple of 32, 0 = 32 = no sorting)
 *               BBL_TILED: rows in blocks of `sell_sigma` rows (0 = 1024,
 *               16..1024) and columns in tiles of as many columns; per row
 *               block the entries are grouped by column tile (16-bit column
 *               in the tile, 16-bit row offsets; at most 65535 entries of
 *               one row block in one tile, BBL_ERR_UNSUPPORTED otherwise;
 *               inside a tile, slot-major per 64-row slice), and the SpMM
 *               stages each touched tile of V in shared memory (b a
 *               multiple of 16 bytes of block elements; other b use the CSR
 *               copy)
 *   keep_fp64   FP32 storage only: also keep an FP64 CSR copy of the values
 *               for the FP64 polish stage and the FP64 residual
 *   check_symmetry  1: verify H_ij == H_ji exactly (BBL_ERR_NOT_SYMMETRIC)
 * The structure (sortedness, range) is always validated on the device
 * before the call returns.  ||H||_inf and diag(H) are computed at creation. */
bbl_status bbl_matrix_create(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                             const void* val, bbl_dtype val_dtype, bbl_dtype storage, bbl_format fmt,
                             int sell_sigma, int keep_fp64, int check_symmetry, void* stream,
                             bbl_matrix** out);
void bbl_matrix_destroy(bbl_matrix* A);
/* n, nnz, ||H||_inf, device bytes held, stored format and precision.  Any output may be NULL. */
bbl_status bbl_matrix_info(const bbl_matrix* A, int64_t* n, int64_t* nnz, double* norm_inf,
                           int64_t* device_bytes, int* fmt, int* storage, int64_t* padded_nnz);

/* A matrix kept as Kronecker factors (fmt BBL_KRON) and applied without
 * storing its entries: the paper's on-the-fly rebuilding of the matrix
 * elements from factors shared by every vector of a block (Sec. I,
 * Sec. III.A, Appendix A), for
 *     H = Hp (x) I_nN + I_nP (x) Hn + sum_{k<K} Cp_k (x) Cn_k,
 * row r = p*nN + q, (A (x) B)[p*nN+q, p'*nN+q'] = A[p,p'] B[q,q'].
 * Factors (host or device arrays, copied): 2 + 2K square CSR matrices in
 * the order Hp, Hn, Cp_0, Cn_0, ..., Cp_{K-1}, Cn_{K-1} (Hp, Cp_k: nP x nP;
 * Hn, Cn_k: nN x nN), packed into fptr (int32 row pointers, factor f's
 * nP+1 or nN+1 of them from ptr_off[f], each starting at 0), fcol (int32,
 * strictly increasing per row) and fval (FP64; with storage BBL_FP32 the
 * operator's factors are their FP32 roundings), factor f's entries from
 * nz_off[f] (host int64 arrays of 2 + 2K offsets).
 *   nP*nN < 2^31; K <= 30; check_symmetry: every factor must be symmetric
 *   (BBL_ERR_NOT_SYMMETRIC), which makes H symmetric.
 * The matrix is the exact Kronecker sum: each entry is the FP64 sum of its
 * factor products (no rounding to the storage type).  diag(H), ||H||_inf
 * and the number of nonzeros of the expansion are computed at creation.
 * SpMM: FP32 blocks in FP32 arithmetic (storage BBL_FP32), FP64 blocks in
 * FP64 (bbl_spmm_f64, or storage BBL_FP64), float-float blocks in the
 * polish; one CTA forms one nN-row slab of W, staging one slab-sized tile
 * in shared memory, so nN * min(b, 16) * 4 bytes (FP32) must fit in about
 * 200 KB (narrower column groups are used for larger nN; beyond
 * nN ~ 4000 * 16 / (element bytes) the SpMM reports BBL_ERR_UNSUPPORTED).
 * bbl_pivot_bootstrap extracts H[S,S] from the factors.  Not accepted by
 * bbl_batch_create.                                                        */
bbl_status bbl_matrix_create_kron(int64_t nP, int64_t nN, int K, const int32_t* fptr, const int32_t* fcol,
                                  const double* fval, const int64_t* ptr_off, const int64_t* nz_off,
                                  bbl_dtype storage, int check_symmetry, void* stream, bbl_matrix** out);

/* SpMM schedule for the CSR path chosen by an autotuner: lanes per row (a
 * power of two <= 32; 0 restores the built-in rule).  Used by bbl_spmm and by
 * every solve on this matrix.                                            */
bbl_status bbl_matrix_set_spmm_lanes(bbl_matrix* A, int lanes_per_row);
/* diag(H) into a caller device buffer (FP64 [n]) */
bbl_status bbl_matrix_diagonal(const bbl_matrix* A, double* d, void* stream);

/* ---------------------------------------------------------------- S1: SpMM
 * W = H V (Sec. II.B, Eq. 3; w_{a,i} = sum_j H_ij v_{a,j}).  V, W: device,
 * n x b row-major, element type = the matrix storage type.  b in 1..16.   */
bbl_status bbl_spmm(const bbl_matrix* A, int b, const void* V, void* W, void* stream);
/* Same product in FP64 arithmetic on FP64 blocks whatever the storage (the
 * final residual of the mixed form).  b in 1..16. */
bbl_status bbl_spmm_f64(const bbl_matrix* A, int b, const double* V, double* W, void* stream);

/* ---------------------------------------------------------------- S2: reorthogonalisation
 * Full reorthogonalisation of W against the stored basis (Sec. II.A; block
 * classical Gram-Schmidt, `passes` passes):  C_p = Q^T W, W <- W - Q C_p.
 *   basis   device, nblocks consecutive n x b row-major blocks (block-major)
 *   W       device n x b, overwritten
 *   coeff   device FP64 [passes][nblocks*b][b] (row-major), or NULL
 * dtype: element type of basis and W (FP64 / FP32; FP32 accumulates the
 * coefficients in FP64 across row chunks).  passes in 1..2.            */
bbl_status bbl_block_reorth(int64_t n, int b, int nblocks, bbl_dtype dtype, const void* basis, void* W,
                            double* coeff, int passes, void* stream);

/* C = Q^T W (FP64, m x b row-major, device) without modifying W: the Gram
 * step of the reorthogonalisation alone (also used for the learned pivot's
 * training targets U^T X).  Layouts as in bbl_block_reorth.              */
bbl_status bbl_block_gram(int64_t n, int b, int nblocks, bbl_dtype dtype, const void* basis, const void* W,
                          double* C, void* stream);

/* C ~= Q16^T W for b = 8: the Gram step of the first of the two classical
 * Gram-Schmidt passes of the full reorthogonalisation (Sec. II.A, Eqs. 7-8)
 * in the FP32 stage (bbl_options.half_first_pass), from Q16, the FP16 copy
 * of an FP32 basis; the FP32 second pass removes what its rounding leaves.
 *   basis16 device FP16, nblocks consecutive n x 8 row-major blocks
 *   W       device FP32 n x 8 (not modified)
 *   C       device FP64 (nblocks*8) x 8 row-major
 * On the tensor cores (mma.sync m16n8k16, FP16 in, FP32 accumulate): per
 * chunk of 1024 rows W is scaled by the power of two that puts its largest
 * |W| in [2^13, 2^14) and rounded to FP16; the chunk's sums stay in FP32,
 * chunks are unscaled exactly and summed in FP64.  Error against Q16^T W:
 * below 2^-10 of |Q16|^T |W| entrywise.
 * Both pointers 16-byte aligned (BBL_ERR_INVALID_ARG otherwise).         */
bbl_status bbl_block_gram_f16(int64_t n, int nblocks, const void* basis16, const float* W, double* C, void* stream);

/* W -= Q C1, then C2 = Q^T W of the updated W, for b = 8 and FP32: the
 * update of the first and the Gram of the second classical Gram-Schmidt
 * pass of the full reorthogonalisation (Sec. II.A, Eqs. 7-8) in one read of
 * the basis (bbl_options.fused_update_gram).
 *   basis   device FP32, nblocks consecutive n x 8 row-major blocks,
 *           1 <= nblocks <= 128 (BBL_ERR_UNSUPPORTED otherwise)
 *   C1      device FP64 (nblocks*8) x 8 row-major (rounded to FP32 for the
 *           products, as in the FP32 update)
 *   W       device FP32 n x 8, updated in place
 *   C2      device FP64 (nblocks*8) x 8 row-major, written
 * Each CTA stages 16 rows of every block in shared memory and forms both
 * products from them on the tensor cores (mma.sync m16n8k8 TF32, FP32
 * accumulate), each FP32 operand split into a TF32 high part and remainder
 * (three products per pair; error per product below 2^-21 of |a b|), except
 * the update's products with the two newest blocks, which are FP32 FMAs
 * (in Lanczos these carry the large coefficients A_j and B_{j-1}).  The
 * update sums over the basis in FP32; the Gram sums a CTA's rows in FP32 and
 * the CTAs in FP64.  basis and W 16-byte aligned (BBL_ERR_INVALID_ARG
 * otherwise).  The call allocates its workspace and synchronises `stream`. */
bbl_status bbl_block_update_gram(int64_t n, int nblocks, const float* basis, const double* C1, float* W, double* C2,
                                 void* stream);

/* W -= Q C for b = 8 and FP32, with the blocks older than the `nnew` newest
 * read from the FP16 copy of the basis: the first pass's update of the
 * full reorthogonalisation (Sec. II.A, Eqs. 7-8) in the FP32 stage
 * (bbl_options.narrow_old_updates, nnew = 2: the blocks j and j-1 whose
 * coefficients are A_j and B_{j-1}^T stay FP32).
 *   basis16  device FP16, nblocks consecutive n x 8 row-major blocks
 *            (round-to-nearest copies of the FP32 blocks)
 *   basis    device FP32, the same blocks
 *   C        device FP64 (nblocks*8) x 8 row-major
 *   W        device FP32 n x 8, updated in place
 *   nnew     0 <= nnew (all blocks FP16 when 0, all FP32 when >= nblocks)
 * The older blocks' product runs on the tensor cores (mma.sync m16n8k16,
 * FP16 in, FP32 accumulate) with their rows of C multiplied by one power of
 * two s (largest entry into [2^13, 2^14); s at most 2^114), rounded to
 * FP16, and the sum
 * multiplied by 1/s: a rounding of those coefficients, which the second
 * Gram-Schmidt pass removes.  The newest blocks are FP32 FMA products with
 * C rounded to FP32, added to the same FP32 sum, which is then subtracted
 * from W.  basis16, basis and W 16-byte aligned (BBL_ERR_INVALID_ARG
 * otherwise).  The call allocates its workspace and synchronises `stream`. */
bbl_status bbl_block_update_f16old(int64_t n, int nblocks, int nnew, const void* basis16, const float* basis,
                                   const double* C, float* W, void* stream);

/* Allocation-free variant of bbl_block_gram (no counterpart in the paper).
 * For callers that must not allocate device memory: e.g. a process whose
 * device memory is already handed out under a fixed budget by a framework's
 * caching allocator, or a latency-critical loop that cannot afford the
 * implicit device synchronisation of cudaFree.  It calls no cudaMalloc,
 * cudaFree or allocating library routine: the per-chunk partial sums live in
 * a fixed 8 MiB file-scope device array that every device loading the
 * library holds until the process exits.
 *   Limit: nblocks*b*b <= 2^20 - 2048 (otherwise BBL_ERR_INVALID_ARG with a
 *   message): the array holds 2048 doubles of chunk tickets (one int per
 *   group of up to 256 columns) ahead of the partial sums.
 *   b in {1, 2, 4, 8, 16}.  Arguments and layouts as in bbl_block_gram.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins.  All calls share the one array and it
 * keeps the last call's contents (every partial a call reads is written by
 * that call first), so calls that overlap on the GPU race with each other:
 * serialise them, e.g. on one stream.  The call synchronises `stream`.     */
bbl_status bbl_block_gram_noalloc(int64_t n, int b, int nblocks, bbl_dtype dtype, const void* basis, const void* W,
                                  double* C, void* stream);

/* ---------------------------------------------------------------- S3: CholQR2
 * W = Q B with Q orthonormal (overwrites W), B upper triangular b x b:
 * G1 = W^T W, R1 = chol(G1), W <- W R1^{-1}, G2, R2, W <- W R2^{-1}, B = R2 R1.
 * (Replaces the paper's spectral factorisation of the overlap, Eqs. 9-11.)
 *   B          device FP64 b x b row-major
 *   defl_abs   a column whose Cholesky pivot is <= defl_abs^2 is deflated
 *   n_deflated host int, may be NULL: number of deflated columns.  Deflated
 *              columns of Q are zero and their rows of B are zero (the solver
 *              replaces them); the call then returns BBL_OK.               */
bbl_status bbl_cholqr2(int64_t n, int b, bbl_dtype dtype, void* W, double* B, double defl_abs,
                       int* n_deflated, void* stream);

/* ---------------------------------------------------------------- S4: Ritz solve
 * Lowest nev eigenpairs of the symmetric band matrix T (Eq. 12), m x m with
 * bandwidth p (T_ij = 0 for |i-j| > p), given in lower band storage
 * Tband[i*(p+1) + d] = T[i][i-d] (d = 0..p; entries with i-d < 0 ignored).
 *   theta  device FP64 [nev] ascending;  S device FP64 m x nev row-major,
 *   unit columns (sign: first largest-magnitude entry positive).
 * Method: Sylvester-inertia bisection (LDL^T of T - sigma I) then inverse
 * iteration (banded LU with partial pivoting) and Rayleigh quotients; the
 * vectors of clustered eigenvalues are orthonormalised together.  For
 * p in {1, 2, 4, 8} the recurrences run in FP32 and float-float (~48-bit)
 * arithmetic; normalisation and Rayleigh quotients are FP64.
 * 1 <= nev <= min(m, 32), p <= 16, m <= 16384.                                   */
bbl_status bbl_ritz_banded(int m, int p, int nev, const double* Tband, double* theta, double* S,
                           void* stream);

/* ---------------------------------------------------------------- S5: Ritz vectors
 * X = Q S: basis as in bbl_block_reorth (m = nblocks*b columns), S device
 * FP64 m x k row-major, X device FP64 n x k row-major.  k in 1..16.
 * FP64 basis: FP64 arithmetic.  FP32 basis: S rounded to FP32, products
 * summed in FP32 within tiles of 256 basis columns and in FP64 across tiles
 * (error below 256 * 2^-24 * sum_a |Q_ia S_ac| per entry).              */
bbl_status bbl_ritz_vectors(int64_t n, int b, int nblocks, bbl_dtype dtype, const void* basis, int k,
                            const double* S, double* X, void* stream);

/* ---------------------------------------------------------------- S6: pivots
 * Random pivot: n x b i.i.d. N(0,1) from splitmix64 (counter 2k, 2k+1 of
 * element k = i*b + c, Box-Muller), P device FP64.                       */
bbl_status bbl_pivot_random(int64_t n, int b, uint64_t seed, double* P, void* stream);
/* Bootstrapped pivot (Sec. II.B "bootstrap", Sec. III): S = the trunc_dim
 * rows with the smallest H_ii (ties: lower index), eigenvectors of the
 * lowest b eigenvalues of H[S,S] (block Lanczos on the GPU to sub_tol, or a
 * dense solve when trunc_dim <= b), zero-padded into P (device FP64 n x b
 * row-major).  If b > trunc_dim the remaining columns are random.  The
 * sub-solve keeps A's FP32 values in FP32 storage (FP32 stage, no polish)
 * when A is stored in FP32 and sub_tol >= 1e-5, else it runs in FP64.    */
bbl_status bbl_pivot_bootstrap(const bbl_matrix* A, int64_t trunc_dim, int b, double sub_tol, uint64_t seed,
                               double* P, void* stream);

/* Rayleigh-Ritz on the span of a pivot block P (host or device FP64 n x b):
 * Q = orth(P), the b Ritz values of Q^T H Q (theta, host, ascending) and the
 * residual norms ||H Q s_i - theta_i Q s_i||_2 (resid, host).  This is the
 * cheap one-SpMM test used to choose between a learned and a bootstrapped
 * pivot (the paper's Sec. II.B condition: the pivot must overlap the wanted
 * eigenvectors).                                                          */
bbl_status bbl_pivot_rr_residual(const bbl_matrix* A, int b, const double* P, double* theta, double* resid,
                                 void* stream);

/* Pivot-eigenvector overlap (Sec. II.B: block Lanczos only reaches the
 * eigenvectors its pivot overlaps; Sec. III.A: states the pivot misses
 * converge late, after higher "intruder" states).  For each of k vectors
 * x_i (unit eigenvectors, e.g. bbl_solve's), overlap[i] = ||Q^T x_i||_2 with
 * Q = orth(P) (CholQR2 in FP64; a pivot column dependent on the others to
 * 1e-10 of the largest column norm is dropped): 1 when x_i lies in span(P),
 * 0 when it is orthogonal to it.
 *   P        host or device FP64 n x b row-major;  X host or device FP64
 *            n x k row-major;  overlap host FP64 [k];  b, k in 1..16.   */
bbl_status bbl_pivot_overlap(int64_t n, int b, const double* P, int k, const double* X, double* overlap,
                             void* stream);

/* ---------------------------------------------------------------- learned pivot (MLP)
 * A small network g -> y = f(g) (1 -> H -> H -> O, exact-erf GELU), FP32
 * master weights used in BF16, FP32 activations and accumulation, MSE loss,
 * Adam; no counterpart in the paper (a proposal step in front of the
 * bootstrapped pivot).  Parameters are packed FP32:
 *   W1[H] b1[H] W2[H*H] b2[H] W3[O*H] b3[O]   (matrices row-major out x in).
 * g, target, y: device FP32 (batch, batch x O, batch x O).                */
typedef struct bbl_mlp bbl_mlp;
bbl_status bbl_mlp_create(int hidden, int out_dim, bbl_mlp** out);
void bbl_mlp_destroy(bbl_mlp* M);
int bbl_mlp_num_params(const bbl_mlp* M);
/* host or device packed parameters; resets the Adam state */
bbl_status bbl_mlp_set_params(bbl_mlp* M, const float* packed, void* stream);
/* parameters and/or the last gradients (host or device; either may be NULL) */
bbl_status bbl_mlp_get_params(const bbl_mlp* M, float* packed, float* grads, void* stream);
bbl_status bbl_mlp_forward(bbl_mlp* M, int batch, const float* g, float* y, void* stream);
/* forward + MSE loss (host) + backward into the internal gradient buffer */
bbl_status bbl_mlp_loss_grad(bbl_mlp* M, int batch, const float* g, const float* target, float* loss, void* stream);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) from the stored gradients */
bbl_status bbl_mlp_adam_step(bbl_mlp* M, float lr, void* stream);
/* `epochs` full-batch steps (one CUDA graph per epoch); loss_hist host [epochs] or NULL */
bbl_status bbl_mlp_train(bbl_mlp* M, int batch, const float* g, const float* target, int epochs, float lr,
                         float* loss_hist, void* stream);
/* P = U C(g): C = f(g) reshaped (nblocks_U*b_U) x b, U device FP32 basis of
 * nblocks_U row-major n x b_U blocks, P device FP64 n x b.  Requires
 * nblocks_U * b_U * b == out_dim.                                        */
bbl_status bbl_pivot_learned(bbl_mlp* M, float g, int64_t n, int b_U, int nblocks_U, const float* U, int b,
                             double* P, void* stream);

/* ---------------------------------------------------------------- batched form
 * Many independent solves in one graph launch (no counterpart in the paper;
 * its use here: many truncated-space bootstraps or training-data solves).
 * The problems are stacked row-wise into one block-diagonal CSR matrix:
 * problem s owns rows [offsets[s], offsets[s+1]) and may only reference
 * columns in the same range (checked, BBL_ERR_INVALID_ARG otherwise).
 * Arrays as in bbl_matrix_create (host or device, copied).               */
typedef struct bbl_batch bbl_batch;
bbl_status bbl_batch_create(int count, const int64_t* offsets, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                            const void* val, bbl_dtype val_dtype, bbl_dtype storage, bbl_format fmt, int sell_sigma,
                            void* stream, bbl_batch** out);
void bbl_batch_destroy(bbl_batch* B);
/* the stacked block-diagonal matrix (owned by the batch), e.g. for timing SpMM schedules */
bbl_status bbl_batch_matrix(bbl_batch* B, bbl_matrix** A);
/* SpMM schedule chosen by an autotuner: CSR lanes per row (0 = built-in rule) */
bbl_status bbl_batch_set_schedule(bbl_batch* B, int lanes_per_row);
/* Block Lanczos on every problem, in lock-step: one iteration is one fixed
 * kernel sequence over all problems; with use_graph = 1 it is captured as the
 * body of a CUDA graph while-node and the whole solve is one graph launch,
 * with use_graph = 0 the host drives the same sequence.  Each problem stops
 * when its nev estimates ||B_j s_i[last b]|| are <= tol*||H_s||_inf, tested
 * on opt->check_every's schedule (0: adaptive, per problem, as in
 * bbl_solve); random pivots (opt->seed).  FP32 storage with opt->polish
 * (default on) and nev in {1, 2, 4, 8, 16}: the problems whose true FP64
 * residuals miss tol after the FP32 run go on from their FP32 Ritz vectors
 * (block size nev) with FP64 blocks and FP64 arithmetic on the FP32 values,
 * in a second lock-step run over those problems only.  Outputs (host):
 * evals, resid [count x nev] (true FP64 residuals), iters [count] (blocks of
 * both runs), status [count] (BBL_OK when the true residuals meet tol,
 * BBL_ERR_NOT_CONVERGED, BBL_ERR_NUMERICAL for a breakdown).
 * b in {1, 2, 4, 8, 16}, nev <= 16.
 * Returns BBL_OK when every problem converged.                           */
bbl_status bbl_batch_solve(bbl_batch* B, int nev, int b, const bbl_options* opt, int use_graph, double* evals,
                           double* resid, int* iters, int* status, bbl_stats* stats);

/* ---------------------------------------------------------------- solve
 * Block Lanczos for the nev lowest eigenpairs (Sec. II.B, Eqs. 4-12).
 *   pivot   host or device FP64 n x b, or NULL (random, opt->seed)
 *   evals   host FP64 [nev] ascending
 *   evecs   host or device FP64 n x nev row-major, or NULL
 *   resid   host FP64 [nev]: true ||H x_i - theta_i x_i||_2 in FP64, or NULL
 *   stats   host, or NULL
 * b in 1..16, nev in 1..min(64, max_vectors).  Returns BBL_OK when
 * converged, BBL_ERR_NOT_CONVERGED (outputs filled) when the basis is full.
 * Device work is ordered on opt->stream; the call synchronises it.      */
bbl_status bbl_solve(const bbl_matrix* A, int nev, int b, const double* pivot, const bbl_options* opt,
                     double* evals, double* evecs, double* resid, bbl_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* BBL_H */
