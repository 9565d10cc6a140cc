/*
 * sma.h -- C ABI of the GB300 structured-matrix-approximation library.
 *
 * Kilmer & Saibaba, "Structured Matrix Approximations via Tensor
 * Decompositions" (arXiv 2105.01170), Algorithm 1 (Section 3.1):
 *   (1) determine the tuples (A_k) and (E_k)            -> sma_create
 *   (2) X := T_E[A]  (Section 3, matrix-to-tensor map)    -> sma_compress
 *   (3) compress X (t-SVDM, or the Tucker/HOSVD variants
 *       of Sections 2.4, 5.1, 5.2, 6.2, 6.3, 7.4)         -> sma_compress
 *   (4) A_hat := M_E[T]  (Section 3, tensor-to-matrix map)
 *       kept in factored form: sum of Kronecker products
 *       (Theorem 'tuckerkron', eq. structTucker) or block
 *       low rank (eq. blockTuck)                           -> sma_compress
 *       applied as a matvec                                 -> sma_apply
 *       or expanded densely for validation                  -> sma_reconstruct
 *   (5) rank and error; the Frobenius error of A_hat equals
 *       the tensor truncation error (Lemma 1, Lemma 2)     -> sma_result
 *
 * Conventions shared by every call
 *   - Every matrix is column-major.  Block (a, b) of an (ell*m) x (q*n) block
 *     matrix starts at row a*m, column b*n.
 *   - block_map is a host int32 array of ell*q entries, column-major (entry
 *     (a, b) at a + b*ell); each entry is the distinct-block index k in
 *     [0, p) or -1 for a zero block.  Every k in [0, p) must occur.
 *   - The mapped tensor is stored frontal-slice: X is m x n x p with
 *     X[:, :, k] = sqrt(eta_k) A_k (the paper's m x p x n tensor with modes 2
 *     and 3 swapped).
 *   - Precision SMA_FP64 takes and returns double; SMA_MIXED takes and returns
 *     float (the transform as 3-piece bf16 products and the Kronecker-sum
 *     matvec as 2-piece fp16 products of power-of-two-scaled operands, on
 *     tensor cores with fp32 accumulation; unfolding Grams in fp64; Jacobi
 *     SVD in fp32 with fp64 rotation angles for nearly parallel columns;
 *     fp64 energy sums).
 *   - Pointers to A, X and Y may be device memory or host memory; host
 *     buffers are copied on the handle's stream (only the bytes the call
 *     needs), except a page-locked (pinned) host A of a one-level problem,
 *     whose representative blocks the gather kernel reads in place over the
 *     host link.  Either way the host input must stay unchanged until the
 *     call's work on the stream has completed.  Device memory owned by the handle is allocated in sma_create
 *     and released in sma_destroy; no other call allocates, except sma_apply,
 *     which grows a per-handle workspace the first time it sees a larger nrhs.
 *   - All work is ordered on the stream given in sma_options (NULL = legacy
 *     default stream).  Calls on one handle are not thread-safe.
 *   - Errors are returned as sma_status; nothing is thrown across the ABI.
 *     Kernels report failures through a device status word that is read by
 *     sma_get_result.
 */
#ifndef SMA_H_
#define SMA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sma_ctx* sma_handle;

typedef enum {
  SMA_OK = 0,
  SMA_ERR_ARG = 1,          /* a size, pointer or option is invalid          */
  SMA_ERR_STRUCT = 2,       /* block_map does not cover 0..p-1 / out of range */
  SMA_ERR_CUDA = 3,         /* a CUDA runtime call failed                     */
  SMA_ERR_ALLOC = 4,        /* device allocation failed                       */
  SMA_ERR_NOCONVERGE = 5,   /* Jacobi hit max_sweeps before convergence       */
  SMA_ERR_TIMEOUT = 6,      /* a bounded device wait gave up                  */
  SMA_ERR_NONFINITE = 7,    /* NaN/Inf met in the input or a result           */
  SMA_ERR_STATE = 8,        /* call out of order (e.g. apply before compress) */
  SMA_ERR_UNSUPPORTED = 9,  /* option combination not implemented             */
  SMA_ERR_NOT_SPD = 10      /* SMA_TUCKER_SPD: the diagonal block T_0 has a
                               Cholesky pivot that is not positive and finite */
} sma_status;

typedef enum { SMA_FP64 = 0, SMA_MIXED = 1 } sma_precision;

typedef enum {
  /* t-SVDM: Xhat = X x3 M, SVD of every frontal slice, truncation, x3 M^T.
   * Factored result: A_hat = sum_i struct_E(M[i,:]) (x) L_i R_i.           */
  SMA_TSVDM = 0,
  /* Tucker-1 along the block index (Section 6.3): T = G x V, V the leading
   * left singular vectors of the block-index unfolding; the Kronecker rank.
   * Factored result: A_hat = sum_j struct_E(V[:,j]) (x) G_j.               */
  SMA_TUCKER_BLOCKMODE = 1,
  /* Two-sided compression with one shared U (Sections 5.1 and 6.2): SPSD
   * preserving block low rank (I (x) U) struct_E(U^T A_k U) (I (x) U^T).    */
  SMA_TUCKER_SHARED_U = 2,
  /* Tucker-2 on block rows and block columns (eq. blockTuck with V = I):
   * (I (x) U) struct_E(U^T A_k W) (I (x) W^T).                            */
  SMA_TUCKER_ROWCOL = 3,
  /* Multilevel (Section 7): truncated HOSVD of the weighted coefficient
   * tensor of a three-level structured matrix with m = n = 1; result
   * sum_j G_j struct1(U1_j) (x) struct2(U2_j) (x) struct3(U3_j).           */
  SMA_HOSVD_MULTILEVEL = 4,
  /* Positive-definiteness preserving block low rank (Section 5.2) for an SPD
   * T = I (x) T_0 + sum_k E_k (x) T_k: square blocks (m = n) and a square
   * block map (ell = q) whose diagonal holds one distinct block T_0 that
   * occurs nowhere else, and p >= 2.  T_0 = L L^T (Cholesky on the device,
   * in the element type); the other blocks become A_k = L^-1 T_k L^-T with
   * the map renumbered 0..p-2 (T_0's positions empty), and their tensor is
   * compressed as in SMA_TUCKER_SHARED_U.  Factored result:
   *   T_hat = (I (x) L)(I + (I (x) U) struct_E(U^T A_k U) (I (x) U^T))(I (x) L^T),
   * symmetric positive definite at every rank.  The tolerance, norm,
   * tensor_err and ranks in sma_result refer to the tensor of the A_k
   * (||A - A_hat||_F by Lemma 1, A = sum_k E_k (x) A_k).  A T_0 that is
   * not numerically SPD sets SMA_ERR_NOT_SPD in device_status (L = 0).   */
  SMA_TUCKER_SPD = 5,
  /* CP (Kruskal) form by alternating least squares (Section 2.3; Theorem
   * tildeA and Corollary kronsumcp): slice k of X is approximated by
   * Xf diag(Yf[k, :]) Zf^T with r = fixed_rank terms (1 <= r <= 64, r <= p),
   * cp_iters iterations from the caller's initial Xf, Zf (each iteration
   * updates Yf, then Xf, then Zf as least-squares solutions through the
   * normal equations, whose r x r matrices are solved in fp64; no column
   * normalisation).  Factored result: the Kronecker sum
   *   A_hat = sum_j struct_E(Yf[:, j]) (x) Xf[:, j] Zf[:, j]^T,
   * applied and reconstructed like SMA_TUCKER_BLOCKMODE; tensor_err is
   * ||X - T||_F measured directly.  A singular normal-equations matrix sets
   * SMA_ERR_NONFINITE.  All problems must have the same m and n.           */
  SMA_CP_ALS = 6
} sma_decomp;

typedef enum { SMA_M_DCT2 = 0, SMA_M_IDENTITY = 1, SMA_M_USER = 2 } sma_transform;

typedef enum {
  SMA_INPUT_DENSE = 0,   /* A is the full (ell*m) x (q*n) matrix, leading dim lda    */
  SMA_INPUT_BLOCKS = 1   /* A is the p distinct blocks A_k, each m x n with leading
                            dim lda, block k starting at A + k*lda*n (BSR-like)      */
} sma_input_layout;

/* One structured block matrix (Section 3: ell x q blocks of m x n, p distinct).
 * Multilevel (Section 7), with SMA_HOSVD_MULTILEVEL: level t has an
 * level_ell[t] x level_q[t] map level_maps[t] with level_p[t] distinct
 * indices, level 1 outermost; ell, q, p and block_map are then ignored.
 *   levels = 3, m = n = 1 (Section 7.2): the distinct scalars are passed in
 *     SMA_INPUT_BLOCKS layout in the order i1 + p1*(i2 + p2*i3).
 *   levels = 2, any m x n blocks (Section 7.1): the matrix is
 *     (ell1 ell2 m) x (q1 q2 n), block row a1*ell2 + a2 and block column
 *     b1*q2 + b2 holding A^(i1,i2); in SMA_INPUT_BLOCKS layout the distinct
 *     blocks come in the order i1 + p1*i2.  The fourth-order tensor
 *     (m x n x p1 x p2) is compressed by a truncated HOSVD over its four
 *     modes (tol^2 ||X||^2 / 4 each, or fixed_rank per mode), and the result
 *     is the Kronecker sum over (j1, j2) of struct1(Y1[:, j1]) (x)
 *     struct2(Y2[:, j2]) (x) Xf G[:, :, j1, j2] Zf^T; sma_result.ranks are
 *     (kx, kz, k1, k2) and n_kron_terms = k1 k2.                          */
typedef struct {
  int32_t ell, q, m, n, p;
  const int32_t* block_map;           /* host, ell*q, column-major          */
  int32_t levels;                     /* 1 (default), 2 or 3                */
  const int32_t* level_ell;           /* [levels]                           */
  const int32_t* level_q;             /* [levels]                           */
  const int32_t* level_p;             /* [levels]                           */
  const int32_t* const* level_maps;   /* [levels] host column-major maps    */
} sma_problem;

/* Preconditioning of the t-SVDM slice SVDs (an implementation choice; the
 * paper only needs the SVD).  SMA_PRECOND_QRCP factors each slice (or its
 * transpose) as B P = Q1 R1 by a column-pivoted Householder QR and runs the
 * one-sided Jacobi SVD on R1^T, which converges in fewer sweeps (Drmac and
 * Veselic 2008).  SMA_PRECOND_QRCP2 adds a second (unpivoted) QR,
 * R1^T = Q2 R2, and runs the Jacobi on R2^T (fewer sweeps again; slices
 * with max(m, n) <= 256, otherwise it acts as SMA_PRECOND_QRCP).
 * SMA_PRECOND_AUTO takes both QRs when min(m, n) >= 128 (and
 * max(m, n) <= 256), the first one alone when min(m, n) >= 128 otherwise. */
typedef enum {
  SMA_PRECOND_AUTO = 0,
  SMA_PRECOND_NONE = 1,
  SMA_PRECOND_QRCP = 2,
  SMA_PRECOND_QRCP2 = 3
} sma_precondition;

typedef struct {
  sma_precision prec;
  sma_decomp decomp;
  sma_transform mkind;
  sma_input_layout layout;
  const double* M_user;   /* host p x p column-major orthogonal, for SMA_M_USER */
  int32_t fixed_rank;     /* > 0: rank per slice (t-SVDM) / per mode (Tucker)   */
  double rel_tol;         /* used when fixed_rank == 0: ||A - A_hat||_F <=
                             rel_tol ||A||_F (global over slices for t-SVDM)   */
  int32_t max_sweeps;     /* Jacobi sweep limit (0 = 30)                        */
  void* stream;           /* cudaStream_t                                       */
  int32_t profile;        /* != 0: record per-stage CUDA events (sma_profile)   */
  int32_t graph;          /* != 0: capture sma_compress into a CUDA graph on the
                             second call with the same A pointers and leading
                             dimensions, and replay it while they are unchanged
                             (needs a non-NULL stream; stage timing is then
                             reported for the whole compression only)          */
  sma_precondition precondition;  /* t-SVDM slice SVD preconditioning          */
  int32_t autotune;       /* 1: on the first compression of each slice shape,
                             time the candidate slice-SVD plans on the actual
                             slices (twice each) and keep the fastest; the
                             choice is cached for the process.  0: default
                             plan.  Trial runs are not part of sma_profile's
                             stage times.                                     */
  /* Randomized block-index factor (Section 6.3, the variant used for the
   * largest matrix of the Kronecker-sum experiment), SMA_TUCKER_BLOCKMODE
   * only: with sketch_cols = s > 0, V is taken from the sketch
   * Y[:, :, k] = Omega^T X[:, :, k] Psi (s x s x p) instead of from X: the
   * s^2 x s^2 Gram of its block-index unfolding is eigen-solved, and the
   * fixed_rank (required, 1 <= fixed_rank <= s^2) leading left singular
   * vectors of the unfolding are recovered as Y_(3) W Sigma^-1.  The core,
   * the Kronecker terms and the error (measured as ||X - T||_F) are those of
   * X.  All problems must have the same m and n.  sma_export(2) then
   * returns the s^2 eigenvalues of the sketch's Gram.                      */
  int32_t sketch_cols;
  const double* sketch_omega;   /* host, m x s column-major (e.g. N(0,1))  */
  const double* sketch_psi;     /* host, n x s column-major                */
  /* SMA_CP_ALS: iterations (>= 1) and the initial factors, host, column-
   * major: cp_init_x m x fixed_rank, cp_init_z n x fixed_rank.             */
  int32_t cp_iters;
  const double* cp_init_x;
  const double* cp_init_z;
} sma_options;

typedef struct {
  int32_t total_rank;     /* t-SVDM: sum_i rho_i; Tucker: product of ranks      */
  int32_t n_kron_terms;   /* Kronecker terms (t-SVDM: slices with rho_i > 0)    */
  int32_t ranks[4];       /* Tucker mode ranks (unused entries 0)               */
  int32_t sweeps_max;     /* largest Jacobi sweep count used                    */
  int32_t device_status;  /* bit set of sma_status values raised by kernels     */
  double norm;            /* ||A||_F = ||X||_F                                   */
  double tensor_err;      /* ||X - T||_F = ||A - A_hat||_F (Lemma 1)             */
  double rel_err;         /* tensor_err / norm                                   */
  double orth_defect;     /* max |U^T U - I| over the orthonormal factors       */
  /* Section 6.2: |tr A - tr A_hat| / |tr A|, from the slice traces of X and of
   * the approximation on the device (tr A = sum_k tr(E_k) tr(X_k)); 0 when the
   * block grid or the blocks are not square, for the three-level form, and
   * for SMA_TUCKER_SPD, whose T_hat keeps the diagonal blocks exactly.      */
  double trace_relerr;
  /* Entries stored by the compressed form over the m n p entries of the
   * distinct blocks (Section 6.2 quotes (r^2 T + N r) / (N^2 T) for the
   * shared-U form): t-SVDM R (m + n + 1) with R = total_rank; block-index
   * Tucker (p + m n) r; CP (m + n + p) r; shared U m r + r^2 p (the SPD form
   * adds L, m (m + 1) / 2, over m n (p + 1) with its diagonal block); rows and
   * columns m r1 + n r3 + r1 r3 p; two levels m r1 + n r2 + p1 k1 + p2 k2 +
   * r1 r2 k1 k2; three levels sum_t p_t k_t + k1 k2 k3 over p1 p2 p3.        */
  double storage_ratio;
} sma_result;

/* Validate the problems, derive eta_k and the weights 1/sqrt(eta_k), build M
 * (DCT-II computed in fp64 on the host), allocate every device buffer the
 * compression needs, and build what depends on M and the maps alone (M's
 * split operand planes on the mixed path, the t-SVDM's Kronecker factors
 * C_i = struct_E(M[i, :])) on the device, synchronously.  nprob >= 1 problems share the options;
 * they are compressed together by one sma_compress call (batched launches).
 * Errors: SMA_ERR_ARG (sizes <= 0, nprob < 1, bad enum, M_user NULL),
 * SMA_ERR_STRUCT (map entry outside [-1, p) or a k that never occurs; for
 * SMA_TUCKER_SPD also a diagonal that is not one distinct block, a block
 * that is on the diagonal and off it, or p < 2), SMA_ERR_ARG also for
 * SMA_TUCKER_SPD with m != n or ell != q,
 * SMA_ERR_UNSUPPORTED, SMA_ERR_ALLOC, SMA_ERR_CUDA.  On error *h is NULL.  */
sma_status sma_create(sma_handle* h, const sma_problem* probs, int32_t nprob,
                      const sma_options* opt);

/* Steps (2)-(5) for every problem: A[i] points to problem i's input (layout
 * per options, element type per precision), lda[i] its leading dimension.
 * Enqueued on the handle's stream.  With several t-SVDM problems the slice
 * SVDs of all problems run in one launch per distinct slice size.  If res is non-NULL the call waits for the
 * stream and fills res[0..nprob-1]; with res == NULL it returns at once and
 * results are read later with sma_get_result.
 * Errors: SMA_ERR_ARG (NULL A, lda too small), SMA_ERR_CUDA; device-side
 * problems (non-convergence, non-finite data) are reported in
 * res->device_status and as the return value when res is non-NULL.        */
sma_status sma_compress(sma_handle h, const void* const* A, const int64_t* lda,
                        sma_result* res);

/* Wait for the handle's stream and copy problem i's report to *res.        */
sma_status sma_get_result(sma_handle h, int32_t i, sma_result* res);

/* Copy the retained per-slice ranks (t-SVDM: p entries) or the Tucker mode
 * ranks (up to 3 entries) of problem i to host array ranks; *count receives
 * the number written.  Waits for the stream.                                */
sma_status sma_get_ranks(sma_handle h, int32_t i, int32_t* ranks, int32_t* count);

/* Dense A_hat = M_E[T] of problem i ((ell*m) x (q*n), leading dim ld) written
 * to Ahat (device or host).  Validation only: O(ell q m n) memory.  For
 * SMA_TUCKER_SPD this is T_hat = (I (x) L)(I + M_E[T])(I (x) L^T), built in
 * two temporary (ell m)^2 device buffers allocated by this call.           */
sma_status sma_reconstruct(sma_handle h, int32_t i, void* Ahat, int64_t ld);

/* Y = A_hat X for nrhs right-hand sides (step 4, the factored matvec):
 * X is (q*n) x nrhs with leading dim ldx, Y is (ell*m) x nrhs with leading
 * dim ldy; each column of X is vec of an n x q matrix (Section 2.2,
 * vec(D X C^T) = (C (x) D) vec(X)).  SMA_TUCKER_SPD applies T_hat as
 * (I (x) L)(X' + A_hat X') with X' = (I (x) L^T) X.  Errors: SMA_ERR_STATE before a
 * successful sma_compress, SMA_ERR_ARG, SMA_ERR_ALLOC, SMA_ERR_CUDA.       */
sma_status sma_apply(sma_handle h, int32_t i, const void* X, int64_t ldx,
                     void* Y, int64_t ldy, int32_t nrhs);

/* Inspection of intermediate device buffers for step-by-step validation.
 * Copies `count` elements (element type per precision, except sigma: double)
 * of buffer `which` of problem i to dst (device or host); *avail receives the
 * number of elements the buffer holds (call with count = 0 to query).
 *   0 = X (m*n*p, the gathered tensor, step 2)
 *   1 = Xhat (m*n*p, X x3 M)
 *   2 = sigma (p * min(m,n) doubles, per slice descending)
 *   3 = T (m*n*p, the approximation tensor, after sma_reconstruct)
 *   4 = Tucker factor of the compressed mode (rows x rank, column-major)
 *   5 = SMA_TUCKER_SPD: the Cholesky factor L of T_0 (m x m, column-major,
 *       zero above the diagonal)
 *   6, 7 = SMA_CP_ALS: the factors Xf (m x r) and Zf (n x r); the block-
 *       index factor Yf is buffer 4 (p x p storage, the first r columns)   */
sma_status sma_export(sma_handle h, int32_t i, int32_t which, void* dst,
                      int64_t count, int64_t* avail);

/* Stages of the path timed when sma_options.profile != 0.                   */
typedef enum {
  SMA_STAGE_GATHER = 0,     /* step 1: struct_E gather and ||X||_F              */
  SMA_STAGE_TRANSFORM = 1,  /* X x3 M (t-SVDM) or the unfolding Gram (Tucker)   */
  SMA_STAGE_SVD = 2,        /* Jacobi SVD of the slices / Gram eigen-solve /
                               the CP iterations                               */
  SMA_STAGE_TRUNCATE = 3,   /* rank selection and error                         */
  SMA_STAGE_FACTORS = 4,    /* truncated slices / core, struct_E terms          */
  SMA_STAGE_REPORT = 5,     /* orthogonality check                              */
  SMA_STAGE_APPLY = 6,      /* the factored matvec                              */
  SMA_STAGE_PRECOND = 7,    /* QR preconditioning of the slice SVDs and its
                               rebuild of the discarded columns               */
  SMA_STAGE_COUNT = 8
} sma_stage;

/* Device time of each stage in ms, summed over the calls since the last
 * reset, measured with CUDA events recorded on the handle's stream around
 * the stage's kernels (ms[SMA_STAGE_COUNT]); calls[s] receives how many times
 * stage s ran (may be NULL); *launches the number of kernels the library
 * launched (may be NULL).  Waits for the stream.  reset != 0 clears the sums
 * after reading.  Errors: SMA_ERR_STATE when profiling is off.              */
sma_status sma_profile(sma_handle h, double* ms, int64_t* calls, int64_t* launches,
                       int32_t reset);

/* Batched one-sided Jacobi SVD of p fp32 slices that allocates no device
 * memory.  The paper has no counterpart: this is a deployment variant of the
 * per-slice SVD of the t-SVDM step for callers that cannot call cudaMalloc
 * where they need the work done (the execution callback of an inference-
 * engine plugin, which must not allocate; a loop whose device memory is
 * budgeted once by another allocator) and therefore cannot create a handle.
 * Its scratch -- the working copy of slices too large for shared memory and
 * the status word -- is a fixed 8 MiB __device__ array that every GPU loading
 * the library holds until the process exits.
 *   X      device, m x n x p fp32, slice k at X + k*m*n (column-major, ld m)
 *   W      device out, max(m,n) x min(m,n) x p: U Sigma of each slice (of its
 *          transpose when m < n), columns by decreasing singular value
 *   V      device out, min(m,n) x min(m,n) x p: the matching right vectors,
 *          so that slice = W V^T (m >= n) or slice = V W^T (m < n)
 *   sigma  device out, min(m,n) x p doubles, descending per slice
 *   sweeps device out, p int32 (may be NULL): sweeps used per slice
 *   status device out, one int32 (may be NULL): bit set of the sma_status
 *          values the kernel raised (NOCONVERGE, NONFINITE)
 *   max_sweeps (0 = 30); stream: cudaStream_t (NULL = legacy default stream)
 * Limit: a slice that does not fit in shared memory needs
 * (max(m,n) + min(m,n)) * min(m,n) floats of scratch; a slice needing more
 * than the 8 MiB array is rejected with SMA_ERR_ARG, as is a slice whose two
 * stacked columns (2 (m + n) floats) do not fit in shared memory, a NULL
 * pointer or a size <= 0; all of these are rejected on the host, before any
 * launch.  Larger p is processed in stream-ordered chunks that reuse the
 * array.  SMA_ERR_CUDA if a CUDA call fails.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress and caches it with the device's current context; make
 * that first call before any stream capture.  A call in a new context (after
 * cudaDeviceReset) repeats the lookup, so that first call in the new context
 * also belongs before any capture.  Every call shares the one array and
 * clears its status word
 * on entry, so calls whose work overlaps on the GPU (several streams or host
 * threads) race on it and must be serialised by the caller.                */
sma_status sma_slice_svd_noalloc(const float* X, int32_t m, int32_t n, int32_t p, float* W,
                                 float* V, double* sigma, int32_t* sweeps, int32_t* status,
                                 int32_t max_sweeps, void* stream);

sma_status sma_destroy(sma_handle h);

const char* sma_status_string(sma_status s);

/* Library version string and build target ("sm_103a").                     */
const char* sma_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SMA_H_ */
