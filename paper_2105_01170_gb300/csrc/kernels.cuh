// Kernel parameter blocks and launchers of the sma path (host side).
#pragma once
#include <vector>

#include "common.cuh"

namespace sma {

// ---- step 1: struct_E gather --------------------------------------------
// X[:, :, k] = w[k] * A_rep(k); rep_off gives the element offset of the
// representative block (dense layout: a*m + b*n*lda; blocks layout:
// k*n*lda).  wf holds w[k] as the fp32 pair (RN32(w), RN32(w - RN32(w))),
// which the fp32 form scales with (to the fp64 reference's value).  Output T
// = the input's type.
template <typename TS, typename T>
cudaError_t gather(const TS* A, int64_t lda, const int64_t* rep_off /*device, p*/,
                   const double* w /*device, p*/, const float* wf /*device, 2p*/, int m, int n,
                   int p, T* X, double* partial /*device, >= 1024*/, cudaStream_t st);
// The gathers of many problems (device inputs) in one launch, then each
// problem's ||X||^2 (a second launch, one CTA per problem).  part0: the
// first of the problem's nparts CTAs (ascending over the descriptors; the
// launch has the sum of nparts CTAs).
struct GatherDesc {
  const void* A;
  int64_t lda;
  const int64_t* rep_off;
  const double* w;
  const float* wf;
  int m, n, p;
  void* X;
  double* partial;
  double* norm2;
  int part0, nparts;
};
template <typename T>
cudaError_t gather_batched(const GatherDesc* d, int nprob, int total_parts, cudaStream_t st);
// ||X||_F^2 from the per-CTA partial sums written by gather.
cudaError_t finish_norm(const double* partial, int nparts, double* out, cudaStream_t st);
// out[e] = sum_s part[e + s count] for e < count, s < nslab (fixed order: the
// split-K partial products of a Gram).
cudaError_t sum_slabs(const double* part, int nslab, int64_t count, double* out, cudaStream_t st);
// Two-level Kronecker terms (Section 7): t = j1 + k1 j2 < k1 k2 (device k1,
// k2): Gt[:, t] = G[:, j1, j2] (G mn x p1 x p2, Gt mn x p1 p2) and
// V[i1 + p1 i2, t] = Y1[i1, j1] Y2[i2, j2] (V p1 p2 x p1 p2, Y1 p1 x p1,
// Y2 p2 x p2); later terms zero; *nterms = k1 k2.
template <typename T>
cudaError_t ml2_terms(const T* G, int mn, int p1, int p2, const T* Y1, const T* Y2, const int* k1,
                      const int* k2, T* Gt, T* V, int* nterms, cudaStream_t st);
// V[:, j] *= 1 / sqrt(ev[j]) for j < *r (device count), V with leading
// dimension ld (at most ld columns), rows entries per column; a column whose
// ev[j] <= 0 is zeroed.
cudaError_t scale_cols_rsqrt(double* V, int64_t ld, int rows, const double* ev, const int* r,
                             cudaStream_t st);
int gather_parts(int m, int n, int p);
// ||X - T||_F^2 over `count` elements (fp64 accumulation; nparts partial sums
// as for gather); two launches.  Tt == nullptr gives ||X||_F^2.
template <typename T>
cudaError_t residual_norm2(const T* X, const T* Tt, int64_t count, double* partial, int nparts,
                           double* out, cudaStream_t st);
// out[k] = trace of slice k (m x n, ld m) of an m x n x p tensor, fp64
// (Section 6.2's trace error: tr A = sum_k tr(E_k) tr(X_k)).
template <typename T>
cudaError_t slice_traces(const T* src, int m, int n, int p, double* out, cudaStream_t st);
// y = a x + b y over n fp64 elements.
cudaError_t axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t st);

// ---- step 3: Jacobi SVD ---------------------------------------------------
// Per-slice pointers for batched launches over slices of several problems.
template <typename T>
struct SliceDesc {
  const T* src;      // m x n slice, ld m
  T* U;              // mm x rc out
  T* V;              // rc x rc out
  double* sigma;     // rc out
  int* sweeps;       // 1 out (may be null)
  int* status;       // status word of the slice's problem
};
template <typename T>
struct JacobiParams {
  const SliceDesc<T>* desc = nullptr;           // if set: slice s uses desc[s]
  const T* src = nullptr; int64_t src_bs = 0;   // slices m x n, ld m
  int m = 0, n = 0;
  int mm = 0, rc = 0, trans = 0, ldS = 0, bcols = 0, g = 1, sort_n = 1;
  int max_sweeps = 30;
  double tol = 0.0;
  T* W = nullptr; int64_t W_bs = 0;             // block-mode workspace ((mm+rc) x rc per slice)
  T* U = nullptr; int64_t U_bs = 0;             // out: W = U Sigma, mm x rc per slice (sorted)
  T* V = nullptr; int64_t V_bs = 0;             // out: V, rc x rc per slice (sorted)
  double* sigma = nullptr;                      // out: rc per slice, descending
  int* sweeps = nullptr;                        // out: per slice
  int* status = nullptr;                        // status bits (atomicOr)
  int tile = 0;                                 // register-tiled sweeps (JacobiPlan::tile)
  // Rotation log (plans with JacobiPlan::rec): the kernel keeps no V rows and
  // records every tile task's scaled rotations here instead (U and sigma as
  // usual, V not written); jacobi_v_replay forms the columns of V needed.
  float4* vlog = nullptr; int64_t vlog_bs = 0;  // float4s per slice (jacobi_log_size)
  int vlog_sweeps = 0;                          // sweeps the log holds (the sweep limit then)
  int* order = nullptr;                         // out: pre-sort column of sorted column j
  int* vlsweeps = nullptr;                      // out: sweeps that rotated, per slice
};
struct JacobiPlan {
  int trans, mm, rc, ldS, bcols, sort_n, threads, g, block_mode, vec;
  int tile;   // 0: one pair per group of g lanes; 1, 2: register tiles of that many
              // float4 rows per lane on groups of g lanes (mm <= 4 g tile)
  int rec;    // 1: the rotation-log form (fp32 register tiles on whole warps)
  size_t smem;
};
// rec: the rotation-log form where the shape allows it (else as without).
template <typename T> JacobiPlan jacobi_plan(int m, int n, int max_smem, bool rec = false);
// The default plan and the autotuner's alternatives to it (same storage mode
// and the same rec).
template <typename T>
std::vector<JacobiPlan> jacobi_plan_candidates(int m, int n, int max_smem, bool rec = false);
// Sweeps the rotation log holds for a sweep limit of max_sweeps (at most
// kVlogMaxSweeps: the preconditioned slices converge in about 8), and the
// float4s of log per slice for plan pl and that many sweeps.
constexpr int kVlogMaxSweeps = 20;
inline int jacobi_log_sweeps(int max_sweeps) {
  return max_sweeps < 1 ? 1 : (max_sweeps < kVlogMaxSweeps ? max_sweeps : kVlogMaxSweeps);
}
size_t jacobi_log_size(const JacobiPlan& pl, int sweeps);
// After a rotation-log Jacobi run P (plan pl): V[:, j] for the columns
// j = ranks[s]..rc-1 of every slice s (all of them where ranks is NULL),
// the logged tasks applied in reverse order to the unit vector of the
// pre-sort column order[j].  The other columns of V are not written.
cudaError_t jacobi_v_replay(const JacobiParams<float>& P, const JacobiPlan& pl, const int* ranks,
                            int nslices, cudaStream_t st);
template <typename T>
cudaError_t jacobi_svd(const JacobiParams<T>& P, int nslices, int threads, size_t smem,
                       cudaStream_t st);
// One square matrix (P.mm == P.rc, not transposed) over many CTAs of a
// cooperative launch: blocks of bcols columns, one block pair per CTA and
// round of a block tournament, a bounded grid barrier between rounds.  The
// plan's block_mode field holds the CTA count; smem == 0 when it does not
// fit.  cs: barrier counter, per-sweep rotation counts (max_sweeps ints) and
// an abort flag in device memory, cleared by the launcher on the stream.
struct CoopSync {
  unsigned* bar;
  int* rot;
  int* abort_flag;
};
template <typename T> JacobiPlan jacobi_coop_plan(int rows, int max_smem);
// One square fp32 matrix of order rows (8 * CTAs <= rows <= 256, rows % 4 ==
// 0) over a cluster of CTAs: 2 x CTAs blocks of bcols columns, one block pair
// per CTA and round of a block tournament, the hardware cluster barrier
// between rounds.  The plan's block_mode field holds the CTA count; smem == 0
// when the shape does not qualify.  rot_count: max_sweeps ints in device
// memory, cleared by the launcher; P.W: the (2 rows) x rows workspace.
JacobiPlan jacobi_cluster_plan(int rows, int max_smem);
cudaError_t jacobi_svd_cluster(const JacobiParams<float>& P, const JacobiPlan& pl, int* rot_count,
                               cudaStream_t st);
template <typename T>
cudaError_t jacobi_svd_coop(const JacobiParams<T>& P, const JacobiPlan& pl, const CoopSync& cs,
                            cudaStream_t st);

// ---- QR preconditioning of the slice SVD (qr.cu) ---------------------------
// Shared-memory plan: the factorisation keeps nslot columns of a slice in
// shared memory and novf = rc - nslot in the global overflow G; the finish
// kernel keeps up to fslot of the columns it builds in shared memory.
struct QrPlan {
  int nslot = 0, novf = 0, fslot = 0;
  size_t smem_qr = 0, smem_fin = 0;
};
template <typename T> QrPlan qr_plan(int mm, int rc, int max_smem);
template <typename T>
struct QrParams {
  const T* src = nullptr; int64_t src_bs = 0;   // slices m x n, ld m
  int m = 0, mm = 0, rc = 0, trans = 0;         // B = slice (trans = 0) or its transpose
  QrPlan plan{};
  T* F = nullptr; int64_t F_bs = 0;             // out: reflectors and R1, mm x rc per slice
  T* G = nullptr; int64_t G_bs = 0;             // overflow columns, mm x novf per slice
  T* tau = nullptr;                             // out: rc per slice
  int* perm = nullptr;                          // out: rc per slice
  T* Jin = nullptr; int64_t J_bs = 0;           // out: R1^T, rc x rc per slice
  const T* W = nullptr; int64_t W_bs = 0;       // Jacobi W of R1^T (rc x rc)
  const T* V = nullptr; int64_t V_bs = 0;       // Jacobi V of R1^T (rc x rc)
  T* Rt = nullptr; int64_t Rt_bs = 0;           // out: P W, rc x rc
  T* L = nullptr; int64_t L_bs = 0;             // out: Q1 [V_d; 0], mm x rc
};
// B P = Q1 R1 for every slice's working matrix B (mm x rc); writes R1^T.
template <typename T> cudaError_t qrcp(const QrParams<T>& P, int nslices, cudaStream_t st);
// Unpivoted blocked Householder QR of every slice's n x n matrix (mm == rc
// == n <= kQrWarpRows, ld m), same outputs as qrcp with perm = identity.
template <typename T> cudaError_t qr_blocked(const QrParams<T>& P, int nslices, cudaStream_t st);
// Working matrices of at most this many rows rebuild their discarded columns
// with the columns held in registers (and may take the second QR).
constexpr int kQrWarpRows = 256;
// The rebuild factors of the discarded columns d = ranks[s]..rc-1.  One QR
// (P2 null): Rt_d = P W_d and L_d = Q1 [V_d; 0].  Two QRs (P2: the second
// QR R1^T P2 = Q2 R2 whose R2^T the Jacobi factored; needs
// mm <= kQrWarpRows): Rt_d = P (Q2 V_d) and L_d = Q1 [P2 W_d; 0].
template <typename T>
cudaError_t qr_finish(const QrParams<T>& P, const QrParams<T>* P2, const int* ranks, int nslices,
                      cudaStream_t st);

// ---- step 4: truncation ---------------------------------------------------
// sigma: rc x p (descending per slice).  Tolerance rule when fixed_rank <= 0.
// energies != 0: sigma holds energies (Gram eigenvalues) instead.
// Writes ranks[p], off[p+1] (exclusive prefix), stats[1] = discarded energy,
// iscal[0] = total rank, iscal[1] = #slices with rank > 0.
// The truncation of several t-SVDM problems in one launch (one CTA each).
struct TruncDesc {
  const double* sigma;
  int rc, p;
  const double* normX2;
  int* ranks;
  int* off;
  double* err2;
  int* iscal;
  double* suf;
};
// The t-SVDM's per-slice work after the truncation, for a batch of slices of
// one shape from many problems (one launch): the truncated slice
// D = Xhat - W_d V_d^T (d the columns from the slice's retained rank on;
// trans: D = Xhat - V_d W_d^T) and the orthogonality defect max |U_r^T U_r -
// I| of its retained left factor U = W Sigma^-1.
template <typename T>
struct PostDesc {
  const T* Xh;          // m x n slice (ld m)
  T* D;                 // m x n out
  const T* W;           // mm x rc, ld mm (the Jacobi W = U Sigma, sorted)
  const T* V;           // rc x rc, ld rc
  const double* sigma;  // rc, descending
  const int* rank;      // the slice's retained rank
  double* orth;         // out
};
template <typename T>
cudaError_t slice_post(const PostDesc<T>* d, int count, int m, int n, int mm, int rc, int trans,
                       cudaStream_t st);
cudaError_t truncate_ranks_batched(const TruncDesc* d, int nprob, double rel_tol, int fixed_rank,
                                   cudaStream_t st);
cudaError_t truncate_ranks(const double* sigma, int rc, int p, const double* normX2,
                           double rel_tol, int fixed_rank, int* ranks, int* off,
                           double* err2, int* iscal, double* scratch /*(rc+1)*p*/,
                           cudaStream_t st, int energies = 0);

// ---- helpers of steps 3-5 ------------------------------------------------
// C_i = struct_E(coef[i, :]) for i < nterms: C[a + ell*b + ell*q*i] =
// coef[i*cs_i + k*cs_k] / sqrt(eta_k) with k = map(a, b) (0 if k < 0).
// As build_struct_terms, writing only the nnz positions nzpos[] (block
// indices nzk[]) of every term; C's other positions must already be zero.
template <typename T>
cudaError_t build_struct_terms_nz(const int* nzpos, const int* nzk, int nnz, const double* isq,
                                  int ell, int q, const T* coef, int64_t cs_i, int64_t cs_k,
                                  int nterms, const int* nterms_dev, T* C, cudaStream_t st);
template <typename T>
cudaError_t build_struct_terms(const int* map, const double* inv_sqrt_eta, int ell, int q,
                               const T* coef, int64_t cs_i, int64_t cs_k, int nterms,
                               const int* nterms_dev, T* C, cudaStream_t st);
// Ahat (ell*m x q*n, ld) = M_E[T]: block (a,b) = T[:,:,k] / sqrt(eta_k).
template <typename T>
cudaError_t scatter_ME(const int* map, const double* inv_sqrt_eta, int ell, int q, int m,
                       int n, const T* Tt, T* Ahat, int64_t ld, cudaStream_t st);
// max |G_i[a,b] / (s_a s_b) - delta_ab| over the leading r_i x r_i block of
// each of p Gram matrices (s = per-slice scales, rc per slice; NULL = 1).
template <typename T>
cudaError_t orth_defect(const T* Gm, int rc, int p, const int* ranks, const double* scale,
                        double* out, cudaStream_t st);
// The same defect for Gm = W_i^T W_i (W_i: the K x rc block of slice i, ld
// ldw, slices w_bs apart) without forming the Grams; zeroes out[p] first.
template <typename T>
cudaError_t orth_gram_defect(const T* W, int ldw, int64_t w_bs, int K, int rc, int p,
                             const int* ranks, const double* scale, double* out,
                             cudaStream_t st);
// ---- multilevel (three levels, m = n = 1) ---------------------------------
struct MlMaps {
  const int* map[3];
  const double* isq[3];
  int ell[3], q[3], p[3];
};
// X[i1 + p1 (i2 + p2 i3)] = w1[i1] w2[i2] w3[i3] a[...] and per-CTA ||X||^2
// partial sums (nparts CTAs, as for gather).
template <typename T>
cudaError_t ml_gather(const T* a, const double* w1, const double* w2, const double* w3, int p1,
                      int p2, int p3, T* X, double* partial, int nparts, cudaStream_t st);
// out[a s_a + b s_b + j s_j] = coef[map(a,b) + p j] / sqrt(eta), j < nterms.
template <typename T>
cudaError_t struct_strided(const int* map, const double* isq, int ell, int q, const T* coef, int p,
                           int nterms, int64_t s_a, int64_t s_b, int64_t s_j, T* out,
                           cudaStream_t st);
template <typename T>
cudaError_t ml_scatter(const MlMaps& mp, const T* Tt, T* Ahat, int64_t ld, cudaStream_t st);
// V[a3 + l3 j12 + l3 k12 c] = sum_j3 G[j12 + k12 j3] U[a3 + l3 j3 + l3 k3 c]
// for a3 < l3, c < ncol, j12 < k12, j3 < k3 (k3 <= 16): the core contraction of
// the three-level matvec, memory-bound, coalesced over a3.
template <typename T>
cudaError_t ml_core(const T* G, int k12, int k3, const T* U, int l3, int64_t ncol, T* V,
                    cudaStream_t st);

// ---- three-level matvec in the factors' structured form (ml_apply.cu) -------
// Level t (0 outermost): l[t] x q[t] map with p[t] distinct values, its
// nonzero positions as a compressed-row list (ptr: l[t] + 1 offsets; col:
// the column b; kk: the distinct index map(a, b)), 1/sqrt(eta) per distinct
// index, the factor U_t (p[t] x p[t], leading r[t] columns used); G the core
// (p0 x p1 x p2); c1, c2, b the coefficient buffers (r0 nnz0, r1 nnz1,
// r0 r1 nnz2 entries).
template <typename T>
struct MlApply {
  int l[3], q[3], p[3], r[3], nnz[3];
  const int* ptr[3];
  const int* col[3];
  const int* kk[3];
  const double* isq[3];
  const T* U[3];
  const T* G;
  T* c1;
  T* c2;
  T* b;
};
// Shared memory of ml_xy_kernel for these sizes.
template <typename T>
size_t ml_apply_smem(const MlApply<T>& P);
// Y (l0 l1 l2 x nv, ld ldy) = A_hat X (q0 q1 q2 x nv, ld ldx) through W
// (l1 l2 r0 q0 nv elements); coef: recompute c1, c2, b first.
template <typename T>
cudaError_t ml_apply(const MlApply<T>& P, bool coef, const T* X, int64_t ldx, T* W, T* Y,
                     int64_t ldy, int nv, cudaStream_t st);

// copy and precision conversion helpers
// dst[i0 + n0 (i1 + n1 i2)] = src[i0 s0 + i1 s1 + i2 s2] (fp64)
cudaError_t permute3(const double* src, int64_t s0, int64_t s1, int64_t s2, int n0, int n1, int n2,
                     double* dst, cudaStream_t st);
template <typename TD, typename TS>
cudaError_t convert(const TS* src, TD* dst, int64_t count, cudaStream_t st);

// Mixed Gram eigen-solve preconditioner (gram_pre.cu): G = L L^T with L =
// P R^T from the diagonally pivoted Cholesky P^T G P = R^T R in fp64 (G n x n
// column-major, n <= kPcholMaxRows; work: n^2 doubles); L in fp64 and, scaled
// by 1 / sqrt(max_j G_jj), in fp32 (both n x n column-major).
constexpr int kPcholMaxRows = 256;
cudaError_t gram_pchol(const double* G, int n, double* work, double* L, float* L32, int* status,
                       cudaStream_t st);
// After the Jacobi of L V (W_f = L V V2 = U Sigma, sig = Sigma): U = W_f
// Sigma^-1 (e_j where sigma_j is 0 or not finite) and sig <- sig^2, the
// eigenvalues of G.
cudaError_t gram_pchol_finish(const double* Wf, double* sig, int n, double* U, cudaStream_t st);

// ---- CP by alternating least squares (cp.cu) --------------------------------
constexpr int kCpMaxRank = 64;
// out[(a + ra b), j] = A[a, j] B[b, j]: the Khatri-Rao (columnwise Kronecker)
// product of A (ra x r) and B (rb x r), out (ra rb x r); all ld = rows.
template <typename T>
cudaError_t khatri_rao(const T* A, int ra, const T* B, int rb, int r, T* out, cudaStream_t st);
// out (rows x r, ld ldo) = M (rows x r, ld rows) ((B1^T B1) .* (B2^T B2))^-1,
// B1 n1 x r, B2 n2 x r, r <= kCpMaxRank; the r x r system in fp64 (one CTA);
// a singular system sets SMA_ERR_NONFINITE in *status and writes zeros.
template <typename T>
cudaError_t cp_solve(const T* B1, int n1, const T* B2, int n2, int r, const T* M, int rows, T* out,
                     int64_t ldo, int* status, cudaStream_t st);
// out[e] = sum_s part[e + s count] in a fixed order (fp64 accumulation).
template <typename T>
cudaError_t sum_slabs_t(const T* part, int nslab, int64_t count, T* out, cudaStream_t st);
// *dst = v on the stream.
cudaError_t set_int(int* dst, int v, cudaStream_t st);

// ---- Section 5.2 (SPD-preserving form) -------------------------------------
// T_0 (m x m, ld ld0) = L L^T and L^-1, one CTA, both m x m column-major
// (ld m); a pivot that is not positive and finite zeroes L and L^-1 and sets
// SMA_ERR_NOT_SPD in *status.
template <typename T>
cudaError_t chol_inv(const T* T0, int64_t ld0, int m, T* L, T* Linv, int* status,
                     cudaStream_t st);
// A(i, i) += 1 for i < n.
template <typename T>
cudaError_t add_identity(T* A, int64_t ld, int64_t n, cudaStream_t st);
// Y[:, s] += X[:, s], rows entries per column, s < cols.
template <typename T>
cudaError_t add_into(const T* X, int64_t ldx, T* Y, int64_t ldy, int64_t rows, int cols,
                     cudaStream_t st);

}  // namespace sma
