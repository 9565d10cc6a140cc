// C ABI of the structured-matrix-approximation path (include/sma.h).
//
// Host side only: validation of the structure description, derivation of
// eta_k and the weights (Section 3), the transform M, device buffers, and the
// enqueueing of the kernels of gemm.cu, jacobi.cu, steps.cu and tc_gemm.cu.
// Every arithmetic step of the path runs in those kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <initializer_list>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_gemm.cuh"

using namespace sma;

namespace {

// Gram eigen-solves of this order and larger run over many CTAs
// (jacobi_svd_coop); smaller ones in one CTA.
constexpr int kCoopMinRows = 40;
// fp32 Gram solves (single matrices) of this order and larger run over a
// cluster of CTAs (jacobi_svd_cluster)
constexpr int kClusterMinRows = 128;
// SMA_PRECOND_AUTO preconditions the slice SVD by a column-pivoted QR from
// this min(m, n) on (below it the factorisation costs more than the sweeps
// it saves), and by two from kQr2AutoMin on
constexpr int kQrAutoMin = 128;
constexpr int kQr2AutoMin = 128;

#define SMA_CK(...)                                 \
  do {                                              \
    cudaError_t e_ = (__VA_ARGS__);                           \
    if (e_ != cudaSuccess) {                        \
      last_cuda_error() = e_;                       \
      return SMA_ERR_CUDA;                          \
    }                                               \
  } while (0)

#define SMA_TRY(...)                  \
  do {                                \
    sma_status s_ = (__VA_ARGS__);              \
    if (s_ != SMA_OK) return s_;      \
  } while (0)

cudaError_t& last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

// The device-side address of page-locked host memory the GPU can read in
// place (registered or allocated pinned host memory), or null for pageable
// memory, which has to be copied first.
const void* mapped_host_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Orthonormal DCT-II in fp64 (the transform M of the t-SVDM):
// M[k, j] = a_k cos(pi (2j+1) k / (2p)), a_0 = sqrt(1/p), a_k = sqrt(2/p).
std::vector<double> dct2(int p) {
  std::vector<double> M((size_t)p * p);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < p; ++k) {
    const double a = std::sqrt((k == 0 ? 1.0 : 2.0) / p);
    for (int j = 0; j < p; ++j) M[k + (size_t)j * p] = a * std::cos(pi * (2 * j + 1) * k / (2.0 * p));
  }
  return M;
}

struct DevBuf {
  std::vector<void*> ptrs;
  ~DevBuf() {
    for (void* q : ptrs) cudaFree(q);
  }
  template <typename U>
  sma_status alloc(U** out, size_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(U)) != cudaSuccess) {
      cudaGetLastError();
      return SMA_ERR_ALLOC;
    }
    ptrs.push_back(q);
    *out = static_cast<U*>(q);
    return SMA_OK;
  }
  void release(void* q) {
    for (auto& x : ptrs)
      if (x == q) {
        cudaFree(x);
        x = nullptr;
      }
  }
};

// Per-problem state, one element type T (double: SMA_FP64, float: SMA_MIXED).
template <typename T>
struct Prob {
  // host description
  int ell = 0, q = 0, m = 0, n = 0, p = 0;
  std::vector<int32_t> map;                 // column-major
  std::vector<int64_t> eta;
  std::vector<int> rep_a, rep_b;            // representative block (Section 3)
  // plan
  JacobiPlan jp{};
  int rc = 0, mm = 0;
  // common device buffers
  int* d_map = nullptr;
  int* d_nzpos = nullptr;                   // map positions with a block (column-major)
  int* d_nzk = nullptr;                     // their block index k
  int nnz = 0;
  double* d_w = nullptr;                    // sqrt(eta_k)
  float* d_wf = nullptr;                    // sqrt(eta_k) as fp32 pairs (hi, lo)
  double* d_isq = nullptr;                  // 1/sqrt(eta_k)
  int64_t* d_rep = nullptr;
  int64_t rep_lda = -1;
  int rep_layout = -1;
  T* X = nullptr;
  double* partial = nullptr;
  int nparts = 0;
  double* stats = nullptr;                  // [0] ||X||^2, [1] discarded energy
  // Section 6.2 trace error: tr(E_k) = d_k / sqrt(eta_k) per distinct block
  // (d_k = diagonal positions holding k; empty when the grid or the blocks
  // are not square), device buffer for the 2p slice traces, host M (t-SVDM)
  std::vector<double> trw;
  double* traces = nullptr;
  std::vector<double> Mh;
  int* iscal = nullptr;                     // [0] total rank [1] terms [2..4] mode ranks
  int* status = nullptr;
  int* sweeps = nullptr;
  double* orth = nullptr;                   // per slice / factor
  int n_orth = 0;
  // staging for host inputs
  T* stage = nullptr;
  // t-SVDM
  T* Mt = nullptr;                          // M, p x p column-major
  T* Xh = nullptr;
  T* Wj = nullptr;
  T* U = nullptr;                           // Jacobi W = U Sigma (sorted), jp.mm x rc per slice
  T* V = nullptr;                           // Jacobi V, rc x rc per slice
  // rotation log of the fp32 Jacobi (jp.rec): the kernel records its
  // rotations instead of forming V, and after the truncation the replay
  // forms the columns of V the rebuild reads (the discarded ones)
  float4* vlog = nullptr;
  int64_t vlog_bs = 0;                      // float4s per slice
  int* vorder = nullptr;                    // pre-sort column of each sorted column
  int* vlsw = nullptr;                      // rotating sweeps per slice
  // column-pivoted QR preconditioning (qr.cu): the Jacobi then runs on the
  // rc x rc factor R1^T, and the rebuild uses L = Q1 V (discarded columns)
  // and Rt = P W in place of the slice's own W and V
  bool qr = false;
  bool tuned = false;                       // Jacobi plan chosen by the autotuner
  int trans = 0;                            // slices processed transposed (m < n)
  QrPlan qplan{};
  T* qF = nullptr;
  T* qG = nullptr;
  T* qtau = nullptr;
  int* qperm = nullptr;
  T* qJ = nullptr;
  T* qRt = nullptr;
  T* qL = nullptr;
  // second QR (unpivoted, blocked), of R1^T = Q2 R2: the Jacobi runs on
  // R2^T, and the rebuild uses L = Q1 [W_d; 0] and Rt = P Q2 V_d
  bool qr2 = false;
  T* qF2 = nullptr;
  T* qtau2 = nullptr;
  int* qperm2 = nullptr;
  T* qJ2 = nullptr;
  double* sigma = nullptr;
  double* suf = nullptr;
  int* ranks = nullptr;
  int* off = nullptr;
  T* Gorth = nullptr;
  // Kronecker-sum terms: D (m x n x nterms_max) and C (ell x q x nterms_max)
  T* D = nullptr;
  T* C = nullptr;
  int nterms_max = 0;
  // Tucker
  double* X64 = nullptr;                    // fp64 copy of X (Gram accumulation)
  double* Xu = nullptr;                     // an unfolding of X64 laid out contiguously
  double* gram = nullptr;
  double* gvec = nullptr;                   // Jacobi output of the Gram (vectors)
  double* gsig = nullptr;                   // Gram eigenvalues
  double* Wg = nullptr;                     // block-mode Jacobi workspace for the Gram
  double* gW = nullptr;                     // Jacobi W output for the Gram (unused values)
  SliceDesc<double>* gdesc = nullptr;       // per Gram slot: the Jacobi's pointers
  size_t gstride = 0;                       // elements between the two Gram slots
  int gdim = 0;
  // mixed path: fp32 copies of the Grams, their fp32 eigenvectors, the unused
  // W output and block-mode workspace of the fp32 Jacobi; the fp64 residual
  // correction's Rayleigh-Ritz matrices S = U^T G U, their eigenvectors Z,
  // two temporaries and the correction's sweep counts
  float* g32 = nullptr;
  float* gv32 = nullptr;
  float* gw32 = nullptr;
  float* wg32 = nullptr;
  SliceDesc<float>* gdesc32 = nullptr;
  double* gS = nullptr;
  double* gZ = nullptr;
  double* gT1 = nullptr;
  double* gT2 = nullptr;
  int* sweepsS = nullptr;
  SliceDesc<double>* gdescS = nullptr;
  T* F1 = nullptr;                          // leading factor (rows), T
  T* F2 = nullptr;                          // second factor (cols), T
  T* core = nullptr;                        // r1 x r3 x p core slices
  T* tmp = nullptr;
  T* mid = nullptr;                         // struct_E(core) dense (ell r1 x q r3)
  int r1max = 0, r3max = 0;
  // randomized block-index factor (Section 6.3): Omega (m x sk), Psi (n x sk),
  // the sketch Y (sk x sk x p, T and fp64) and Omega^T X_k (sk x n x p)
  int sk = 0;
  // CP by alternating least squares: the factors Xf (m x r), Zf (n x r), their
  // initial values, and the Khatri-Rao / contraction / per-block workspaces
  // (Yf, p x r, lives in F1)
  int cp_r = 0;
  T* cXf = nullptr;
  T* cZf = nullptr;
  T* cXf0 = nullptr;
  T* cZf0 = nullptr;
  T* cKR = nullptr;
  T* cM = nullptr;
  T* cSlab = nullptr;
  size_t cSlab_elems = 0;
  T* Om = nullptr;
  T* Ps = nullptr;
  T* Ysk = nullptr;
  double* Y64 = nullptr;
  T* Ytmp = nullptr;
  // multilevel (three levels, m = n = 1; Section 7)
  int L = 1;
  int lell[3] = {0, 0, 0}, lq[3] = {0, 0, 0}, lp[3] = {0, 0, 0};
  std::vector<int32_t> lmap[3];
  int* d_lmap[3] = {nullptr, nullptr, nullptr};
  // the levels' maps as compressed-row lists (row offsets, columns, distinct
  // index) for the structured matvec, and its coefficient buffers
  int* d_lptr[3] = {nullptr, nullptr, nullptr};
  int* d_lcol[3] = {nullptr, nullptr, nullptr};
  int* d_lkk[3] = {nullptr, nullptr, nullptr};
  int lnnz[3] = {0, 0, 0};
  T* mlc1 = nullptr;
  T* mlc2 = nullptr;
  T* mlcb = nullptr;
  double* d_lw[3] = {nullptr, nullptr, nullptr};
  double* d_lisq[3] = {nullptr, nullptr, nullptr};
  T* Uml[3] = {nullptr, nullptr, nullptr};  // factors (p_t x p_t, leading k_t used)
  T* T1 = nullptr;
  T* T2 = nullptr;
  T* Gc = nullptr;                          // core, p1 x p2 x p3 (leading k's used)
  T* Gcmp = nullptr;                        // compact core k1 k2 x k3
  T* C1i = nullptr;                         // struct_1 terms, l1 x (k1 q1) interleaved
  T* C2i = nullptr;                         // struct_2 terms, l2 x (k2 q2) interleaved
  T* C3st = nullptr;                        // struct_3 terms, (l3 k3) x q3 stacked
  T* U3x = nullptr;
  size_t U3x_elems = 0;
  T* Vml = nullptr;
  size_t Vml_elems = 0;
  T* Wml = nullptr;
  size_t Wml_elems = 0;
  bool ml_valid = false;
  bool ml_cvalid = false;                   // the structured matvec's coefficients
  // two levels with m x n blocks (Section 7): the one-level problem of the
  // product map; the factors of the four modes (m, n, p1, p2) and the core
  // and term workspaces of the Kronecker sum over (j1, j2)
  bool ml2 = false;
  T* mlF[4] = {nullptr, nullptr, nullptr, nullptr};
  T* mlT1 = nullptr;
  T* mlT2 = nullptr;
  T* mlG = nullptr;
  T* mlGt = nullptr;
  // reconstruction
  T* Tt = nullptr;
  // apply workspace
  T* Z = nullptr;
  size_t Z_elems = 0;
  T* Z2 = nullptr;
  size_t Z2_elems = 0;
  T* Xs = nullptr;
  size_t Xs_elems = 0;
  T* Ys = nullptr;
  size_t Ys_elems = 0;
  // tcgen05 operands of the Kronecker-sum matvec (mixed path): Z^T and the
  // concatenated terms D^T as two scaled fp16 planes each, K-major; tcmx:
  // max |X|, max |C|, max row L1 of C, max |D|; tcsc: the scales from them
  uint16_t* Zp = nullptr;
  size_t Zp_elems = 0;
  int64_t Zp_K = -1;
  uint16_t* Dp = nullptr;
  size_t Dp_elems = 0;
  unsigned* tcmx = nullptr;
  float* tcsc = nullptr;
  // tcgen05 operands of the transform X x3 M (mixed t-SVDM)
  __nv_bfloat16* Xp = nullptr;             // X as [mn][Kp] planes
  __nv_bfloat16* Mp = nullptr;             // M as [p][Kp] planes
  int64_t Mkp = 0;
  int64_t Dp_K = -1;
  bool dp_valid = false;
  // tcgen05 operands of the mid-index contraction: the right-hand sides as
  // [(c + n s)][Kq] planes and the terms C_j as [(a + ell j)][Kq] planes
  uint16_t* Xq = nullptr;
  size_t Xq_elems = 0;
  int64_t Xq_shape = -1;
  uint16_t* Cq = nullptr;
  size_t Cq_elems = 0;
  bool cq_valid = false;
  // tcgen05 operands of the block-low-rank and SPD matvecs: the compressed
  // factors (the A operands of their products) as scaled fp16 planes, built
  // on first use after a compression
  struct TcOperand {
    const void* src = nullptr;
    int M = 0, K = 0;
    int64_t rs = 0, cs = 0, Kp = 0;
    uint16_t* planes = nullptr;
    size_t elems = 0;
    unsigned* mx = nullptr;   // max |A|
    float* s = nullptr;       // its power-of-two scale
    bool valid = false;
  };
  std::vector<TcOperand> tca;
  // Section 5.2 (SMA_TUCKER_SPD): T_0 = L L^T is split off the diagonal and
  // every field above describes the inner problem of the A_k = L^-1 T_k L^-T
  bool spd = false;
  int k0 = -1;                              // T_0's block index in the caller's numbering
  int psrc = 0;                             // distinct blocks in the caller's input
  T* T0 = nullptr;                          // m x m
  T* Lc = nullptr;                          // L, m x m lower triangular
  T* Linv = nullptr;                        // L^-1, m x m
  T* Sx = nullptr;                          // apply workspace (I (x) L^T) X
  size_t Sx_elems = 0;
  T* Sy = nullptr;                          // apply workspace, inner product plus X'
  size_t Sy_elems = 0;
  bool compressed = false;
  bool post_batched = false;                // rebuild and report in the bin's slice_post
  // host copies of results
  int h_iscal[8] = {0};
};

// Slices of one size across all problems: one batched Jacobi launch.
template <typename T>
struct SvdBin {
  int m = 0, n = 0, count = 0;
  bool tuned = false;
  JacobiPlan jp{};
  SliceDesc<T>* desc = nullptr;   // device
  T* W = nullptr;                 // block-mode workspace
  // the slices (of problems without the QR preconditioning) whose truncated
  // rebuild and orthogonality defect run as one launch after the truncation
  PostDesc<T>* post = nullptr;    // device
  int post_count = 0;
  int pm = 0, pn = 0, pmm = 0, prc = 0, ptrans = 0;
};

}  // namespace

struct sma_ctx {
  sma_options opt{};
  cudaStream_t st = nullptr;
  int nprob = 0;
  int max_smem = 0;
  int tc_ok = 0;
  DevBuf mem;
  std::vector<Prob<double>> p64;
  std::vector<Prob<float>> p32;
  std::vector<SvdBin<double>> bins64;
  std::vector<SvdBin<float>> bins32;
  TruncDesc* tdesc = nullptr;   // device, one per t-SVDM problem (batched truncation)
  int nsm = 0;                   // SMs of the device
  // Tucker / HOSVD Grams: split-K partial products and the cooperative
  // Jacobi's barrier state, shared by the problems (one stream)
  double* gpart = nullptr;
  size_t gpart_elems = 0;
  unsigned* coop_bar = nullptr;
  int* coop_rot = nullptr;
  int* coop_abort = nullptr;
  // CUDA graph of sma_compress (options.graph)
  std::vector<const void*> warm_ptrs, graph_ptrs;
  // the problems' device status words, contiguous
  int* status_pool = nullptr;
  int status_used = 0;
  // the batched gather's descriptors (host copy as last uploaded, device)
  std::vector<GatherDesc> gdesc_host;
  GatherDesc* gdesc_dev = nullptr;
  int gdesc_parts = 0;
  std::vector<int64_t> warm_lda, graph_lda;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_launches = 0;
  bool capturing = false;
  // profiling: CUDA events around each stage on the handle's stream
  bool prof = false;
  struct Pend {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> ev_free, ev_all;
  std::vector<Pend> pend;
  cudaEvent_t cur_a = nullptr;
  int cur_stage = -1;
  double acc_ms[SMA_STAGE_COUNT] = {0};
  int64_t acc_calls[SMA_STAGE_COUNT] = {0};
  int64_t launches = 0;
  // the B operand of the block-low-rank matvecs' tcgen05 products (scaled
  // fp16 planes), its maximum and the product's scales
  uint16_t* tcb = nullptr;
  size_t tcb_elems = 0;
  unsigned* tcb_mx = nullptr;
  float* tcb_sc = nullptr;
  // many-problem t-SVDM: the problems' transforms (independent products,
  // each on its own buffers) fan out over these streams, forked from and
  // joined back into the handle's stream by events (graph capture records
  // the fork and join as edges)
  static constexpr int kAux = 8;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kAux] = {};
  int naux = 0;
  ~sma_ctx() {
    for (cudaEvent_t e : ev_all) cudaEventDestroy(e);
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    for (int k = 0; k < naux; ++k) {
      cudaStreamDestroy(aux[k]);
      cudaEventDestroy(join_ev[k]);
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
  }
};

namespace {

cudaEvent_t ev_get(sma_ctx* h) {
  if (!h->ev_free.empty()) {
    cudaEvent_t e = h->ev_free.back();
    h->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  h->ev_all.push_back(e);
  return e;
}

void stage_begin(sma_ctx* h, int s) {
  if (!h->prof || h->capturing) return;
  h->cur_a = ev_get(h);
  if (h->cur_a) cudaEventRecord(h->cur_a, h->st);
  h->cur_stage = h->cur_a ? s : -1;
}

void stage_end(sma_ctx* h) {
  if (!h->prof || h->capturing || h->cur_stage < 0) return;
  cudaEvent_t b = ev_get(h);
  if (b) {
    cudaEventRecord(b, h->st);
    h->pend.push_back({h->cur_stage, h->cur_a, b});
  }
  h->cur_stage = -1;
}

// every kernel launch of the library goes through SMA_K (counted)
#define SMA_K(...)          \
  do {                      \
    ++h->launches;          \
    SMA_CK(__VA_ARGS__);    \
  } while (0)

template <typename T>
std::vector<Prob<T>>& probs(sma_ctx* h);
template <>
std::vector<Prob<double>>& probs<double>(sma_ctx* h) { return h->p64; }
template <>
std::vector<Prob<float>>& probs<float>(sma_ctx* h) { return h->p32; }
template <typename T>
std::vector<SvdBin<T>>& bins(sma_ctx* h);
template <>
std::vector<SvdBin<double>>& bins<double>(sma_ctx* h) { return h->bins64; }
template <>
std::vector<SvdBin<float>>& bins<float>(sma_ctx* h) { return h->bins32; }

// Section 7.2: one map per level; every index of level t occurs.
sma_status validate_levels(const sma_problem& pr, std::vector<int64_t> eta[3]) {
  if (pr.levels != 2 && pr.levels != 3) return SMA_ERR_UNSUPPORTED;
  if (pr.levels == 3 && (pr.m != 1 || pr.n != 1)) return SMA_ERR_ARG;
  if (pr.m <= 0 || pr.n <= 0) return SMA_ERR_ARG;
  if (!pr.level_ell || !pr.level_q || !pr.level_p || !pr.level_maps) return SMA_ERR_ARG;
  for (int t = 0; t < pr.levels; ++t) {
    const int ell = pr.level_ell[t], q = pr.level_q[t], p = pr.level_p[t];
    const int32_t* map = pr.level_maps[t];
    if (ell <= 0 || q <= 0 || p <= 0 || !map) return SMA_ERR_ARG;
    if ((int64_t)p > (int64_t)ell * q) return SMA_ERR_STRUCT;
    eta[t].assign(p, 0);
    for (int64_t e = 0; e < (int64_t)ell * q; ++e) {
      const int k = map[e];
      if (k < -1 || k >= p) return SMA_ERR_STRUCT;
      if (k >= 0) ++eta[t][k];
    }
    for (int k = 0; k < p; ++k)
      if (eta[t][k] == 0) return SMA_ERR_STRUCT;
  }
  return SMA_OK;
}

sma_status validate_problem(const sma_problem& pr, std::vector<int64_t>& eta,
                            std::vector<int>& ra, std::vector<int>& rb) {
  if (pr.levels != 0 && pr.levels != 1) return SMA_ERR_UNSUPPORTED;
  if (pr.ell <= 0 || pr.q <= 0 || pr.m <= 0 || pr.n <= 0 || pr.p <= 0) return SMA_ERR_ARG;
  if (!pr.block_map) return SMA_ERR_ARG;
  if ((int64_t)pr.p > (int64_t)pr.ell * pr.q) return SMA_ERR_STRUCT;
  eta.assign(pr.p, 0);
  ra.assign(pr.p, -1);
  rb.assign(pr.p, -1);
  for (int b = 0; b < pr.q; ++b)
    for (int a = 0; a < pr.ell; ++a) {
      const int k = pr.block_map[a + (size_t)b * pr.ell];
      if (k < -1 || k >= pr.p) return SMA_ERR_STRUCT;
      if (k < 0) continue;
      if (eta[k]++ == 0) {
        ra[k] = a;
        rb[k] = b;
      }
    }
  for (int k = 0; k < pr.p; ++k)
    if (eta[k] == 0) return SMA_ERR_STRUCT;
  return SMA_OK;
}

// Mixed path: the transform runs on tcgen05 (M' = m n rows, N' = p in tiles of 256,
// K = p); M's split planes are built once here.
// Section 5.2 writes an SPD block matrix as T = I (x) T_0 + sum_k E_k (x) T_k:
// k0 is the block index that fills the diagonal (and occurs nowhere else),
// inner the map of the remaining blocks renumbered 0..p-2 with T_0's
// positions empty.  The map must already have passed validate_problem.
sma_status spd_split(const sma_problem& pr, int* k0, std::vector<int32_t>& inner) {
  if (pr.m != pr.n || pr.ell != pr.q) return SMA_ERR_ARG;
  if (pr.p < 2) return SMA_ERR_STRUCT;
  const int ell = pr.ell;
  const int32_t* map = pr.block_map;
  const int32_t d = map[0];
  if (d < 0) return SMA_ERR_STRUCT;
  inner.assign((size_t)ell * ell, -1);
  for (int b = 0; b < ell; ++b)
    for (int a = 0; a < ell; ++a) {
      const int32_t v = map[a + (size_t)b * ell];
      if ((a == b) != (v == d)) return SMA_ERR_STRUCT;
      inner[a + (size_t)b * ell] = v == d ? -1 : (v > d ? v - 1 : v);
    }
  *k0 = d;
  return SMA_OK;
}

template <typename T>
sma_status setup_tc_transform(sma_ctx*, Prob<T>&) {
  return SMA_OK;
}
template <>
sma_status setup_tc_transform<float>(sma_ctx* h, Prob<float>& P) {
  if (!h->tc_ok || P.p > 65535) return SMA_OK;
  const int64_t Kp = tc_pad_k(P.p), mn = (int64_t)P.m * P.n;
  SMA_TRY(h->mem.alloc(&P.Xp, (size_t)3 * mn * Kp));
  SMA_TRY(h->mem.alloc(&P.Mp, (size_t)3 * P.p * Kp));
  SMA_CK(cudaMemset(P.Xp, 0, sizeof(__nv_bfloat16) * (size_t)3 * mn * Kp));
  SMA_CK(cudaMemset(P.Mp, 0, sizeof(__nv_bfloat16) * (size_t)3 * P.p * Kp));
  // plane element (i, k) = M[i, k] (M column-major, ld p)
  ++h->launches;
  SMA_CK(tc_split_transpose(P.Mt, 1, P.p, P.p, P.p, Kp, P.Mp, nullptr));
  SMA_CK(cudaDeviceSynchronize());
  P.Mkp = Kp;
  return SMA_OK;
}

// Per-slot pointers of the Gram eigen-solves (Gram, unused W output,
// eigenvectors, eigenvalues, sweep count), so that Grams of one order can be
// solved by one launch.
template <typename T>
sma_status setup_gram_desc(sma_ctx* h, Prob<T>& P, int nslot) {
  std::vector<SliceDesc<double>> d(nslot);
  for (int sl = 0; sl < nslot; ++sl)
    d[sl] = SliceDesc<double>{P.gram + (size_t)sl * P.gstride, P.gW + (size_t)sl * P.gstride,
                              P.gvec + (size_t)sl * P.gstride, P.gsig + (size_t)sl * P.gdim,
                              P.sweeps + sl, P.status};
  SMA_TRY(h->mem.alloc(&P.gdesc, (size_t)nslot));
  SMA_CK(cudaMemcpy(P.gdesc, d.data(), d.size() * sizeof(SliceDesc<double>), cudaMemcpyHostToDevice));
  return SMA_OK;
}

// Buffers of the mixed path's Gram eigen-solves (fp32 Jacobi, then the fp64
// residual correction) for nslot Gram slots; nothing for the fp64 path.
template <typename T>
sma_status setup_gram_mixed(sma_ctx* h, Prob<T>& P, int nslot) {
  if constexpr (std::is_same<T, float>::value) {
    const size_t gs = P.gstride;
    DevBuf& mem = h->mem;
    SMA_TRY(mem.alloc(&P.g32, gs * nslot));
    SMA_TRY(mem.alloc(&P.gv32, gs * nslot));
    SMA_TRY(mem.alloc(&P.gw32, gs * nslot));
    SMA_TRY(mem.alloc(&P.wg32, gs * 2));
    SMA_TRY(mem.alloc(&P.gS, gs * nslot));
    SMA_TRY(mem.alloc(&P.gZ, gs * nslot));
    SMA_TRY(mem.alloc(&P.gT1, gs));
    SMA_TRY(mem.alloc(&P.gT2, gs));
    SMA_TRY(mem.alloc(&P.sweepsS, nslot));
    std::vector<SliceDesc<float>> d32(nslot);
    std::vector<SliceDesc<double>> dS(nslot);
    for (int sl = 0; sl < nslot; ++sl) {
      d32[sl] = SliceDesc<float>{P.g32 + (size_t)sl * gs, P.gw32 + (size_t)sl * gs,
                                 P.gv32 + (size_t)sl * gs, P.gsig + (size_t)sl * P.gdim,
                                 P.sweeps + sl, P.status};
      dS[sl] = SliceDesc<double>{P.gS + (size_t)sl * gs, P.gW + (size_t)sl * gs,
                                 P.gZ + (size_t)sl * gs, P.gsig + (size_t)sl * P.gdim,
                                 P.sweepsS + sl, P.status};
    }
    SMA_TRY(mem.alloc(&P.gdesc32, (size_t)nslot));
    SMA_TRY(mem.alloc(&P.gdescS, (size_t)nslot));
    SMA_CK(cudaMemcpy(P.gdesc32, d32.data(), nslot * sizeof(SliceDesc<float>),
                      cudaMemcpyHostToDevice));
    SMA_CK(cudaMemcpy(P.gdescS, dS.data(), nslot * sizeof(SliceDesc<double>),
                      cudaMemcpyHostToDevice));
  }
  return SMA_OK;
}

template <typename T>
sma_status setup_multilevel(sma_ctx* h, Prob<T>& P, const sma_problem& pr) {
  auto& mem = h->mem;
  std::vector<int64_t> eta[3];
  SMA_TRY(validate_levels(pr, eta));
  P.L = 3;
  P.m = P.n = 1;
  P.ell = P.q = 1;
  int gdim = 1;
  for (int t = 0; t < 3; ++t) {
    P.lell[t] = pr.level_ell[t];
    P.lq[t] = pr.level_q[t];
    P.lp[t] = pr.level_p[t];
    P.ell *= P.lell[t];
    P.q *= P.lq[t];
    gdim = P.lp[t] > gdim ? P.lp[t] : gdim;
    P.lmap[t].assign(pr.level_maps[t], pr.level_maps[t] + (size_t)P.lell[t] * P.lq[t]);
    std::vector<double> w(P.lp[t]), isq(P.lp[t]);
    for (int k = 0; k < P.lp[t]; ++k) {
      w[k] = std::sqrt((double)eta[t][k]);
      isq[k] = 1.0 / w[k];
    }
    SMA_TRY(mem.alloc(&P.d_lmap[t], P.lmap[t].size()));
    SMA_TRY(mem.alloc(&P.d_lw[t], P.lp[t]));
    SMA_TRY(mem.alloc(&P.d_lisq[t], P.lp[t]));
    SMA_TRY(mem.alloc(&P.Uml[t], (size_t)P.lp[t] * P.lp[t]));
    SMA_CK(cudaMemcpy(P.d_lmap[t], P.lmap[t].data(), P.lmap[t].size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice));
    SMA_CK(cudaMemcpy(P.d_lw[t], w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
    SMA_CK(cudaMemcpy(P.d_lisq[t], isq.data(), isq.size() * sizeof(double), cudaMemcpyHostToDevice));
    // compressed-row list of the map (rows a, nonzero positions in column order)
    std::vector<int> rp(P.lell[t] + 1, 0), cl, kk;
    for (int a = 0; a < P.lell[t]; ++a) {
      for (int b = 0; b < P.lq[t]; ++b) {
        const int k = P.lmap[t][(size_t)a + (size_t)b * P.lell[t]];
        if (k >= 0) {
          cl.push_back(b);
          kk.push_back(k);
        }
      }
      rp[a + 1] = (int)cl.size();
    }
    P.lnnz[t] = (int)cl.size();
    SMA_TRY(mem.alloc(&P.d_lptr[t], rp.size()));
    SMA_TRY(mem.alloc(&P.d_lcol[t], cl.size() > 0 ? cl.size() : 1));
    SMA_TRY(mem.alloc(&P.d_lkk[t], kk.size() > 0 ? kk.size() : 1));
    SMA_CK(cudaMemcpy(P.d_lptr[t], rp.data(), rp.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!cl.empty()) {
      SMA_CK(cudaMemcpy(P.d_lcol[t], cl.data(), cl.size() * sizeof(int), cudaMemcpyHostToDevice));
      SMA_CK(cudaMemcpy(P.d_lkk[t], kk.data(), kk.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  SMA_TRY(mem.alloc(&P.mlc1, (size_t)P.lp[0] * (P.lnnz[0] > 0 ? P.lnnz[0] : 1)));
  SMA_TRY(mem.alloc(&P.mlc2, (size_t)P.lp[1] * (P.lnnz[1] > 0 ? P.lnnz[1] : 1)));
  SMA_TRY(mem.alloc(&P.mlcb, (size_t)P.lp[0] * P.lp[1] * (P.lnnz[2] > 0 ? P.lnnz[2] : 1)));
  P.p = P.lp[0] * P.lp[1] * P.lp[2];
  const size_t np = (size_t)P.p;
  P.gdim = gdim;
  P.gstride = (size_t)gdim * gdim;
  SMA_TRY(mem.alloc(&P.X, np));
  SMA_TRY(mem.alloc(&P.X64, np));
  SMA_TRY(mem.alloc(&P.Xu, np));
  SMA_TRY(mem.alloc(&P.Tt, np));
  SMA_TRY(mem.alloc(&P.T1, np));
  SMA_TRY(mem.alloc(&P.T2, np));
  SMA_TRY(mem.alloc(&P.Gc, np));
  SMA_TRY(mem.alloc(&P.Gcmp, np));
  P.nparts = gather_parts(1, 1, P.p);
  SMA_TRY(mem.alloc(&P.partial, P.nparts));
  SMA_TRY(mem.alloc(&P.stats, 8));
  SMA_TRY(mem.alloc(&P.iscal, 8));
  P.status = h->status_pool + h->status_used++;   // one pool: one clear per compression
  SMA_TRY(mem.alloc(&P.gram, P.gstride * 3));
  SMA_TRY(mem.alloc(&P.gvec, P.gstride * 3));
  SMA_TRY(mem.alloc(&P.gsig, (size_t)gdim * 3));
  SMA_TRY(mem.alloc(&P.suf, (size_t)(gdim + 1) * 3));
  SMA_TRY(mem.alloc(&P.Wg, P.gstride * 2));
  SMA_TRY(mem.alloc(&P.gW, P.gstride * 3));
  SMA_TRY(mem.alloc(&P.sweeps, 3));
  SMA_TRY(mem.alloc(&P.ranks, 3));
  SMA_TRY(mem.alloc(&P.off, 4));
  SMA_TRY(mem.alloc(&P.orth, 3));
  SMA_TRY(setup_gram_desc(h, P, 3));
  SMA_TRY(setup_gram_mixed(h, P, 3));
  SMA_TRY(mem.alloc(&P.Gorth, P.gstride));
  P.n_orth = 3;
  SMA_CK(cudaMemset(P.stats, 0, 8 * sizeof(double)));
  SMA_CK(cudaMemset(P.iscal, 0, 8 * sizeof(int)));
  SMA_CK(cudaMemset(P.status, 0, sizeof(int)));
  return SMA_OK;
}

template <typename T>
sma_status setup_problem(sma_ctx* h, Prob<T>& P, const sma_problem& pr) {
  auto& mem = h->mem;
  const sma_options& o = h->opt;
  sma_problem pin = pr;
  std::vector<int32_t> inner;
  if (o.decomp == SMA_HOSVD_MULTILEVEL) {
    if (pr.levels != 2) return setup_multilevel(h, P, pr);
    // two levels, m x n blocks: the one-level product map, level 1 outermost
    // (block row a1 ell2 + a2, column b1 q2 + b2, block index i1 + p1 i2)
    std::vector<int64_t> leta[3];
    SMA_TRY(validate_levels(pr, leta));
    const int l1 = pr.level_ell[0], q1 = pr.level_q[0], p1 = pr.level_p[0];
    const int l2 = pr.level_ell[1], q2 = pr.level_q[1], p2 = pr.level_p[1];
    inner.assign((size_t)l1 * l2 * q1 * q2, -1);
    const int64_t L = (int64_t)l1 * l2;
    for (int b1 = 0; b1 < q1; ++b1)
      for (int a1 = 0; a1 < l1; ++a1) {
        const int i1 = pr.level_maps[0][a1 + (size_t)b1 * l1];
        if (i1 < 0) continue;
        for (int b2 = 0; b2 < q2; ++b2)
          for (int a2 = 0; a2 < l2; ++a2) {
            const int i2 = pr.level_maps[1][a2 + (size_t)b2 * l2];
            if (i2 >= 0) inner[(a1 * l2 + a2) + (size_t)(b1 * q2 + b2) * L] = i1 + p1 * i2;
          }
      }
    pin.levels = 1;
    pin.ell = l1 * l2;
    pin.q = q1 * q2;
    pin.p = p1 * p2;
    pin.block_map = inner.data();
    P.ml2 = true;
    P.lell[0] = l1; P.lq[0] = q1; P.lp[0] = p1;
    P.lell[1] = l2; P.lq[1] = q2; P.lp[1] = p2;
  }
  if (o.decomp == SMA_TUCKER_SPD) {
    SMA_TRY(validate_problem(pr, P.eta, P.rep_a, P.rep_b));
    SMA_TRY(spd_split(pr, &P.k0, inner));
    pin.block_map = inner.data();
    pin.p = pr.p - 1;
    P.spd = true;
  }
  P.psrc = pr.p;
  SMA_TRY(validate_problem(pin, P.eta, P.rep_a, P.rep_b));
  P.ell = pin.ell; P.q = pin.q; P.m = pin.m; P.n = pin.n; P.p = pin.p;
  P.map.assign(pin.block_map, pin.block_map + (size_t)pin.ell * pin.q);
  const int m = P.m, n = P.n, p = P.p;
  const size_t mnp = (size_t)m * n * p;
  std::vector<double> w(p), isq(p);
  for (int k = 0; k < p; ++k) {
    w[k] = std::sqrt((double)P.eta[k]);
    isq[k] = 1.0 / w[k];
  }
  SMA_TRY(mem.alloc(&P.d_map, P.map.size()));
  SMA_TRY(mem.alloc(&P.d_w, p));
  SMA_TRY(mem.alloc(&P.d_isq, p));
  SMA_TRY(mem.alloc(&P.d_rep, p));
  SMA_CK(cudaMemcpy(P.d_map, P.map.data(), P.map.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  {  // the structure's nonzero positions: the Kronecker factors are written there only
    std::vector<int> nzpos, nzk;
    for (size_t pos = 0; pos < P.map.size(); ++pos)
      if (P.map[pos] >= 0) {
        nzpos.push_back((int)pos);
        nzk.push_back(P.map[pos]);
      }
    P.nnz = (int)nzpos.size();
    SMA_TRY(mem.alloc(&P.d_nzpos, nzpos.size()));
    SMA_TRY(mem.alloc(&P.d_nzk, nzk.size()));
    if (P.nnz > 0) {
      SMA_CK(cudaMemcpy(P.d_nzpos, nzpos.data(), nzpos.size() * sizeof(int), cudaMemcpyHostToDevice));
      SMA_CK(cudaMemcpy(P.d_nzk, nzk.data(), nzk.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  SMA_CK(cudaMemcpy(P.d_w, w.data(), p * sizeof(double), cudaMemcpyHostToDevice));
  SMA_CK(cudaMemcpy(P.d_isq, isq.data(), p * sizeof(double), cudaMemcpyHostToDevice));
  {
    std::vector<float> wf(2 * (size_t)p);
    for (int k = 0; k < p; ++k) {
      wf[2 * k] = (float)w[k];
      wf[2 * k + 1] = (float)(w[k] - (double)wf[2 * k]);
    }
    SMA_TRY(mem.alloc(&P.d_wf, wf.size()));
    SMA_CK(cudaMemcpy(P.d_wf, wf.data(), wf.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  SMA_TRY(mem.alloc(&P.X, mnp));
  P.nparts = gather_parts(m, n, p);
  SMA_TRY(mem.alloc(&P.partial, P.nparts));
  SMA_TRY(mem.alloc(&P.stats, 8));
  SMA_TRY(mem.alloc(&P.iscal, 8));
  P.status = h->status_pool + h->status_used++;   // one pool: one clear per compression
  SMA_TRY(mem.alloc(&P.Tt, mnp));
  SMA_CK(cudaMemset(P.stats, 0, 8 * sizeof(double)));
  SMA_CK(cudaMemset(P.iscal, 0, 8 * sizeof(int)));
  SMA_CK(cudaMemset(P.status, 0, sizeof(int)));
  if (P.ell == P.q && m == n && !P.spd) {
    P.trw.assign(p, 0.0);
    for (int a = 0; a < P.ell; ++a) {
      const int k = P.map[(size_t)a + (size_t)a * P.ell];
      if (k >= 0) P.trw[k] += isq[k];
    }
    SMA_TRY(mem.alloc(&P.traces, 2 * (size_t)p));
  }

  if (o.decomp == SMA_TSVDM) {
    std::vector<double> M;
    if (o.mkind == SMA_M_DCT2) {
      M = dct2(p);
    } else if (o.mkind == SMA_M_IDENTITY) {
      M.assign((size_t)p * p, 0.0);
      for (int k = 0; k < p; ++k) M[k + (size_t)k * p] = 1.0;
    } else {
      if (!o.M_user) return SMA_ERR_ARG;
      M.assign(o.M_user, o.M_user + (size_t)p * p);
    }
    P.Mh = M;
    std::vector<T> Mt(M.begin(), M.end());
    SMA_TRY(mem.alloc(&P.Mt, (size_t)p * p));
    SMA_CK(cudaMemcpy(P.Mt, Mt.data(), Mt.size() * sizeof(T), cudaMemcpyHostToDevice));
    SMA_TRY(setup_tc_transform(h, P));
    P.trans = m < n ? 1 : 0;
    P.mm = m < n ? n : m;
    P.rc = m < n ? m : n;
    P.qplan = qr_plan<T>(P.mm, P.rc, h->max_smem);
    const bool qr_fits = P.qplan.smem_qr <= (size_t)h->max_smem &&
                         P.qplan.smem_fin <= (size_t)h->max_smem && P.qplan.fslot >= 0;
    P.qr = qr_fits && (o.precondition == SMA_PRECOND_QRCP || o.precondition == SMA_PRECOND_QRCP2 ||
                       (o.precondition == SMA_PRECOND_AUTO && P.rc >= kQrAutoMin));
    P.qr2 = P.qr && P.mm <= kQrWarpRows &&
            (o.precondition == SMA_PRECOND_QRCP2 ||
             (o.precondition == SMA_PRECOND_AUTO && P.rc >= kQr2AutoMin));
    // one fp32 problem per handle: the rotation-log Jacobi where the shape
    // allows it (the batched path keeps V in its kernel)
    const bool rec = sizeof(T) == 4 && h->nprob == 1;
    const int jm = P.qr ? P.rc : m, jn = P.qr ? P.rc : n;
    P.jp = jacobi_plan<T>(jm, jn, h->max_smem, rec);
    if (P.jp.smem == 0) return SMA_ERR_UNSUPPORTED;   // a column too long for shared memory
    if (P.jp.rec) {
      // the log for the largest geometry among the autotuner's candidates
      const int lsw = jacobi_log_sweeps(h->opt.max_sweeps > 0 ? h->opt.max_sweeps : 30);
      size_t lf = 0;
      for (const JacobiPlan& c : jacobi_plan_candidates<T>(jm, jn, h->max_smem, true))
        lf = std::max(lf, jacobi_log_size(c, lsw));
      P.vlog_bs = (int64_t)lf;
      SMA_TRY(mem.alloc(&P.vlog, lf * p));
      SMA_TRY(mem.alloc(&P.vorder, (size_t)P.rc * p));
      SMA_TRY(mem.alloc(&P.vlsw, (size_t)p));
    }
    SMA_TRY(mem.alloc(&P.Xh, mnp));
    if (P.jp.block_mode)
      SMA_TRY(mem.alloc(&P.Wj, (size_t)(P.jp.mm + P.jp.rc) * P.jp.rc * p));
    SMA_TRY(mem.alloc(&P.U, (size_t)P.jp.mm * P.rc * p));
    if (P.qr) {
      const size_t frc = (size_t)P.mm * P.rc * p, rr = (size_t)P.rc * P.rc * p;
      SMA_TRY(mem.alloc(&P.qF, frc));
      if (P.qplan.novf > 0) SMA_TRY(mem.alloc(&P.qG, (size_t)P.mm * P.qplan.novf * p));
      SMA_TRY(mem.alloc(&P.qtau, (size_t)P.rc * p));
      SMA_TRY(mem.alloc(&P.qperm, (size_t)P.rc * p));
      SMA_TRY(mem.alloc(&P.qJ, rr));
      SMA_TRY(mem.alloc(&P.qRt, rr));
      SMA_TRY(mem.alloc(&P.qL, frc));
    }
    if (P.qr2) {
      const size_t rr = (size_t)P.rc * P.rc * p;
      SMA_TRY(mem.alloc(&P.qF2, rr));
      SMA_TRY(mem.alloc(&P.qtau2, (size_t)P.rc * p));
      SMA_TRY(mem.alloc(&P.qperm2, (size_t)P.rc * p));
      SMA_TRY(mem.alloc(&P.qJ2, rr));
    }
    SMA_TRY(mem.alloc(&P.V, (size_t)P.rc * P.rc * p));
    SMA_TRY(mem.alloc(&P.sigma, (size_t)P.rc * p));
    SMA_TRY(mem.alloc(&P.suf, (size_t)(P.rc + 1) * p));
    SMA_TRY(mem.alloc(&P.sweeps, p));
    SMA_TRY(mem.alloc(&P.ranks, p));
    SMA_TRY(mem.alloc(&P.off, p + 1));
    SMA_TRY(mem.alloc(&P.orth, p));
    P.n_orth = p;
    P.nterms_max = p;
    SMA_TRY(mem.alloc(&P.D, mnp));
    SMA_TRY(mem.alloc(&P.C, (size_t)P.ell * P.q * p));
    SMA_CK(cudaMemset(P.C, 0, sizeof(T) * (size_t)P.ell * P.q * p));   // zero off the structure
    // the structured Kronecker factors C_i = struct_E(M[i, :]) depend only on
    // M and the map: built once here, not in every compression
    ++h->launches;
    SMA_CK(build_struct_terms_nz<T>(P.d_nzpos, P.d_nzk, P.nnz, P.d_isq, P.ell, P.q, P.Mt, 1, p, p,
                                    nullptr, P.C, nullptr));
    SMA_CK(cudaDeviceSynchronize());
  } else if (o.decomp == SMA_CP_ALS) {
    const int r = o.fixed_rank;
    if (r > p) return SMA_ERR_ARG;
    P.cp_r = r;
    const size_t big = std::max({(size_t)m * n, (size_t)n * p, (size_t)m * p});
    SMA_TRY(mem.alloc(&P.cXf, (size_t)m * r));
    SMA_TRY(mem.alloc(&P.cZf, (size_t)n * r));
    SMA_TRY(mem.alloc(&P.cXf0, (size_t)m * r));
    SMA_TRY(mem.alloc(&P.cZf0, (size_t)n * r));
    SMA_TRY(mem.alloc(&P.cKR, big * r));
    SMA_TRY(mem.alloc(&P.cM, (size_t)std::max({m, n, p}) * r));
    // per-block partials of the mode-2 contraction, or split-K partials of
    // the other two (at most 2 nsm / tiles + 1 chunks of M x r)
    P.cSlab_elems = std::max((size_t)p * n * r,
                             (size_t)(2 * h->nsm + 1) * std::max({m, n, p}) * r);
    SMA_TRY(mem.alloc(&P.cSlab, P.cSlab_elems));
    std::vector<T> x0(o.cp_init_x, o.cp_init_x + (size_t)m * r);
    std::vector<T> z0(o.cp_init_z, o.cp_init_z + (size_t)n * r);
    SMA_CK(cudaMemcpy(P.cXf0, x0.data(), x0.size() * sizeof(T), cudaMemcpyHostToDevice));
    SMA_CK(cudaMemcpy(P.cZf0, z0.data(), z0.size() * sizeof(T), cudaMemcpyHostToDevice));
    SMA_TRY(mem.alloc(&P.F1, (size_t)p * p));        // Yf (p x r)
    SMA_TRY(mem.alloc(&P.D, mnp));                   // Xf[:, j] Zf[:, j]^T (m x n x r)
    SMA_TRY(mem.alloc(&P.C, (size_t)P.ell * P.q * p));
    SMA_CK(cudaMemset(P.C, 0, sizeof(T) * (size_t)P.ell * P.q * p));
    SMA_TRY(mem.alloc(&P.orth, 1));
    SMA_TRY(mem.alloc(&P.sweeps, 1));
    P.n_orth = 0;
    P.nterms_max = p;
  } else {
    // Tucker family: fp64 Gram and its Jacobi eigen-solve
    int gdim = 0;
    if (o.decomp == SMA_TUCKER_BLOCKMODE) {
      gdim = p;
      P.sk = o.sketch_cols > 0 ? o.sketch_cols : 0;
      if (P.sk * P.sk > gdim) gdim = P.sk * P.sk;
    }
    else if (o.decomp == SMA_TUCKER_SHARED_U || o.decomp == SMA_TUCKER_SPD) gdim = m;
    else if (o.decomp == SMA_TUCKER_ROWCOL) gdim = (m > n ? m : n);
    else if (P.ml2) gdim = std::max({m, n, P.lp[0], P.lp[1]});
    else return SMA_ERR_UNSUPPORTED;
    if ((o.decomp == SMA_TUCKER_SHARED_U || o.decomp == SMA_TUCKER_SPD) && m != n)
      return SMA_ERR_ARG;
    if (P.sk > 0 && o.fixed_rank > p) return SMA_ERR_ARG;
    P.gdim = gdim;
    P.gstride = (size_t)gdim * gdim;
    if (P.sk == 0) {
      // the fp64 copy of X the Grams are formed from (the sketch forms its own)
      SMA_TRY(mem.alloc(&P.X64, mnp));
      SMA_TRY(mem.alloc(&P.Xu, mnp));
    }
    const int nslot = P.ml2 ? 4 : 2;
    SMA_TRY(mem.alloc(&P.Wg, (size_t)gdim * gdim * 2));
    SMA_TRY(mem.alloc(&P.gW, (size_t)gdim * gdim * nslot));
    SMA_TRY(mem.alloc(&P.gram, (size_t)gdim * gdim * nslot));
    SMA_TRY(mem.alloc(&P.gvec, (size_t)gdim * gdim * nslot));
    SMA_TRY(mem.alloc(&P.gsig, (size_t)gdim * nslot));
    SMA_TRY(mem.alloc(&P.suf, (size_t)(gdim + 1) * nslot));
    SMA_TRY(mem.alloc(&P.sweeps, nslot));
    SMA_TRY(mem.alloc(&P.ranks, nslot));
    SMA_TRY(mem.alloc(&P.off, nslot + 1));
    SMA_TRY(mem.alloc(&P.orth, nslot));
    SMA_TRY(setup_gram_desc(h, P, nslot));
    SMA_TRY(setup_gram_mixed(h, P, nslot));
    P.n_orth = P.ml2 ? 4 : ((o.decomp == SMA_TUCKER_ROWCOL) ? 2 : 1);
    if (P.sk > 0) {
      const int s2 = P.sk * P.sk;
      SMA_TRY(mem.alloc(&P.Om, (size_t)m * P.sk));
      SMA_TRY(mem.alloc(&P.Ps, (size_t)n * P.sk));
      SMA_TRY(mem.alloc(&P.Ysk, (size_t)s2 * p));
      SMA_TRY(mem.alloc(&P.Y64, (size_t)s2 * p));
      SMA_TRY(mem.alloc(&P.Ytmp, (size_t)P.sk * n * p));
      std::vector<T> om(o.sketch_omega, o.sketch_omega + (size_t)m * P.sk);
      std::vector<T> ps(o.sketch_psi, o.sketch_psi + (size_t)n * P.sk);
      SMA_CK(cudaMemcpy(P.Om, om.data(), om.size() * sizeof(T), cudaMemcpyHostToDevice));
      SMA_CK(cudaMemcpy(P.Ps, ps.data(), ps.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
    if (P.ml2) {
      const int dims[4] = {m, n, P.lp[0], P.lp[1]};
      for (int t = 0; t < 4; ++t) SMA_TRY(mem.alloc(&P.mlF[t], (size_t)dims[t] * dims[t]));
      SMA_TRY(mem.alloc(&P.mlT1, mnp));
      SMA_TRY(mem.alloc(&P.mlT2, mnp));
      SMA_TRY(mem.alloc(&P.mlG, mnp));
      SMA_TRY(mem.alloc(&P.mlGt, mnp));
      SMA_TRY(mem.alloc(&P.F1, (size_t)p * p));        // coefficient vectors (p x terms)
      SMA_TRY(mem.alloc(&P.D, mnp));                   // D_t = Xf G_t Zf^T (m x n x terms)
      SMA_TRY(mem.alloc(&P.C, (size_t)P.ell * P.q * p));
      SMA_CK(cudaMemset(P.C, 0, sizeof(T) * (size_t)P.ell * P.q * p));
      SMA_TRY(mem.alloc(&P.Gorth, (size_t)gdim * gdim));
      P.nterms_max = p;
    } else if (o.decomp == SMA_TUCKER_BLOCKMODE) {
      SMA_TRY(mem.alloc(&P.F1, (size_t)p * p));        // V (p x r)
      SMA_TRY(mem.alloc(&P.D, mnp));                   // G_j slices (m x n x r)
      SMA_TRY(mem.alloc(&P.C, (size_t)P.ell * P.q * p));
      SMA_CK(cudaMemset(P.C, 0, sizeof(T) * (size_t)P.ell * P.q * p));
      SMA_TRY(mem.alloc(&P.Gorth, (size_t)p * p));
      P.nterms_max = p;
    } else {
      P.r1max = m;
      P.r3max = (o.decomp == SMA_TUCKER_SHARED_U || o.decomp == SMA_TUCKER_SPD) ? m : n;
      SMA_TRY(mem.alloc(&P.F1, (size_t)m * m));
      SMA_TRY(mem.alloc(&P.F2, (size_t)n * n));
      SMA_TRY(mem.alloc(&P.core, (size_t)P.r1max * P.r3max * p));
      SMA_TRY(mem.alloc(&P.tmp, (size_t)(m > n ? m : n) * (m > n ? m : n) * p));
      SMA_TRY(mem.alloc(&P.mid, (size_t)P.ell * P.r1max * P.q * P.r3max));
      SMA_TRY(mem.alloc(&P.Gorth, (size_t)(m > n ? m : n) * (m > n ? m : n)));
    }
    if (P.spd) {
      SMA_TRY(mem.alloc(&P.T0, (size_t)m * m));
      SMA_TRY(mem.alloc(&P.Lc, (size_t)m * m));
      SMA_TRY(mem.alloc(&P.Linv, (size_t)m * m));
    }
  }
  return SMA_OK;
}

template <typename T>
sma_status make_T(sma_ctx* h, Prob<T>& P);
template <typename T>
sma_status contract_split_k(sma_ctx* h, GemmParams<T> g, T* part, size_t part_elems);

// ---------------------------------------------------------------------------
// step 1 (gather) shared by all decompositions
// ---------------------------------------------------------------------------
// Element offsets of the representative blocks in the input (dense layout,
// or the caller's block list), uploaded when the leading dimension or the
// layout changes.
template <typename T>
sma_status rep_offsets(sma_ctx* h, Prob<T>& P, int64_t use_lda, int layout, bool dense) {
  if (P.rep_lda == use_lda && P.rep_layout == layout) return SMA_OK;
  const int m = P.m, n = P.n, p = P.p;
  std::vector<int64_t> off(p);
  for (int k = 0; k < p; ++k) {
    // a caller's block list (not a staged copy of a dense input) also holds T_0
    const int ks = k + (P.spd && !dense && k >= P.k0 ? 1 : 0);
    off[k] = layout == 0 ? (int64_t)P.rep_a[k] * m + (int64_t)P.rep_b[k] * n * use_lda
                         : (int64_t)ks * n * use_lda;
  }
  SMA_CK(cudaMemcpyAsync(P.d_rep, off.data(), p * sizeof(int64_t), cudaMemcpyHostToDevice, h->st));
  SMA_CK(cudaStreamSynchronize(h->st));  // off[] is a stack buffer
  P.rep_lda = use_lda;
  P.rep_layout = layout;
  return SMA_OK;
}

// The gathers of every problem of the handle in one launch (several one-
// level problems with device inputs and no SPD split); false when the
// batched form does not apply and each problem gathers on its own.
template <typename T>
sma_status gather_all(sma_ctx* h, const void* const* A, const int64_t* lda, bool* done) {
  *done = false;
  auto& ps = probs<T>(h);
  if (ps.size() < 2) return SMA_OK;
  const bool dense = h->opt.layout == SMA_INPUT_DENSE;
  for (int i = 0; i < h->nprob; ++i) {
    const auto& P = ps[i];
    const int64_t need_rows = dense ? (int64_t)P.ell * P.m : P.m;
    if (P.L == 3 || P.spd || !A[i] || lda[i] < need_rows || !is_device_ptr(A[i])) return SMA_OK;
  }
  std::vector<GatherDesc> gd(h->nprob);
  int parts = 0;
  for (int i = 0; i < h->nprob; ++i) {
    auto& P = ps[i];
    SMA_TRY(rep_offsets(h, P, lda[i], dense ? 0 : 1, dense));
    gd[i] = GatherDesc{A[i], lda[i], P.d_rep, P.d_w, P.d_wf, P.m, P.n, P.p, P.X, P.partial,
                       P.stats, parts, P.nparts};
    parts += P.nparts;
  }
  auto eq = [](const GatherDesc& a, const GatherDesc& b) {
    return a.A == b.A && a.lda == b.lda && a.rep_off == b.rep_off && a.w == b.w && a.wf == b.wf &&
           a.m == b.m && a.n == b.n && a.p == b.p && a.X == b.X && a.partial == b.partial &&
           a.norm2 == b.norm2 && a.part0 == b.part0 && a.nparts == b.nparts;
  };
  bool same = gd.size() == h->gdesc_host.size();
  for (size_t i = 0; same && i < gd.size(); ++i) same = eq(gd[i], h->gdesc_host[i]);
  if (!same) {
    if (h->capturing) return SMA_OK;   // new descriptors are uploaded outside a capture only
    if (!h->gdesc_dev) SMA_TRY(h->mem.alloc(&h->gdesc_dev, (size_t)h->nprob));
    h->gdesc_host = gd;
    SMA_CK(cudaMemcpyAsync(h->gdesc_dev, h->gdesc_host.data(), gd.size() * sizeof(GatherDesc),
                           cudaMemcpyHostToDevice, h->st));
    SMA_CK(cudaStreamSynchronize(h->st));
    h->gdesc_parts = parts;
  }
  stage_begin(h, SMA_STAGE_GATHER);
  h->launches += 1;   // the norm launch (SMA_K counts the gather)
  SMA_K(gather_batched<T>(h->gdesc_dev, h->nprob, h->gdesc_parts, h->st));
  stage_end(h);
  *done = true;
  return SMA_OK;
}

template <typename T>
sma_status do_gather(sma_ctx* h, Prob<T>& P, const void* Ain, int64_t lda) {
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, p = P.p;
  const bool dense = h->opt.layout == SMA_INPUT_DENSE;
  const int64_t need_rows = dense ? (int64_t)P.ell * m : m;
  if (!Ain || lda < need_rows) return SMA_ERR_ARG;
  const T* A = static_cast<const T*>(Ain);
  stage_begin(h, SMA_STAGE_GATHER);
  int64_t use_lda = lda;
  int layout = dense ? 0 : 1;
  if (P.spd) {
    // the diagonal block T_0: block (0, 0) of the matrix, or block k0 of the list
    const T* src = A + (dense ? 0 : (int64_t)P.k0 * n * lda);
    SMA_CK(cudaMemcpy2DAsync(P.T0, m * sizeof(T), src, lda * sizeof(T), m * sizeof(T), n,
                             is_device_ptr(Ain) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             st));
  }
  const void* mapped = is_device_ptr(Ain) ? nullptr : mapped_host_ptr(Ain);
  if (mapped) {
    // page-locked host input: the gather reads the representative blocks in
    // place, over the host link, instead of staging them with copies
    A = static_cast<const T*>(mapped);
  } else if (!is_device_ptr(Ain)) {
    // pageable host input: copy only the representative blocks to a staging
    // buffer (the block list keeps the caller's numbering, T_0 included)
    if (!P.stage) SMA_TRY(h->mem.alloc(&P.stage, (size_t)m * n * (dense ? p : P.psrc)));
    if (dense) {
      for (int k = 0; k < p; ++k) {
        const T* src = A + (int64_t)P.rep_a[k] * m + (int64_t)P.rep_b[k] * n * lda;
        SMA_CK(cudaMemcpy2DAsync(P.stage + (size_t)k * m * n, m * sizeof(T), src, lda * sizeof(T),
                                 m * sizeof(T), n, cudaMemcpyHostToDevice, st));
      }
    } else {
      SMA_CK(cudaMemcpy2DAsync(P.stage, m * sizeof(T), A, lda * sizeof(T), m * sizeof(T),
                               (size_t)n * P.psrc, cudaMemcpyHostToDevice, st));
    }
    A = P.stage;
    use_lda = m;
    layout = 1;
  }
  SMA_TRY(rep_offsets(h, P, use_lda, layout, dense));
  SMA_K(gather<T, T>(A, use_lda, P.d_rep, P.d_w, P.d_wf, m, n, p, P.X, P.partial, st));
  SMA_K(finish_norm(P.partial, P.nparts, P.stats, st));
  stage_end(h);
  return SMA_OK;
}

// ---------------------------------------------------------------------------
// contraction dispatch: the mixed path sends large fp32 GEMMs to tcgen05
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t contract(sma_ctx* h, const GemmParams<T>& g) {
  return gemm<T>(g, h->st);
}
template <>
cudaError_t contract<float>(sma_ctx* h, const GemmParams<float>& g) {
  if (h->tc_ok && tc_gemm_eligible(g)) return tc_gemm_bf16x3(g, h->st);
  return gemm<float>(g, h->st);
}

// ---------------------------------------------------------------------------
// t-SVDM (steps 2-5)
// ---------------------------------------------------------------------------
// Xhat = X x3 M on tcgen05: A = X as K-major planes (element (e, k) =
// X[e + mn k]), B = M planes (element (i, k) = M[i, k]); Xhat written
// column-major (ld mn).  False when not set up for it.
template <typename T>
bool tc_transform(sma_ctx*, Prob<T>&) {
  return false;
}
template <>
bool tc_transform<float>(sma_ctx* h, Prob<float>& P) {
  if (!P.Xp || !P.Mp) return false;
  const int64_t mn = (int64_t)P.m * P.n;
  if (mn > 0x7fffffff) return false;
  ++h->launches;
  if (tc_split_transpose(P.X, 1, mn, (int)mn, P.p, P.Mkp, P.Xp, h->st) != cudaSuccess) return false;
  ++h->launches;
  return tc_gemm_planes(P.Xp, P.Mp, (int)mn, P.p, P.Mkp, P.Xh, mn, P.status, h->st, true) ==
         cudaSuccess;
}

// Xhat = X x3 M:  Xhat_mat (mn x p) = X_mat (mn x p) * M^T, on h->st
template <typename T>
sma_status transform_one(sma_ctx* h, Prob<T>& P) {
  if (tc_transform(h, P)) return SMA_OK;
  const int p = P.p;
  const int64_t mn = (int64_t)P.m * P.n;
  GemmParams<T> g;
  g.M = (int)mn; g.N = p; g.K = p;
  g.A = P.X; g.a_rs = 1; g.a_cs = mn;
  g.B = P.Mt; g.b_rs = p; g.b_cs = 1;
  g.C = P.Xh; g.c_rs = 1; g.c_cs = mn;
  SMA_K(contract<T>(h, g));
  return SMA_OK;
}

template <typename T>
sma_status tsvdm_pre(sma_ctx* h, Prob<T>& P) {
  stage_begin(h, SMA_STAGE_TRANSFORM);
  const sma_status s = transform_one(h, P);
  stage_end(h);
  return s;
}

// The transforms of all problems of a many-problem handle: problem i on
// auxiliary stream i mod naux, after everything already enqueued on the
// handle's stream, which waits for all of them before its next work.  Each
// problem's product reads and writes only its own buffers.
template <typename T>
sma_status transform_fanout(sma_ctx* h) {
  auto& ps = probs<T>(h);
  cudaStream_t main_st = h->st;
  SMA_CK(cudaEventRecord(h->fork_ev, main_st));
  for (int k = 0; k < h->naux; ++k) SMA_CK(cudaStreamWaitEvent(h->aux[k], h->fork_ev, 0));
  sma_status s = SMA_OK;
  for (int i = 0; i < h->nprob && s == SMA_OK; ++i) {
    h->st = h->aux[i % h->naux];
    s = transform_one(h, ps[i]);
  }
  h->st = main_st;
  // join every branch, also after a failed enqueue (a capture must end joined)
  for (int k = 0; k < h->naux; ++k) {
    const cudaError_t e1 = cudaEventRecord(h->join_ev[k], h->aux[k]);
    const cudaError_t e2 = cudaStreamWaitEvent(main_st, h->join_ev[k], 0);
    if (s == SMA_OK && (e1 != cudaSuccess || e2 != cudaSuccess)) s = SMA_ERR_CUDA;
  }
  return s;
}

template <typename T>
JacobiParams<T> jacobi_params(sma_ctx* h, const JacobiPlan& jp) {
  JacobiParams<T> J;
  J.mm = jp.mm; J.rc = jp.rc; J.trans = jp.trans; J.ldS = jp.ldS; J.bcols = jp.bcols;
  J.g = jp.g; J.sort_n = jp.sort_n; J.tile = jp.tile;
  J.max_sweeps = h->opt.max_sweeps > 0 ? h->opt.max_sweeps : 30;
  J.tol = 4.0 * std::sqrt((double)jp.mm) * Eps<T>::v;
  return J;
}

template <typename T>
QrParams<T> qr_params(const Prob<T>& P) {
  QrParams<T> q;
  q.src = P.Xh; q.src_bs = (int64_t)P.m * P.n;
  q.m = P.m; q.mm = P.mm; q.rc = P.rc; q.trans = P.trans;
  q.plan = P.qplan;
  q.F = P.qF; q.F_bs = (int64_t)P.mm * P.rc;
  q.G = P.qG; q.G_bs = (int64_t)P.mm * P.qplan.novf;
  q.tau = P.qtau; q.perm = P.qperm;
  q.Jin = P.qJ; q.J_bs = (int64_t)P.rc * P.rc;
  q.W = P.U; q.W_bs = (int64_t)P.rc * P.rc;
  q.V = P.V; q.V_bs = (int64_t)P.rc * P.rc;
  q.Rt = P.qRt; q.Rt_bs = (int64_t)P.rc * P.rc;
  q.L = P.qL; q.L_bs = (int64_t)P.mm * P.rc;
  return q;
}

// The second QR: R1^T (rc x rc, the first QR's Jacobi input) = Q2 R2
// (perm2 = identity).
template <typename T>
QrParams<T> qr2_params(const Prob<T>& P) {
  QrParams<T> q;
  q.src = P.qJ; q.src_bs = (int64_t)P.rc * P.rc;
  q.m = P.rc; q.mm = P.rc; q.rc = P.rc; q.trans = 0;
  q.F = P.qF2; q.F_bs = (int64_t)P.rc * P.rc;
  q.tau = P.qtau2; q.perm = P.qperm2;
  q.Jin = P.qJ2; q.J_bs = (int64_t)P.rc * P.rc;
  return q;
}

// The Jacobi input of a preconditioned problem: R2^T after two QRs, else R1^T.
template <typename T>
const T* qr_jacobi_input(const Prob<T>& P) {
  return P.qr2 ? P.qJ2 : P.qJ;
}

// Both QRs of a preconditioned problem's slices.
template <typename T>
cudaError_t qr_precondition(const Prob<T>& P, cudaStream_t st) {
  cudaError_t e = qrcp<T>(qr_params(P), P.p, st);
  if (e == cudaSuccess && P.qr2) e = qr_blocked<T>(qr2_params(P), P.p, st);
  return e;
}

// ---- autotuner of the slice-SVD plan ---------------------------------------
// On the first compression of a slice shape (options.autotune), every
// candidate plan (jacobi_plan_candidates) runs twice on the actual slices and
// the fastest second run wins; the choice is cached for the process, keyed by
// the Jacobi input shape and the element type.  The problems' device status
// words are saved and restored around the trial runs, which write only the
// outputs the real run overwrites.
std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}
std::map<uint64_t, JacobiPlan>& tune_cache() {
  static std::map<uint64_t, JacobiPlan> c;
  return c;
}

template <typename T>
sma_status tune_plan(sma_ctx* h, JacobiParams<T> J, int count, int jm, int jn, JacobiPlan& plan,
                     const std::vector<int*>& status_words) {
  const uint64_t key = ((uint64_t)(uint32_t)jm << 32) | ((uint64_t)(uint32_t)jn << 8) |
                       ((uint64_t)(plan.rec ? 1 : 0) << 4) | sizeof(T);
  {
    std::lock_guard<std::mutex> g(tune_mutex());
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {
      plan = it->second;
      return SMA_OK;
    }
  }
  cudaStream_t st = h->st;
  int* saved = nullptr;
  SMA_TRY(h->mem.alloc(&saved, status_words.size()));
  for (size_t i = 0; i < status_words.size(); ++i)
    SMA_CK(cudaMemcpyAsync(saved + i, status_words[i], sizeof(int), cudaMemcpyDeviceToDevice, st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SMA_CK(cudaEventCreate(&e0));
  SMA_CK(cudaEventCreate(&e1));
  JacobiPlan best = plan;
  float best_ms = 3.0e38f;
  cudaError_t err = cudaSuccess;
  for (const JacobiPlan& c : jacobi_plan_candidates<T>(jm, jn, h->max_smem, plan.rec != 0)) {
    if (c.block_mode != plan.block_mode) continue;
    JacobiParams<T> Jc = J;
    Jc.mm = c.mm; Jc.rc = c.rc; Jc.trans = c.trans; Jc.ldS = c.ldS; Jc.bcols = c.bcols;
    Jc.g = c.g; Jc.sort_n = c.sort_n; Jc.tile = c.tile;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
      err = cudaEventRecord(e0, st);
      if (err == cudaSuccess) err = jacobi_svd<T>(Jc, count, c.threads, c.smem, st);
      ++h->launches;
      if (err == cudaSuccess) err = cudaEventRecord(e1, st);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (err != cudaSuccess) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SMA_CK(err);
  for (size_t i = 0; i < status_words.size(); ++i)
    SMA_CK(cudaMemcpyAsync(status_words[i], saved + i, sizeof(int), cudaMemcpyDeviceToDevice, st));
  SMA_CK(cudaStreamSynchronize(st));
  h->mem.release(saved);
  plan = best;
  std::lock_guard<std::mutex> g(tune_mutex());
  tune_cache()[key] = best;
  return SMA_OK;
}

// The slice-SVD parameters of a single t-SVDM problem under plan jp.
template <typename T>
JacobiParams<T> tsvdm_jparams(sma_ctx* h, const Prob<T>& P, const JacobiPlan& jp) {
  const int m = P.m, n = P.n, rc = P.rc;
  JacobiParams<T> J = jacobi_params<T>(h, jp);
  if (P.qr) {
    J.src = qr_jacobi_input(P); J.src_bs = (int64_t)rc * rc; J.m = rc; J.n = rc;
  } else {
    J.src = P.Xh; J.src_bs = (int64_t)m * n; J.m = m; J.n = n;
  }
  J.W = P.Wj; J.W_bs = (int64_t)(jp.mm + jp.rc) * jp.rc;
  J.U = P.U; J.U_bs = (int64_t)jp.mm * rc;
  J.V = P.V; J.V_bs = (int64_t)rc * rc;
  J.sigma = P.sigma; J.sweeps = P.sweeps; J.status = P.status;
  if (jp.rec) {
    J.vlog = P.vlog; J.vlog_bs = P.vlog_bs; J.order = P.vorder; J.vlsweeps = P.vlsw;
    J.vlog_sweeps = jacobi_log_sweeps(J.max_sweeps);
  }
  return J;
}

template <typename T>
sma_status tsvdm_svd(sma_ctx* h, Prob<T>& P) {
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, p = P.p, rc = P.rc;
  if (P.qr) {
    stage_begin(h, SMA_STAGE_PRECOND);
    SMA_K(qr_precondition<T>(P, st));
    stage_end(h);
  }
  auto params = [&](const JacobiPlan& jp) { return tsvdm_jparams<T>(h, P, jp); };
  if (h->opt.autotune && !h->capturing && !P.tuned) {
    SMA_TRY(tune_plan<T>(h, params(P.jp), p, P.qr ? rc : m, P.qr ? rc : n, P.jp, {P.status}));
    P.tuned = true;
  }
  stage_begin(h, SMA_STAGE_SVD);
  SMA_K(jacobi_svd<T>(params(P.jp), p, P.jp.threads, P.jp.smem, st));
  stage_end(h);
  return SMA_OK;
}

// all slices of all t-SVDM problems, one launch per slice size
template <typename T>
sma_status tsvdm_svd_batched(sma_ctx* h) {
  stage_begin(h, SMA_STAGE_PRECOND);
  for (auto& P : probs<T>(h))
    if (P.qr) SMA_K(qr_precondition<T>(P, h->st));
  stage_end(h);
  auto params = [&](const SvdBin<T>& b, const JacobiPlan& jp) {
    JacobiParams<T> J = jacobi_params<T>(h, jp);
    J.desc = b.desc;
    J.m = b.m;
    J.n = b.n;
    J.W = b.W;
    J.W_bs = (int64_t)(jp.mm + jp.rc) * jp.rc;
    return J;
  };
  if (h->opt.autotune && !h->capturing) {
    std::vector<int*> sw;
    for (auto& P : probs<T>(h)) sw.push_back(P.status);
    for (auto& b : bins<T>(h))
      if (!b.tuned) {
        SMA_TRY(tune_plan<T>(h, params(b, b.jp), b.count, b.m, b.n, b.jp, sw));
        b.tuned = true;
      }
  }
  stage_begin(h, SMA_STAGE_SVD);
  for (auto& b : bins<T>(h)) SMA_K(jacobi_svd<T>(params(b, b.jp), b.count, b.jp.threads, b.jp.smem, h->st));
  stage_end(h);
  return SMA_OK;
}

// Truncation of every problem of the handle in one launch (several problems).
template <typename T>
sma_status truncate_all(sma_ctx* h) {
  stage_begin(h, SMA_STAGE_TRUNCATE);
  SMA_K(truncate_ranks_batched(h->tdesc, h->nprob, h->opt.rel_tol, h->opt.fixed_rank, h->st));
  stage_end(h);
  return SMA_OK;
}

template <typename T>
sma_status tsvdm_post(sma_ctx* h, Prob<T>& P, bool truncated) {
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, p = P.p, mm = P.mm, rc = P.rc;
  const int64_t mn = (int64_t)m * n;
  // truncation
  if (!truncated) {
    stage_begin(h, SMA_STAGE_TRUNCATE);
    SMA_K(truncate_ranks(P.sigma, rc, p, P.stats, h->opt.rel_tol, h->opt.fixed_rank, P.ranks,
                         P.off, P.stats + 1, P.iscal, P.suf, st, 0));
    stage_end(h);
  }
  if constexpr (std::is_same<T, float>::value) {
    if (P.jp.rec) {
      // the columns of V the rebuild reads, from the rotation log
      stage_begin(h, SMA_STAGE_SVD);
      SMA_K(jacobi_v_replay(tsvdm_jparams<T>(h, P, P.jp), P.jp, P.ranks, p, st));
      stage_end(h);
    }
  }
  if (P.qr) {
    stage_begin(h, SMA_STAGE_PRECOND);
    const QrParams<T> q2 = qr2_params(P);
    SMA_K(qr_finish<T>(qr_params(P), P.qr2 ? &q2 : nullptr, P.ranks, p, st));
    stage_end(h);
  }
  stage_begin(h, SMA_STAGE_FACTORS);
  // truncated slices: D_i = Xhat_i - W_d V_d^T (W = U Sigma, d = the
  // discarded columns rho_i..rc-1), or Xhat_i - V_d W_d^T when the slice was
  // processed transposed.  Subtracting the discarded part keeps the error of
  // the rebuilt slice proportional to the discarded energy, not to ||Xhat_i||.
  // With the QR preconditioning the slice is (Q1 V)(P W)^T: L = Q1 [V_d; 0]
  // and Rt = P W take the places of W and V; after two QRs it is
  // (Q1 W)(P Q2 V)^T, with L = Q1 [W_d; 0] and Rt = P Q2 V_d.
  const int64_t urc = (int64_t)mm * rc, vrc = (int64_t)rc * rc;
  T* const Lf = P.qr ? P.qL : P.U;
  T* const Rf = P.qr ? P.qRt : P.V;
  SMA_CK(cudaMemcpyAsync(P.D, P.Xh, sizeof(T) * (size_t)mn * p, cudaMemcpyDeviceToDevice, st));
  {
    GemmParams<T> g;
    g.M = m; g.N = n; g.K = rc; g.dKoff = P.ranks;
    if (!P.trans) {
      g.A = Lf; g.a_rs = 1; g.a_cs = mm; g.a_b1 = urc;
      g.B = Rf; g.b_rs = rc; g.b_cs = 1; g.b_b1 = vrc;
    } else {
      g.A = Rf; g.a_rs = 1; g.a_cs = rc; g.a_b1 = vrc;
      g.B = Lf; g.b_rs = mm; g.b_cs = 1; g.b_b1 = urc;
    }
    g.C = P.D; g.c_rs = 1; g.c_cs = m; g.c_b1 = mn;
    g.alpha = T(-1); g.beta = T(1);
    g.nb1 = p;
    SMA_K(contract<T>(h, g));
  }
  stage_end(h);
  // orthogonality of the retained columns of the Jacobi W (the slice's left
  // singular vectors, or with the QR preconditioning its right ones)
  stage_begin(h, SMA_STAGE_REPORT);
  {
    const int jmm = P.jp.mm;
    SMA_K(orth_gram_defect<T>(P.U, jmm, (int64_t)jmm * rc, jmm, rc, p, P.ranks, P.sigma, P.orth,
                              st));
  }
  stage_end(h);
  return SMA_OK;
}

// Gram of an unfolding in fp64 followed by its Jacobi eigen-solve.
// Y (rows x K) given by strides; result: gvec (rows x rows, sorted), gsig
// (eigenvalues), rank written to ranks[slot] by the truncation kernel.
// One unfolding Gram of a Tucker variant: Y (rows x K, element (i, k) at
// Ysrc[i y_rs + k y_cs], summed over nb1 batch entries y_b1 apart; Ysrc =
// the fp64 copy of X unless given) and its share of the tolerance budget.
struct GramSpec {
  int rows, K;
  int64_t y_rs, y_cs;
  int nb1;
  int64_t y_b1;
  double share;
  const double* src;
};

// G_slot = Y Y^T in fp64.
template <typename T>
sma_status gram_form(sma_ctx* h, Prob<T>& P, int slot, const GramSpec& gs) {
  cudaStream_t st = h->st;
  const int rows = gs.rows, K = gs.K, nb1 = gs.nb1;
  const int64_t y_rs = gs.y_rs, y_cs = gs.y_cs, y_b1 = gs.y_b1;
  const double* Ysrc = gs.src ? gs.src : P.X64;
  stage_begin(h, SMA_STAGE_TRANSFORM);
  double* G = P.gram + (size_t)slot * P.gstride;
  {
    // the unfolding Y (rows x Ktot): strided in X64, or laid out contiguously
    // first when it sums over a batch index
    GemmParams<double> g;
    g.M = rows; g.N = rows;
    if (nb1 > 1) {
      SMA_K(permute3(Ysrc, y_rs, y_cs, y_b1, rows, K, nb1, P.Xu, st));
      g.K = K * nb1;
      g.A = P.Xu; g.a_rs = 1; g.a_cs = rows;
      g.B = P.Xu; g.b_rs = rows; g.b_cs = 1;
    } else {
      g.K = K;
      g.A = Ysrc; g.a_rs = y_rs; g.a_cs = y_cs;
      g.B = Ysrc; g.b_rs = y_cs; g.b_cs = y_rs;
    }
    g.C = G; g.c_rs = 1; g.c_cs = rows;
    // G = Y Y^T has few output tiles: split K so that about two CTAs per SM
    // take part, each writing its partial product, then sum the partials in
    // a fixed order (deterministic)
    const int64_t tiles = (int64_t)((rows + 63) / 64) * ((rows + 63) / 64);
    int64_t nsplit = (2 * (int64_t)h->nsm + tiles - 1) / tiles;
    if (nsplit > g.K / 64) nsplit = g.K / 64;
    if (nsplit > 1) {
      const int kc = (int)(((g.K + nsplit - 1) / nsplit + 15) / 16 * 16);
      nsplit = (g.K + kc - 1) / kc;
    }
    if (nsplit > 1 && (size_t)nsplit * rows * rows <= h->gpart_elems) {
      g.kchunk = (int)(((g.K + nsplit - 1) / nsplit + 15) / 16 * 16);
      g.nb1 = (int)nsplit;
      g.C = h->gpart; g.c_b1 = (int64_t)rows * rows;
      SMA_K(gemm<double>(g, st));
      SMA_K(sum_slabs(h->gpart, (int)nsplit, (int64_t)rows * rows, G, st));
    } else {
      SMA_K(gemm<double>(g, st));
    }
  }
  stage_end(h);
  return SMA_OK;
}

// Buffers of a group of Jacobi eigen-solves of symmetric matrices of one
// order: matrix c at src + c stride, its eigenvectors to vec + c stride (the
// Jacobi's W = A V output to wout + c stride, not used), eigenvalues in
// descending order to sig + c sstride, sweep counts to sweeps + c; work is the
// block-mode / cooperative workspace; desc the per-matrix descriptors of a
// one-launch group (or null).
template <typename E>
struct EigBufs {
  const E* src;
  E* vec;
  E* wout;
  double* sig;
  size_t stride, sstride;
  int* sweeps;
  E* work;
  const SliceDesc<E>* desc;
};

// One-sided Jacobi eigen-solves of `count` matrices of order rows in the
// element type E: one cooperative launch each from kCoopMinRows up,
// otherwise one single-CTA launch for the whole group (one CTA per matrix,
// through the descriptors).
template <typename T, typename E>
sma_status eig_jacobi(sma_ctx* h, Prob<T>& P, const EigBufs<E>& b, int count, int rows,
                      int coop_min_rows = kCoopMinRows) {
  cudaStream_t st = h->st;
  JacobiPlan jp = jacobi_plan<E>(rows, rows, h->max_smem);
  JacobiPlan cp{};
  if (rows >= coop_min_rows) cp = jacobi_coop_plan<E>(rows, h->max_smem);
  const bool coop = rows >= coop_min_rows && cp.smem > 0 && h->coop_bar;
  if (coop) jp = cp;
  if (jp.smem == 0) return SMA_ERR_UNSUPPORTED;   // columns too long for shared memory
  JacobiParams<E> J;
  J.m = rows; J.n = rows;
  J.mm = jp.mm; J.rc = jp.rc; J.trans = 0; J.ldS = jp.ldS; J.bcols = jp.bcols; J.g = jp.g;
  J.sort_n = jp.sort_n; J.tile = jp.tile;
  J.max_sweeps = h->opt.max_sweeps > 0 ? h->opt.max_sweeps : 30;
  J.tol = 4.0 * std::sqrt((double)rows) * Eps<E>::v;
  J.status = P.status;
  if (!coop && !jp.block_mode && count > 1 && b.desc) {
    J.desc = b.desc;
    SMA_K(jacobi_svd<E>(J, count, jp.threads, jp.smem, st));
    return SMA_OK;
  }
  // one fp32 matrix of order >= kClusterMinRows: over a cluster of CTAs
  JacobiPlan cl{};
  if constexpr (std::is_same<E, float>::value)
    if (!coop && rows >= kClusterMinRows && h->coop_rot) cl = jacobi_cluster_plan(rows, h->max_smem);
  if (cl.smem > 0) {
    J.ldS = cl.ldS; J.bcols = cl.bcols; J.g = cl.g; J.sort_n = cl.sort_n; J.tile = cl.tile;
  }
  for (int c = 0; c < count; ++c) {
    J.src = b.src + (size_t)c * b.stride; J.src_bs = 0;
    J.W = (jp.block_mode || coop) ? b.work : nullptr; J.W_bs = 0;
    J.U = b.wout + (size_t)c * b.stride; J.U_bs = 0;
    J.V = b.vec + (size_t)c * b.stride; J.V_bs = 0;
    J.sigma = b.sig + (size_t)c * b.sstride;
    J.sweeps = b.sweeps + c;
    if (coop) {
      SMA_K(jacobi_svd_coop<E>(J, cp, CoopSync{h->coop_bar, h->coop_rot, h->coop_abort}, st));
    } else if (cl.smem > 0) {
      if constexpr (std::is_same<E, float>::value) {
        J.W = b.work;
        SMA_K(jacobi_svd_cluster(J, cl, h->coop_rot, st));
      }
    } else {
      SMA_K(jacobi_svd<E>(J, 1, jp.threads, jp.smem, st));
    }
  }
  return SMA_OK;
}

// C_c = op(A_c) op(B_c) for nb pairs of n x n fp64 matrices (ld n, matrix c
// at offset c stride in each of A, B, C; stride 0 shares a matrix), op =
// transpose when ta / tb.  One matrix: K split over the GPU (partials summed
// in a fixed order); several: one batched launch.
template <typename T>
sma_status gemm64_square(sma_ctx* h, int n, const double* A, bool ta, const double* B, bool tb,
                         double* C, int nb = 1, int64_t a_stride = 0, int64_t b_stride = 0,
                         int64_t c_stride = 0) {
  GemmParams<double> g;
  g.M = n; g.N = n; g.K = n;
  g.A = A; g.a_rs = ta ? n : 1; g.a_cs = ta ? 1 : n;
  g.B = B; g.b_rs = tb ? n : 1; g.b_cs = tb ? 1 : n;
  g.C = C; g.c_rs = 1; g.c_cs = n;
  if (nb > 1) {
    g.a_b1 = a_stride; g.b_b1 = b_stride; g.c_b1 = c_stride;
    g.nb1 = nb;
    SMA_K(contract<double>(h, g));
    return SMA_OK;
  }
  // (the split-K form uses the batch index for its K chunks: strides stay 0)
  return contract_split_k<double>(h, g, h->gpart, h->gpart_elems);
}

// The mixed path's Gram eigen-solve.  The Gram G itself is formed in fp64
// (exact products of the fp32 data: the truncation compares tail energies
// with tol^2 ||X||^2, far below fp32 resolution).  Its eigenvectors are
// found by the fp32 Jacobi, then one residual-correction pass in fp64
// restores fp64 accuracy:
//   1. U = the fp32 eigenvectors in fp64; one Newton-Schulz step
//      U <- U (3 I - U^T U) / 2 makes U orthonormal to fp64 accuracy (the
//      fp32 solve leaves |U^T U - I| near 1e-6, the step squares it);
//   2. Rayleigh-Ritz: S = U^T G U in fp64 -- nearly diagonal, except within
//      clusters of eigenvalues that fp32 cannot separate (the small tail
//      the truncation reads);
//   3. the fp64 Jacobi of S (a few sweeps from a nearly diagonal start):
//      S = Z Lambda Z^T; the Ritz values Lambda are G's eigenvalues to fp64
//      accuracy and U Z its eigenvectors.
// Orders from kPcholMinRows to kPcholMaxRows take the preconditioned form
// (gram_pre.cu), one Gram at a time:
//   1. G = L L^T, L = P R^T by the diagonally pivoted Cholesky in fp64 (R is
//      the R factor of the column-pivoted QR of the unfolding's transpose);
//   2. the fp32 Jacobi of L (as fast to converge as a QR-preconditioned
//      slice): L V ~ U Sigma;
//   3. V in fp64, made orthonormal to fp64 accuracy by two Newton-Schulz
//      steps V <- V (3 I - V^T V) / 2;
//   4. the fp64 Jacobi of L V, whose columns are already orthogonal up to the
//      fp32 solve's accuracy, so it takes a few sweeps: L V V2 = U Sigma,
//      and G = U Sigma^2 U^T to fp64 accuracy.
constexpr int kPcholMinRows = 128;

template <typename T>
sma_status gram_solve_pchol(sma_ctx* h, Prob<T>& P, int slot, int rows) {
  cudaStream_t st = h->st;
  const size_t gs = P.gstride;
  const int64_t nn = (int64_t)rows * rows;
  double* L = P.gS + slot * gs;
  SMA_K(gram_pchol(P.gram + slot * gs, rows, P.gT1, L, P.g32 + slot * gs, P.status, st));
  const EigBufs<float> b32{P.g32 + slot * gs, P.gv32 + slot * gs, P.gw32 + slot * gs,
                           P.gsig + (size_t)slot * P.gdim, gs, (size_t)P.gdim, P.sweeps + slot,
                           P.wg32, nullptr};
  SMA_TRY(eig_jacobi<T, float>(h, P, b32, 1, rows, 1 << 30));
  double* V = P.gvec + slot * gs;
  SMA_K(convert<double, float>(P.gv32 + slot * gs, V, nn, st));
  for (int it = 0; it < 2; ++it) {
    SMA_TRY(gemm64_square<T>(h, rows, V, true, V, false, P.gT1));     // V^T V
    SMA_TRY(gemm64_square<T>(h, rows, V, false, P.gT1, false, P.gT2));  // V (V^T V)
    SMA_K(axpby(-0.5, P.gT2, 1.5, V, nn, st));                        // V (3I - V^T V) / 2
  }
  SMA_TRY(gemm64_square<T>(h, rows, L, false, V, false, P.gT1));      // L V
  const EigBufs<double> bX{P.gT1, P.gZ + slot * gs, P.gW + slot * gs,
                           P.gsig + (size_t)slot * P.gdim, gs, (size_t)P.gdim, P.sweepsS + slot,
                           P.Wg, nullptr};
  SMA_TRY(eig_jacobi<T, double>(h, P, bX, 1, rows));
  SMA_K(gram_pchol_finish(P.gW + slot * gs, P.gsig + (size_t)slot * P.gdim, rows, V, st));
  return SMA_OK;
}

template <typename T>
sma_status gram_solve_mixed(sma_ctx* h, Prob<T>& P, int slot, int count, int rows) {
  cudaStream_t st = h->st;
  const size_t gs = P.gstride;
  const int64_t nn = (int64_t)rows * rows;
  if (rows >= kPcholMinRows && rows <= kPcholMaxRows) {
    for (int c = 0; c < count; ++c) SMA_TRY(gram_solve_pchol(h, P, slot + c, rows));
    return SMA_OK;
  }
  for (int c = 0; c < count; ++c)
    SMA_K(convert<float, double>(P.gram + (slot + c) * gs, P.g32 + (slot + c) * gs, nn, st));
  const EigBufs<float> b32{P.g32 + slot * gs, P.gv32 + slot * gs, P.gw32 + slot * gs,
                           P.gsig + (size_t)slot * P.gdim, gs, (size_t)P.gdim, P.sweeps + slot,
                           P.wg32, P.gdesc32 ? P.gdesc32 + slot : nullptr};
  // the single-CTA register-tiled fp32 Jacobi (its rounds synchronise within
  // the CTA; the cooperative form waits on a grid barrier every round, which
  // dominates once the arithmetic is fp32)
  SMA_TRY(eig_jacobi<T, float>(h, P, b32, count, rows, 1 << 30));
  // the residual correction of the group's `count` Grams, batched over them
  // (slots gs apart; the temporaries hold one Gram, so batches of one for
  // the large orders that have the split-K products)
  double* U0 = P.gvec + slot * gs;
  const int nb = count;
  const int64_t bs = (int64_t)gs;
  SMA_K(convert<double, float>(P.gv32 + slot * gs, U0, (int64_t)gs * (count - 1) + nn, st));
  for (int c0 = 0; c0 < count; c0 += (nb > 1 && rows < 64) ? nb : 1) {
    const int cnt = (nb > 1 && rows < 64) ? nb : 1;
    double* U = U0 + c0 * gs;
    const double* Gm = P.gram + (slot + c0) * gs;
    double* Sm = P.gS + (slot + c0) * gs;
    double* T1 = cnt > 1 ? P.gW + (slot + c0) * gs : P.gT1;   // the fp64 Jacobi's W output
    double* T2 = cnt > 1 ? P.gZ + (slot + c0) * gs : P.gT2;   // slots serve as scratch here
    const int64_t ts = cnt > 1 ? bs : 0;
    SMA_TRY(gemm64_square<T>(h, rows, U, true, U, false, T1, cnt, bs, bs, ts));    // U^T U
    SMA_TRY(gemm64_square<T>(h, rows, U, false, T1, false, T2, cnt, bs, ts, ts));  // U (U^T U)
    for (int c = 0; c < cnt; ++c)                                                  // U(3I-U^TU)/2
      SMA_K(axpby(-0.5, T2 + c * ts, 1.5, U + c * gs, nn, st));
    SMA_TRY(gemm64_square<T>(h, rows, Gm, false, U, false, T1, cnt, bs, bs, ts));  // G U
    SMA_TRY(gemm64_square<T>(h, rows, U, true, T1, false, Sm, cnt, bs, ts, bs));   // U^T G U
  }
  const EigBufs<double> bS{P.gS + slot * gs, P.gZ + slot * gs, P.gW + slot * gs,
                           P.gsig + (size_t)slot * P.gdim, gs, (size_t)P.gdim, P.sweepsS + slot,
                           P.Wg, P.gdescS ? P.gdescS + slot : nullptr};
  SMA_TRY(eig_jacobi<T, double>(h, P, bS, count, rows));
  for (int c0 = 0; c0 < count; c0 += (nb > 1 && rows < 64) ? nb : 1) {
    const int cnt = (nb > 1 && rows < 64) ? nb : 1;
    double* T1 = cnt > 1 ? P.gW + (slot + c0) * gs : P.gT1;
    const int64_t ts = cnt > 1 ? bs : 0;
    SMA_TRY(gemm64_square<T>(h, rows, U0 + c0 * gs, false, P.gZ + (slot + c0) * gs, false, T1,
                             cnt, bs, bs, ts));                                      // U Z
    for (int c = 0; c < cnt; ++c)
      SMA_CK(cudaMemcpyAsync(U0 + (c0 + c) * gs, T1 + c * ts, sizeof(double) * (size_t)nn,
                             cudaMemcpyDeviceToDevice, st));
  }
  return SMA_OK;
}

// Largest Gram order for which the mixed path solves in fp32 and corrects in
// fp64: up to it the fp32 solve is the single-CTA register-tiled Jacobi;
// above it only the cooperative Jacobi is left, whose rounds each wait on a
// grid barrier, and in fp32 that form is no faster than the fp64 solve (the
// 898^2 block-index Gram: 462 ms against 408 ms measured), so larger orders
// take the fp64 Jacobi on both paths.
constexpr int kMixedGramMaxRows = 256;

// Eigenpairs of the Grams in slots [slot, slot + count), all of order rows
// (fp64 path: the fp64 Jacobi; mixed path: gram_solve_mixed).
template <typename T>
sma_status gram_solve(sma_ctx* h, Prob<T>& P, int slot, int count, int rows) {
  stage_begin(h, SMA_STAGE_SVD);
  sma_status s;
  if (P.g32 && rows <= kMixedGramMaxRows) {
    s = gram_solve_mixed(h, P, slot, count, rows);
  } else {
    const size_t gs = P.gstride;
    const EigBufs<double> b{P.gram + slot * gs, P.gvec + slot * gs, P.gW + slot * gs,
                            P.gsig + (size_t)slot * P.gdim, gs, (size_t)P.gdim, P.sweeps + slot,
                            P.Wg, P.gdesc ? P.gdesc + slot : nullptr};
    s = eig_jacobi<T, double>(h, P, b, count, rows);
  }
  stage_end(h);
  return s;
}

// Rank of slot's mode: the Gram's eigenvalues are the energies sigma^2 of the
// unfolding; the budget is (rel_tol share)^2 ||X||^2, or fixed_rank.
template <typename T>
sma_status gram_truncate(sma_ctx* h, Prob<T>& P, int slot, int rows, double share) {
  stage_begin(h, SMA_STAGE_TRUNCATE);
  SMA_K(truncate_ranks(P.gsig + (size_t)slot * P.gdim, rows, 1, P.stats, h->opt.rel_tol * share,
                        h->opt.fixed_rank, P.ranks + slot, P.off, P.stats + 2 + slot,
                        P.iscal + 2 + slot, P.suf + (size_t)slot * (P.gdim + 1), h->st, 1));
  stage_end(h);
  return SMA_OK;
}

// Every Gram of a compression: form them all, solve consecutive slots of one
// small order together, then the ranks.
template <typename T>
sma_status gram_all(sma_ctx* h, Prob<T>& P, const GramSpec* gs, int n) {
  for (int i = 0; i < n; ++i) SMA_TRY(gram_form(h, P, i, gs[i]));
  for (int i = 0; i < n;) {
    int j = i + 1;
    if (gs[i].rows < kCoopMinRows)
      while (j < n && gs[j].rows == gs[i].rows) ++j;
    SMA_TRY(gram_solve(h, P, i, j - i, gs[i].rows));
    i = j;
  }
  for (int i = 0; i < n; ++i) SMA_TRY(gram_truncate(h, P, i, gs[i].rows, gs[i].share));
  return SMA_OK;
}

template <typename T>
sma_status gram_factor(sma_ctx* h, Prob<T>& P, int slot, int rows, int K, int64_t y_rs,
                       int64_t y_cs, int nb1, int64_t y_b1, double tol_share,
                       const double* Ysrc = nullptr) {
  const GramSpec gs{rows, K, y_rs, y_cs, nb1, y_b1, tol_share, Ysrc};
  SMA_TRY(gram_form(h, P, slot, gs));
  SMA_TRY(gram_solve(h, P, slot, 1, rows));
  return gram_truncate(h, P, slot, rows, tol_share);
}

// Section 6.3, randomized block-index factor: the sketch Y_k = Omega^T X_k Psi
// (sk x sk per block), the sk^2 x sk^2 Gram H = Y_(3)^T Y_(3) of its
// block-index unfolding (p x sk^2) and its eigenpairs (W, sigma^2), then the
// r = fixed_rank leading left singular vectors of the unfolding as
// V = Y_(3) W_r Sigma_r^-1 (fp64, p x r, ld p) in the second Gram slot of gvec.
template <typename T>
sma_status sketch_factor(sma_ctx* h, Prob<T>& P) {
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, p = P.p, sk = P.sk, s2 = sk * sk;
  stage_begin(h, SMA_STAGE_TRANSFORM);
  {
    // Ytmp_k = Omega^T X_k  (sk x n)
    GemmParams<T> g;
    g.M = sk; g.N = n; g.K = m;
    g.A = P.Om; g.a_rs = m; g.a_cs = 1;
    g.B = P.X; g.b_rs = 1; g.b_cs = m; g.b_b1 = (int64_t)m * n;
    g.C = P.Ytmp; g.c_rs = 1; g.c_cs = sk; g.c_b1 = (int64_t)sk * n;
    g.nb1 = p;
    SMA_K(contract<T>(h, g));
    // Y_k = Ytmp_k Psi  (sk x sk)
    GemmParams<T> g2;
    g2.M = sk; g2.N = sk; g2.K = n;
    g2.A = P.Ytmp; g2.a_rs = 1; g2.a_cs = sk; g2.a_b1 = (int64_t)sk * n;
    g2.B = P.Ps; g2.b_rs = 1; g2.b_cs = n;
    g2.C = P.Ysk; g2.c_rs = 1; g2.c_cs = sk; g2.c_b1 = s2;
    g2.nb1 = p;
    SMA_K(contract<T>(h, g2));
    SMA_K(convert<double, T>(P.Ysk, P.Y64, (int64_t)s2 * p, st));
  }
  stage_end(h);
  // H = Y_(3)^T Y_(3): rows e (stride 1), K = p (stride sk^2); its eigenpairs
  // and the rank (fixed_rank, at most sk^2)
  SMA_TRY(gram_factor(h, P, 0, s2, p, 1, s2, 1, 0, 1.0, P.Y64));
  stage_begin(h, SMA_STAGE_FACTORS);
  double* V = P.gvec + P.gstride;
  SMA_CK(cudaMemsetAsync(V, 0, sizeof(double) * (size_t)p * p, st));
  {
    // V(k, j) = sum_e Y_(3)(k, e) W(e, j), j < r
    GemmParams<double> g;
    g.M = p; g.N = s2; g.K = s2; g.dN = P.iscal + 2; g.dstride = 0;
    g.A = P.Y64; g.a_rs = s2; g.a_cs = 1;
    g.B = P.gvec; g.b_rs = 1; g.b_cs = s2;
    g.C = V; g.c_rs = 1; g.c_cs = p;
    SMA_K(gemm<double>(g, st));
  }
  SMA_K(scale_cols_rsqrt(V, p, p, P.gsig, P.iscal + 2, st));
  stage_end(h);
  return SMA_OK;
}

template <typename T>
sma_status compress_tucker(sma_ctx* h, Prob<T>& P) {
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, p = P.p;
  const int64_t mn = (int64_t)m * n;
  const sma_decomp d = h->opt.decomp;
  if (P.X64) SMA_K(convert<double, T>(P.X, P.X64, mn * p, st));
  if (d == SMA_TUCKER_BLOCKMODE) {
    if (P.sk > 0) {
      SMA_TRY(sketch_factor(h, P));
      stage_begin(h, SMA_STAGE_FACTORS);
      SMA_K(convert<T, double>(P.gvec + P.gstride, P.F1, (int64_t)p * p, st));
    } else {
      // block-index unfolding: rows k, K = mn; Y(k, e) = X[e + mn k]
      SMA_TRY(gram_factor(h, P, 0, p, (int)mn, mn, 1, 1, 0, 1.0));
      stage_begin(h, SMA_STAGE_FACTORS);
      SMA_K(convert<T, double>(P.gvec, P.F1, (int64_t)p * p, st));  // V = leading columns
    }
    // G = X x3 V^T: G_mat (mn x r) = X_mat (mn x p) V (p x r)
    GemmParams<T> g;
    g.M = (int)mn; g.N = p; g.K = p; g.dN = P.iscal + 2; g.dstride = 0;
    g.A = P.X; g.a_rs = 1; g.a_cs = mn;
    g.B = P.F1; g.b_rs = 1; g.b_cs = p;
    g.C = P.D; g.c_rs = 1; g.c_cs = mn;
    SMA_K(contract<T>(h, g));
    // C_j = struct_E(V[:, j])
    SMA_K(build_struct_terms_nz<T>(P.d_nzpos, P.d_nzk, P.nnz, P.d_isq, P.ell, P.q, P.F1, p, 1, p,
                                    P.iscal + 2, P.C, st));
    // error ||X - T||_F measured directly (Lemma 1: equal to ||A - A_hat||_F)
    SMA_TRY(make_T(h, P));
    SMA_K(residual_norm2<T>(P.X, P.Tt, mn * p, P.partial, P.nparts, P.stats + 1, st));
    stage_end(h);
    // orthogonality of V_r
    stage_begin(h, SMA_STAGE_REPORT);
    GemmParams<T> go;
    go.M = p; go.N = p; go.K = p; go.dM = P.iscal + 2; go.dN = P.iscal + 2; go.dstride = 0;
    go.A = P.F1; go.a_rs = p; go.a_cs = 1;
    go.B = P.F1; go.b_rs = 1; go.b_cs = p;
    go.C = P.Gorth; go.c_rs = 1; go.c_cs = p;
    SMA_K(gemm<T>(go, st));
    SMA_K(orth_defect<T>(P.Gorth, p, 1, P.iscal + 2, nullptr, P.orth, st));
    stage_end(h);
    return SMA_OK;
  }
  // mode-1 unfolding [X_1 ... X_p] (m x np): Gram = sum_k X_k X_k^T;
  // ROWCOL also the mode-2 unfolding [X_1^T ... X_p^T] (n x mp)
  const int ntr = 2;  // two truncated modes share the budget
  const double share = 1.0 / std::sqrt((double)ntr);
  const GramSpec gs[2] = {{m, (int)(mn * p / m), 1, m, 1, 0, share, nullptr},
                          {n, m, m, 1, p, mn, share, nullptr}};
  SMA_TRY(gram_all(h, P, gs, d == SMA_TUCKER_ROWCOL ? 2 : 1));
  SMA_K(convert<T, double>(P.gvec, P.F1, (int64_t)m * m, st));
  const int* r1 = P.iscal + 2;
  const int* r3 = r1;
  const T* Wf = P.F1;
  int ldw = m;
  if (d == SMA_TUCKER_ROWCOL) {
    SMA_K(convert<T, double>(P.gvec + P.gstride, P.F2, (int64_t)n * n, st));
    r3 = P.iscal + 3;
    Wf = P.F2;
    ldw = n;
  }
  const int r1max = P.r1max, r3max = P.r3max;
  stage_begin(h, SMA_STAGE_FACTORS);
  SMA_CK(cudaMemsetAsync(P.core, 0, sizeof(T) * (size_t)r1max * r3max * p, st));
  // tmp_k = U^T X_k (r1 x n)
  GemmParams<T> g;
  g.M = m; g.N = n; g.K = m; g.dM = r1; g.dstride = 0;
  g.A = P.F1; g.a_rs = m; g.a_cs = 1;
  g.B = P.X; g.b_rs = 1; g.b_cs = m; g.b_b1 = mn;
  g.C = P.tmp; g.c_rs = 1; g.c_cs = m; g.c_b1 = (int64_t)m * n;
  g.nb1 = p;
  SMA_K(contract<T>(h, g));
  // core_k = tmp_k W (r1 x r3), stored r1max x r3max per k
  GemmParams<T> g2;
  g2.M = m; g2.N = ldw; g2.K = n; g2.dM = r1; g2.dN = r3; g2.dstride = 0;
  g2.A = P.tmp; g2.a_rs = 1; g2.a_cs = m; g2.a_b1 = (int64_t)m * n;
  g2.B = Wf; g2.b_rs = 1; g2.b_cs = ldw;
  g2.C = P.core; g2.c_rs = 1; g2.c_cs = r1max; g2.c_b1 = (int64_t)r1max * r3max;
  g2.nb1 = p;
  SMA_K(contract<T>(h, g2));
  // middle factor struct_E(core_k), dense (ell r1max) x (q r3max)
  SMA_K(scatter_ME<T>(P.d_map, P.d_isq, P.ell, P.q, r1max, r3max, P.core, P.mid,
                       (int64_t)P.ell * r1max, st));
  // error ||X - T||_F measured directly
  SMA_TRY(make_T(h, P));
  SMA_K(residual_norm2<T>(P.X, P.Tt, mn * p, P.partial, P.nparts, P.stats + 1, st));
  stage_end(h);
  // orthogonality of U (and W)
  stage_begin(h, SMA_STAGE_REPORT);
  for (int f = 0; f < P.n_orth; ++f) {
    const T* F = f == 0 ? P.F1 : P.F2;
    const int rows = f == 0 ? m : n;
    GemmParams<T> go;
    go.M = rows; go.N = rows; go.K = rows; go.dM = P.iscal + 2 + f; go.dN = P.iscal + 2 + f;
    go.dstride = 0;
    go.A = F; go.a_rs = rows; go.a_cs = 1;
    go.B = F; go.b_rs = 1; go.b_cs = rows;
    go.C = P.Gorth; go.c_rs = 1; go.c_cs = rows;
    SMA_K(gemm<T>(go, st));
    SMA_K(orth_defect<T>(P.Gorth, rows, 1, P.iscal + 2 + f, nullptr, P.orth + f, st));
  }
  stage_end(h);
  return SMA_OK;
}

// Section 7 with two levels and m x n blocks: truncated HOSVD of the fourth-
// order tensor X[a, b, i1, i2] (stored as the one-level tensor of the
// product map, block index i1 + p1 i2), each of the four modes with the
// budget tol^2 ||X||^2 / 4; core G = X x Xf^T x Zf^T x Y1^T x Y2^T; the
// Kronecker sum over (j1, j2) of struct1(Y1[:, j1]) (x) struct2(Y2[:, j2])
// (x) Xf G[:, :, j1, j2] Zf^T kept as one-level terms: coefficient vectors
// Y1[i1, j1] Y2[i2, j2] over the product map and D_t = Xf G_t Zf^T.
template <typename T>
sma_status compress_ml2(sma_ctx* h, Prob<T>& P) {
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, p = P.p, p1 = P.lp[0], p2 = P.lp[1];
  const int64_t mn = (int64_t)m * n;
  SMA_K(convert<double, T>(P.X, P.X64, mn * p, st));
  const double share = 0.5;   // four truncated modes: tol^2 ||X||^2 / 4 each
  const GramSpec gs[4] = {
      {m, (int)(n * (int64_t)p), 1, m, 1, 0, share, nullptr},        // a
      {n, m, m, 1, p, mn, share, nullptr},                           // b
      {p1, (int)mn, mn, 1, p2, mn * p1, share, nullptr},             // i1
      {p2, (int)(mn * p1), mn * p1, 1, 1, 0, share, nullptr}};       // i2
  SMA_TRY(gram_all(h, P, gs, 4));
  stage_begin(h, SMA_STAGE_FACTORS);
  const int dims[4] = {m, n, p1, p2};
  for (int t = 0; t < 4; ++t)
    SMA_K(convert<T, double>(P.gvec + P.gstride * t, P.mlF[t], (int64_t)dims[t] * dims[t], st));
  const T* Xf = P.mlF[0];
  const T* Zf = P.mlF[1];
  const int* kx = P.iscal + 2;
  const int* kz = P.iscal + 3;
  const int* k1 = P.iscal + 4;
  const int* k2 = P.iscal + 5;
  SMA_CK(cudaMemsetAsync(P.mlT1, 0, sizeof(T) * (size_t)mn * p, st));
  SMA_CK(cudaMemsetAsync(P.mlT2, 0, sizeof(T) * (size_t)mn * p, st));
  SMA_CK(cudaMemsetAsync(P.mlG, 0, sizeof(T) * (size_t)mn * p, st));
  {  // T1_k = Xf^T X_k (rows < kx)
    GemmParams<T> g;
    g.M = m; g.N = n; g.K = m; g.dM = kx; g.dstride = 0;
    g.A = Xf; g.a_rs = m; g.a_cs = 1;
    g.B = P.X; g.b_rs = 1; g.b_cs = m; g.b_b1 = mn;
    g.C = P.mlT1; g.c_rs = 1; g.c_cs = m; g.c_b1 = mn;
    g.nb1 = p;
    SMA_K(contract<T>(h, g));
  }
  {  // T2_k = T1_k Zf (kx x kz in m x n storage)
    GemmParams<T> g;
    g.M = m; g.N = n; g.K = n; g.dM = kx; g.dN = kz; g.dstride = 0;
    g.A = P.mlT1; g.a_rs = 1; g.a_cs = m; g.a_b1 = mn;
    g.B = Zf; g.b_rs = 1; g.b_cs = n;
    g.C = P.mlT2; g.c_rs = 1; g.c_cs = m; g.c_b1 = mn;
    g.nb1 = p;
    SMA_K(contract<T>(h, g));
  }
  SMA_CK(cudaMemsetAsync(P.mlT1, 0, sizeof(T) * (size_t)mn * p, st));
  {  // T3[e, j1, i2] = sum_i1 T2[e, i1, i2] Y1[i1, j1]  (j1 < k1)
    GemmParams<T> g;
    g.M = (int)mn; g.N = p1; g.K = p1; g.dN = k1; g.dstride = 0;
    g.A = P.mlT2; g.a_rs = 1; g.a_cs = mn; g.a_b1 = mn * p1;
    g.B = P.mlF[2]; g.b_rs = 1; g.b_cs = p1;
    g.C = P.mlT1; g.c_rs = 1; g.c_cs = mn; g.c_b1 = mn * p1;
    g.nb1 = p2;
    SMA_K(contract<T>(h, g));
  }
  {  // G[e, j1, j2] = sum_i2 T3[e, j1, i2] Y2[i2, j2]  (j2 < k2)
    GemmParams<T> g;
    g.M = (int)(mn * p1); g.N = p2; g.K = p2; g.dN = k2; g.dstride = 0;
    g.A = P.mlT1; g.a_rs = 1; g.a_cs = mn * p1;
    g.B = P.mlF[3]; g.b_rs = 1; g.b_cs = p2;
    g.C = P.mlG; g.c_rs = 1; g.c_cs = mn * p1;
    SMA_K(contract<T>(h, g));
  }
  // terms t = j1 + k1 j2 < k1 k2: core slices and coefficient vectors; the
  // rest zero; the term count in iscal[1]
  SMA_K(ml2_terms<T>(P.mlG, (int)mn, p1, p2, P.mlF[2], P.mlF[3], k1, k2, P.mlGt, P.F1, P.iscal + 1,
                     st));
  {  // D_t = Xf Gt_t Zf^T: Xf Gt_t (K = kx), then (.) Zf^T (K = kz)
    GemmParams<T> g;
    g.M = m; g.N = n; g.K = m; g.dK = kx; g.dstride = 0;
    g.A = Xf; g.a_rs = 1; g.a_cs = m;
    g.B = P.mlGt; g.b_rs = 1; g.b_cs = m; g.b_b1 = mn;
    g.C = P.mlT2; g.c_rs = 1; g.c_cs = m; g.c_b1 = mn;
    g.nb1 = p;
    SMA_K(contract<T>(h, g));
    GemmParams<T> g2;
    g2.M = m; g2.N = n; g2.K = n; g2.dK = kz; g2.dstride = 0;
    g2.A = P.mlT2; g2.a_rs = 1; g2.a_cs = m; g2.a_b1 = mn;
    g2.B = Zf; g2.b_rs = n; g2.b_cs = 1;
    g2.C = P.D; g2.c_rs = 1; g2.c_cs = m; g2.c_b1 = mn;
    g2.nb1 = p;
    SMA_K(contract<T>(h, g2));
  }
  SMA_K(build_struct_terms_nz<T>(P.d_nzpos, P.d_nzk, P.nnz, P.d_isq, P.ell, P.q, P.F1, p, 1, p,
                                  P.iscal + 1, P.C, st));
  SMA_TRY(make_T(h, P));
  SMA_K(residual_norm2<T>(P.X, P.Tt, mn * p, P.partial, P.nparts, P.stats + 1, st));
  stage_end(h);
  stage_begin(h, SMA_STAGE_REPORT);
  for (int t = 0; t < 4; ++t) {
    const int rows = dims[t];
    GemmParams<T> go;
    go.M = rows; go.N = rows; go.K = rows; go.dM = P.iscal + 2 + t; go.dN = P.iscal + 2 + t;
    go.dstride = 0;
    go.A = P.mlF[t]; go.a_rs = rows; go.a_cs = 1;
    go.B = P.mlF[t]; go.b_rs = 1; go.b_cs = rows;
    go.C = P.Gorth; go.c_rs = 1; go.c_cs = rows;
    SMA_K(gemm<T>(go, st));
    SMA_K(orth_defect<T>(P.Gorth, rows, 1, P.iscal + 2 + t, nullptr, P.orth + t, st));
  }
  stage_end(h);
  return SMA_OK;
}

// Section 7: HOSVD of the weighted coefficient tensor of a three-level
// structured matrix (m = n = 1), each mode with the budget tol^2 ||X||^2 / 3.
template <typename T>
sma_status compress_multilevel(sma_ctx* h, Prob<T>& P, const void* Ain) {
  cudaStream_t st = h->st;
  const int p1 = P.lp[0], p2 = P.lp[1], p3 = P.lp[2];
  const int64_t np = P.p;
  if (!Ain) return SMA_ERR_ARG;
  const T* a = static_cast<const T*>(Ain);
  stage_begin(h, SMA_STAGE_GATHER);
  if (!is_device_ptr(Ain)) {
    if (!P.stage) SMA_TRY(h->mem.alloc(&P.stage, (size_t)np));
    SMA_CK(cudaMemcpyAsync(P.stage, a, np * sizeof(T), cudaMemcpyHostToDevice, st));
    a = P.stage;
  }
  SMA_K(ml_gather<T>(a, P.d_lw[0], P.d_lw[1], P.d_lw[2], p1, p2, p3, P.X, P.partial, P.nparts, st));
  SMA_K(finish_norm(P.partial, P.nparts, P.stats, st));
  SMA_K(convert<double, T>(P.X, P.X64, np, st));
  stage_end(h);
  const double share = 1.0 / std::sqrt(3.0);
  const GramSpec gs[3] = {{p1, p2 * p3, 1, p1, 1, 0, share, nullptr},                   // mode 1
                          {p2, p1, p1, 1, p3, (int64_t)p1 * p2, share, nullptr},       // mode 2
                          {p3, p1 * p2, (int64_t)p1 * p2, 1, 1, 0, share, nullptr}};   // mode 3
  SMA_TRY(gram_all(h, P, gs, 3));
  stage_begin(h, SMA_STAGE_FACTORS);
  for (int t = 0; t < 3; ++t)
    SMA_K(convert<T, double>(P.gvec + P.gstride * t, P.Uml[t], (int64_t)P.lp[t] * P.lp[t], st));
  const int* k1 = P.iscal + 2;
  const int* k2 = P.iscal + 3;
  const int* k3 = P.iscal + 4;
  SMA_CK(cudaMemsetAsync(P.T1, 0, np * sizeof(T), st));
  SMA_CK(cudaMemsetAsync(P.T2, 0, np * sizeof(T), st));
  SMA_CK(cudaMemsetAsync(P.Gc, 0, np * sizeof(T), st));
  {  // T1 = U1^T X_(1)  (p1 x p2 p3, leading k1 rows)
    GemmParams<T> g;
    g.M = p1; g.N = p2 * p3; g.K = p1; g.dM = k1; g.dstride = 0;
    g.A = P.Uml[0]; g.a_rs = p1; g.a_cs = 1;
    g.B = P.X; g.b_rs = 1; g.b_cs = p1;
    g.C = P.T1; g.c_rs = 1; g.c_cs = p1;
    SMA_K(contract<T>(h, g));
  }
  {  // T2[:, :, i3] = T1[:, :, i3] U2
    GemmParams<T> g;
    g.M = p1; g.N = p2; g.K = p2; g.dM = k1; g.dN = k2; g.dstride = 0;
    g.A = P.T1; g.a_rs = 1; g.a_cs = p1; g.a_b1 = (int64_t)p1 * p2;
    g.B = P.Uml[1]; g.b_rs = 1; g.b_cs = p2;
    g.C = P.T2; g.c_rs = 1; g.c_cs = p1; g.c_b1 = (int64_t)p1 * p2;
    g.nb1 = p3;
    SMA_K(contract<T>(h, g));
  }
  {  // G = T2_(3)^T ... as (p1 p2) x p3 times U3
    GemmParams<T> g;
    g.M = p1 * p2; g.N = p3; g.K = p3; g.dN = k3; g.dstride = 0;
    g.A = P.T2; g.a_rs = 1; g.a_cs = (int64_t)p1 * p2;
    g.B = P.Uml[2]; g.b_rs = 1; g.b_cs = p3;
    g.C = P.Gc; g.c_rs = 1; g.c_cs = (int64_t)p1 * p2;
    SMA_K(contract<T>(h, g));
  }
  SMA_TRY(make_T(h, P));
  SMA_K(residual_norm2<T>(P.X, P.Tt, np, P.partial, P.nparts, P.stats + 1, st));
  stage_end(h);
  stage_begin(h, SMA_STAGE_REPORT);
  for (int t = 0; t < 3; ++t) {
    const int rows = P.lp[t];
    GemmParams<T> go;
    go.M = rows; go.N = rows; go.K = rows; go.dM = P.iscal + 2 + t; go.dN = P.iscal + 2 + t;
    go.dstride = 0;
    go.A = P.Uml[t]; go.a_rs = rows; go.a_cs = 1;
    go.B = P.Uml[t]; go.b_rs = 1; go.b_cs = rows;
    go.C = P.Gorth; go.c_rs = 1; go.c_cs = rows;
    SMA_K(gemm<T>(go, st));
    SMA_K(orth_defect<T>(P.Gorth, rows, 1, P.iscal + 2 + t, nullptr, P.orth + t, st));
  }
  stage_end(h);
  return SMA_OK;
}

// Section 5.2: T_0 = L L^T and L^-1 on the device, then the gathered tensor
// (X_k = sqrt(eta_k) T_k) becomes X_k = sqrt(eta_k) L^-1 T_k L^-T by two
// batched products, and ||X||_F is taken again.
template <typename T>
sma_status spd_congruence(sma_ctx* h, Prob<T>& P) {
  cudaStream_t st = h->st;
  const int m = P.m, p = P.p;
  const int64_t mm = (int64_t)m * m;
  stage_begin(h, SMA_STAGE_TRANSFORM);
  SMA_K(chol_inv<T>(P.T0, m, m, P.Lc, P.Linv, P.status, st));
  // tmp_k = L^-1 X_k
  GemmParams<T> g;
  g.M = m; g.N = m; g.K = m;
  g.A = P.Linv; g.a_rs = 1; g.a_cs = m;
  g.B = P.X; g.b_rs = 1; g.b_cs = m; g.b_b1 = mm;
  g.C = P.tmp; g.c_rs = 1; g.c_cs = m; g.c_b1 = mm;
  g.nb1 = p;
  SMA_K(contract<T>(h, g));
  // X_k = tmp_k L^-T
  GemmParams<T> g2;
  g2.M = m; g2.N = m; g2.K = m;
  g2.A = P.tmp; g2.a_rs = 1; g2.a_cs = m; g2.a_b1 = mm;
  g2.B = P.Linv; g2.b_rs = m; g2.b_cs = 1;
  g2.C = P.X; g2.c_rs = 1; g2.c_cs = m; g2.c_b1 = mm;
  g2.nb1 = p;
  SMA_K(contract<T>(h, g2));
  SMA_K(residual_norm2<T>(P.X, nullptr, mm * p, P.partial, P.nparts, P.stats, st));
  stage_end(h);
  return SMA_OK;
}

// C = A B for a product with few output tiles and a long K (the CP
// contractions: r columns, K = m n or n p): K split so that about two CTAs
// per SM take part, one partial product per chunk into `part`, then the
// partials summed in chunk order into C (which must be dense, ld M).
template <typename T>
sma_status contract_split_k(sma_ctx* h, GemmParams<T> g, T* part, size_t part_elems) {
  const int64_t tiles = (int64_t)((g.M + 63) / 64) * ((g.N + 63) / 64);
  int64_t nsplit = (2 * (int64_t)h->nsm + tiles - 1) / tiles;
  if (nsplit > g.K / 64) nsplit = g.K / 64;
  const bool dense_c = g.c_rs == 1 && g.c_cs == g.M;
  if (nsplit <= 1 || g.nb1 != 1 || g.nb2 != 1 || !dense_c || g.beta != T(0) || g.dK || g.dKoff ||
      (size_t)nsplit * g.M * g.N > part_elems) {
    SMA_K(contract<T>(h, g));
    return SMA_OK;
  }
  const int kc = (int)(((g.K + nsplit - 1) / nsplit + 15) / 16 * 16);
  nsplit = (g.K + kc - 1) / kc;
  T* C = g.C;
  g.kchunk = kc;
  g.nb1 = (int)nsplit;
  g.C = part; g.c_b1 = (int64_t)g.M * g.N;
  SMA_K(gemm<T>(g, h->st));
  SMA_K(sum_slabs_t<T>(part, (int)nsplit, (int64_t)g.M * g.N, C, h->st));
  return SMA_OK;
}

// CP by alternating least squares from the given Xf, Zf: per iteration Yf,
// then Xf, then Zf, each the least-squares solution with the other two fixed
// (the contraction of X with the Khatri-Rao product of the other two factors,
// solved against the Hadamard product of their Gram matrices); then the
// Kronecker terms of Corollary kronsumcp, D_j = Xf[:, j] Zf[:, j]^T and
// C_j = struct_E(Yf[:, j]), and the error measured on the tensor.
template <typename T>
sma_status compress_cp(sma_ctx* h, Prob<T>& P) {
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, p = P.p, r = P.cp_r;
  const int64_t mn = (int64_t)m * n;
  T* Yf = P.F1;   // p x r, ld p
  stage_begin(h, SMA_STAGE_SVD);
  SMA_CK(cudaMemcpyAsync(P.cXf, P.cXf0, sizeof(T) * (size_t)m * r, cudaMemcpyDeviceToDevice, st));
  SMA_CK(cudaMemcpyAsync(P.cZf, P.cZf0, sizeof(T) * (size_t)n * r, cudaMemcpyDeviceToDevice, st));
  for (int it = 0; it < h->opt.cp_iters; ++it) {
    // Yf: M3 = X_(3) (Xf . Zf)  (p x r), X_(3)(k, a + m b) = X[a + m b + mn k]
    SMA_K(khatri_rao<T>(P.cXf, m, P.cZf, n, r, P.cKR, st));
    {
      GemmParams<T> g;
      g.M = p; g.N = r; g.K = (int)mn;
      g.A = P.X; g.a_rs = mn; g.a_cs = 1;
      g.B = P.cKR; g.b_rs = 1; g.b_cs = mn;
      g.C = P.cM; g.c_rs = 1; g.c_cs = p;
      SMA_TRY(contract_split_k<T>(h, g, P.cSlab, P.cSlab_elems));
    }
    SMA_K(cp_solve<T>(P.cXf, m, P.cZf, n, r, P.cM, p, Yf, p, P.status, st));
    // Xf: M1 = X_(1) (Zf . Yf)  (m x r), X_(1) = [X_1 ... X_p] (m x n p)
    SMA_K(khatri_rao<T>(P.cZf, n, Yf, p, r, P.cKR, st));
    {
      GemmParams<T> g;
      g.M = m; g.N = r; g.K = (int)((int64_t)n * p);
      g.A = P.X; g.a_rs = 1; g.a_cs = m;
      g.B = P.cKR; g.b_rs = 1; g.b_cs = (int64_t)n * p;
      g.C = P.cM; g.c_rs = 1; g.c_cs = m;
      SMA_TRY(contract_split_k<T>(h, g, P.cSlab, P.cSlab_elems));
    }
    SMA_K(cp_solve<T>(P.cZf, n, Yf, p, r, P.cM, m, P.cXf, m, P.status, st));
    // Zf: M2 = sum_k X_k^T Xf diag(Yf[k, :])  (n x r), one partial per block
    SMA_K(khatri_rao<T>(P.cXf, m, Yf, p, r, P.cKR, st));
    {
      GemmParams<T> g;
      g.M = n; g.N = r; g.K = m;
      g.A = P.X; g.a_rs = m; g.a_cs = 1; g.a_b1 = mn;
      g.B = P.cKR; g.b_rs = 1; g.b_cs = (int64_t)m * p; g.b_b1 = m;
      g.C = P.cSlab; g.c_rs = 1; g.c_cs = n; g.c_b1 = (int64_t)n * r;
      g.nb1 = p;
      SMA_K(contract<T>(h, g));
    }
    SMA_K(sum_slabs_t<T>(P.cSlab, p, (int64_t)n * r, P.cM, st));
    SMA_K(cp_solve<T>(P.cXf, m, Yf, p, r, P.cM, n, P.cZf, n, P.status, st));
  }
  stage_end(h);
  stage_begin(h, SMA_STAGE_FACTORS);
  SMA_K(khatri_rao<T>(P.cXf, m, P.cZf, n, r, P.D, st));   // D[(a + m b), j] = Xf[a, j] Zf[b, j]
  SMA_K(set_int(P.iscal + 2, r, st));
  SMA_K(build_struct_terms_nz<T>(P.d_nzpos, P.d_nzk, P.nnz, P.d_isq, P.ell, P.q, P.F1, p, 1, p,
                                  P.iscal + 2, P.C, st));
  SMA_TRY(make_T(h, P));
  SMA_K(residual_norm2<T>(P.X, P.Tt, mn * p, P.partial, P.nparts, P.stats + 1, st));
  stage_end(h);
  return SMA_OK;
}

template <typename T>
sma_status compress_one(sma_ctx* h, Prob<T>& P, const void* A, int64_t lda,
                        bool gathered = false) {
  if (P.L == 3) {
    SMA_TRY(compress_multilevel(h, P, A));
    P.compressed = true;
    P.ml_valid = false;
    P.ml_cvalid = false;
    P.h_iscal[0] = -1;
    return SMA_OK;
  }
  if (!gathered) SMA_TRY(do_gather(h, P, A, lda));
  if (P.spd) SMA_TRY(spd_congruence(h, P));
  if (h->opt.decomp == SMA_TSVDM) SMA_TRY(tsvdm_pre(h, P));
  else if (P.ml2) SMA_TRY(compress_ml2(h, P));
  else if (h->opt.decomp == SMA_CP_ALS) SMA_TRY(compress_cp(h, P));
  else SMA_TRY(compress_tucker(h, P));
  P.compressed = true;
  P.dp_valid = false;
  for (auto& o : P.tca) o.valid = false;
  P.cq_valid = false;
  P.h_iscal[0] = -1;
  return SMA_OK;
}

// Entries the compressed form stores over the entries of the p distinct
// blocks (m n p; Section 6.2 quotes this ratio for the shared-U form,
// (r^2 T + N r) / (N^2 T) with N = m and the T distinct lags).
template <typename T>
double storage_ratio(const sma_ctx* h, const Prob<T>& P, const sma_result& r) {
  const double m = P.m, n = P.n, p = P.p;
  const sma_decomp d = h->opt.decomp;
  double stored = 0.0, dense = m * n * p;
  if (P.L == 3) {
    const double p1 = P.lp[0], p2 = P.lp[1], p3 = P.lp[2];
    stored = p1 * r.ranks[0] + p2 * r.ranks[1] + p3 * r.ranks[2] +
             (double)r.ranks[0] * r.ranks[1] * r.ranks[2];
    dense = p1 * p2 * p3;
  } else if (P.ml2) {
    stored = m * r.ranks[0] + n * r.ranks[1] + (double)P.lp[0] * r.ranks[2] +
             (double)P.lp[1] * r.ranks[3] + (double)r.ranks[0] * r.ranks[1] * r.ranks[2] * r.ranks[3];
  } else if (d == SMA_TSVDM) {
    stored = (double)r.total_rank * (m + n + 1.0);           // U_i, V_i, sigma_i
  } else if (d == SMA_TUCKER_BLOCKMODE) {
    stored = (p + m * n) * r.ranks[0];                       // V and the core slices
  } else if (d == SMA_CP_ALS) {
    stored = (m + n + p) * r.ranks[0];                       // the three factors
  } else {
    // shared U (and the SPD form, which also keeps its Cholesky factor and
    // the diagonal block it replaces) or U and W of the rows-and-columns form
    const double r1 = r.ranks[0], r3 = r.ranks[1];
    stored = m * r1 + (d == SMA_TUCKER_ROWCOL ? n * r3 : 0.0) + r1 * r3 * p;
    if (P.spd) {
      stored += m * (m + 1.0) / 2.0;
      dense = m * n * (p + 1.0);
    }
  }
  return dense > 0 ? stored / dense : 0.0;
}

// Section 6.2's trace error |tr A - tr A_hat| / |tr A| from the traces of
// the slices of X and of the approximation (tr A = sum_k tr(E_k) tr(X_k)),
// computed on the device.  0 when the matrix is not a square grid of square
// blocks, for the three-level form, and for the SPD-preserving form (whose
// T_hat keeps the diagonal blocks, and so the trace, exactly).
template <typename T>
sma_status trace_error(sma_ctx* h, Prob<T>& P, double* out) {
  *out = 0.0;
  if (!P.traces || P.L == 3 || P.trw.empty()) return SMA_OK;
  const int m = P.m, n = P.n, p = P.p;
  // the t-SVDM's approximation is T = D x3 M^T: tr T_k = sum_i M[i, k] tr D_i
  const bool ts = h->opt.decomp == SMA_TSVDM;
  const T* approx = ts ? P.D : P.Tt;
  if (!approx) return SMA_OK;
  SMA_K(slice_traces<T>(P.X, m, n, p, P.traces, h->st));
  SMA_K(slice_traces<T>(approx, m, n, p, P.traces + p, h->st));
  std::vector<double> tr(2 * (size_t)p);
  SMA_CK(cudaMemcpyAsync(tr.data(), P.traces, tr.size() * sizeof(double), cudaMemcpyDeviceToHost,
                         h->st));
  SMA_CK(cudaStreamSynchronize(h->st));
  double trA = 0.0, trH = 0.0;
  for (int k = 0; k < p; ++k) {
    if (P.trw[k] == 0.0) continue;
    double tk = tr[(size_t)p + k];
    if (ts) {
      tk = 0.0;
      for (int i = 0; i < p; ++i) tk += P.Mh[(size_t)i + (size_t)k * p] * tr[(size_t)p + i];
    }
    trA += P.trw[k] * tr[k];
    trH += P.trw[k] * tk;
  }
  *out = trA != 0.0 ? std::fabs(trA - trH) / std::fabs(trA) : 0.0;
  return SMA_OK;
}

template <typename T>
sma_status read_result(sma_ctx* h, Prob<T>& P, sma_result* r) {
  SMA_CK(cudaStreamSynchronize(h->st));
  double stats[8];
  int iscal[8];
  int status = 0;
  SMA_CK(cudaMemcpy(stats, P.stats, sizeof(stats), cudaMemcpyDeviceToHost));
  SMA_CK(cudaMemcpy(iscal, P.iscal, sizeof(iscal), cudaMemcpyDeviceToHost));
  SMA_CK(cudaMemcpy(&status, P.status, sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<double> orth(P.n_orth);
  SMA_CK(cudaMemcpy(orth.data(), P.orth, P.n_orth * sizeof(double), cudaMemcpyDeviceToHost));
  const int nsw = h->opt.decomp == SMA_TSVDM ? P.p : P.n_orth;
  std::vector<int> sw(nsw);
  SMA_CK(cudaMemcpy(sw.data(), P.sweeps, nsw * sizeof(int), cudaMemcpyDeviceToHost));
  memcpy(P.h_iscal, iscal, sizeof(iscal));
  std::memset(r, 0, sizeof(*r));
  r->norm = std::sqrt(stats[0]);
  r->device_status = status;
  r->orth_defect = 0.0;
  for (double v : orth) r->orth_defect = std::fmax(r->orth_defect, v);
  r->sweeps_max = 0;
  for (int v : sw) r->sweeps_max = v > r->sweeps_max ? v : r->sweeps_max;
  const sma_decomp d = h->opt.decomp;
  double err2 = 0.0;
  if (d == SMA_TSVDM) {
    err2 = stats[1];
    r->total_rank = iscal[0];
    r->n_kron_terms = iscal[1];
  } else if (P.ml2) {
    err2 = stats[1];
    for (int t = 0; t < 4; ++t) r->ranks[t] = iscal[2 + t];
    r->total_rank = iscal[2] * iscal[3] * iscal[4] * iscal[5];
    r->n_kron_terms = iscal[1];
  } else if (d == SMA_HOSVD_MULTILEVEL) {
    err2 = stats[1];
    for (int t = 0; t < 3; ++t) r->ranks[t] = iscal[2 + t];
    r->total_rank = iscal[2] * iscal[3] * iscal[4];
    r->n_kron_terms = r->total_rank;
  } else if (d == SMA_TUCKER_BLOCKMODE || d == SMA_CP_ALS) {
    err2 = stats[1];
    r->ranks[0] = iscal[2];
    r->total_rank = iscal[2];
    r->n_kron_terms = iscal[2];
  } else {
    r->ranks[0] = iscal[2];
    r->ranks[1] = d == SMA_TUCKER_ROWCOL ? iscal[3] : iscal[2];
    r->total_rank = r->ranks[0] * r->ranks[1];
    r->n_kron_terms = 0;
    err2 = stats[1];
  }
  r->tensor_err = std::sqrt(std::fmax(err2, 0.0));
  r->rel_err = stats[0] > 0 ? r->tensor_err / r->norm : 0.0;
  r->storage_ratio = storage_ratio(h, P, *r);
  SMA_TRY(trace_error(h, P, &r->trace_relerr));
  return SMA_OK;
}

template <typename T>
sma_status enqueue_compress(sma_ctx* h, const void* const* A, const int64_t* lda) {
  auto& ps = probs<T>(h);
  SMA_CK(cudaMemsetAsync(h->status_pool, 0, sizeof(int) * (size_t)h->nprob, h->st));
  bool gathered = false;
  if (h->opt.decomp == SMA_TSVDM) SMA_TRY(gather_all<T>(h, A, lda, &gathered));
  if (h->opt.decomp == SMA_TSVDM && gathered && h->naux > 0) {
    stage_begin(h, SMA_STAGE_TRANSFORM);
    SMA_TRY(transform_fanout<T>(h));
    stage_end(h);
    for (auto& P : ps) {
      P.compressed = true;
      P.dp_valid = false;
      for (auto& o : P.tca) o.valid = false;
      P.cq_valid = false;
      P.h_iscal[0] = -1;
    }
  } else {
    for (int i = 0; i < h->nprob; ++i) SMA_TRY(compress_one(h, ps[i], A[i], lda[i], gathered));
  }
  if (h->opt.decomp == SMA_TSVDM) {
    if (h->nprob > 1) {
      SMA_TRY(tsvdm_svd_batched<T>(h));
    } else {
      SMA_TRY(tsvdm_svd(h, ps[0]));
    }
    const bool batched = h->nprob > 1 && h->tdesc;
    if (batched) {
      SMA_TRY(truncate_all<T>(h));
      stage_begin(h, SMA_STAGE_FACTORS);
      for (auto& b : bins<T>(h))
        if (b.post_count > 0)
          SMA_K(slice_post<T>(b.post, b.post_count, b.pm, b.pn, b.pmm, b.prc, b.ptrans, h->st));
      stage_end(h);
    }
    for (int i = 0; i < h->nprob; ++i)
      if (!ps[i].post_batched) SMA_TRY(tsvdm_post(h, ps[i], batched));
  }
  return SMA_OK;
}

template <typename T>
void mark_compressed(sma_ctx* h) {
  for (auto& P : probs<T>(h)) {
    P.compressed = true;
    P.dp_valid = false;
    for (auto& o : P.tca) o.valid = false;
    P.cq_valid = false;
    P.ml_valid = false;
    P.ml_cvalid = false;
    P.h_iscal[0] = -1;
  }
}

// Graph mode: run normally the first time a set of inputs is seen (this also
// uploads the representative-block offsets), capture the launches into a
// CUDA graph the second time, replay the graph while inputs are unchanged.
template <typename T>
sma_status run_compress(sma_ctx* h, const void* const* A, const int64_t* lda) {
  std::vector<const void*> ptrs(A, A + h->nprob);
  std::vector<int64_t> ld(lda, lda + h->nprob);
  const bool graph_ok = h->opt.graph && h->st != nullptr;
  if (graph_ok && h->graph_exec && ptrs == h->graph_ptrs && ld == h->graph_lda) {
    SMA_CK(cudaGraphLaunch(h->graph_exec, h->st));
    h->launches += h->graph_launches;
    mark_compressed<T>(h);
    return SMA_OK;
  }
  if (graph_ok && ptrs == h->warm_ptrs && ld == h->warm_lda) {
    bool host_input = false;
    for (const void* q : ptrs) host_input |= !is_device_ptr(q);
    if (!host_input) {
      if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
      }
      SMA_CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
      h->capturing = true;
      const int64_t l0 = h->launches;
      sma_status s = enqueue_compress<T>(h, A, lda);
      h->capturing = false;
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(h->st, &g);
      if (s != SMA_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      SMA_CK(ec);
      const cudaError_t ei = cudaGraphInstantiate(&h->graph_exec, g, 0);
      cudaGraphDestroy(g);
      SMA_CK(ei);
      h->graph_launches = h->launches - l0;
      h->graph_ptrs = ptrs;
      h->graph_lda = ld;
      SMA_CK(cudaGraphLaunch(h->graph_exec, h->st));
      mark_compressed<T>(h);
      return SMA_OK;
    }
  }
  SMA_TRY(enqueue_compress<T>(h, A, lda));
  h->warm_ptrs = ptrs;
  h->warm_lda = ld;
  return SMA_OK;
}

template <typename T>
sma_status compress_all(sma_ctx* h, const void* const* A, const int64_t* lda, sma_result* res) {
  SMA_TRY(run_compress<T>(h, A, lda));
  auto& ps = probs<T>(h);
  if (res) {
    sma_status worst = SMA_OK;
    for (int i = 0; i < h->nprob; ++i) {
      SMA_TRY(read_result(h, ps[i], &res[i]));
      const int ds = res[i].device_status;
      if (ds & SMA_STATUS_BIT(SMA_ERR_NOT_SPD)) worst = SMA_ERR_NOT_SPD;
      else if ((ds & SMA_STATUS_BIT(SMA_ERR_NONFINITE)) && worst != SMA_ERR_NOT_SPD)
        worst = SMA_ERR_NONFINITE;
      else if ((ds & SMA_STATUS_BIT(SMA_ERR_NOCONVERGE)) && worst == SMA_OK) worst = SMA_ERR_NOCONVERGE;
    }
    return worst;
  }
  return SMA_OK;
}

template <typename T>
sma_status grow(sma_ctx* h, T** buf, size_t* have, size_t need) {
  if (*have >= need) return SMA_OK;
  if (*buf) h->mem.release(*buf);
  *buf = nullptr;
  *have = 0;
  SMA_TRY(h->mem.alloc(buf, need));
  *have = need;
  return SMA_OK;
}

// Mixed-path Kronecker-sum matvec on tensor cores: Y^T = Z^T D^T with
// Z = [X_s C_j^T] and D = [D_1 | ... | D_nt].  Both products run in tcgen05
// kernels on the fp16 two-piece split (x s = hi + lo with a power-of-two
// scale s per operand that puts its largest entry below 2^15, the products
// hi hi + hi lo + lo hi, fp32 accumulation): each piece carries 11 bits, the
// pair 22, so a product term is exact to about 2^-21 relative, and half the
// bf16 three-piece form's six products are needed.  The mid-index
// contraction (K = q) writes Z directly as the scaled fp16 planes of the
// long-K product's operand; its scale comes from the bound |Z| <= max |X|
// max_a,j sum_b |C_j[a, b]|.  Returns false when the shapes do not fit the
// kernels (the caller then runs the CUDA-core form).
template <typename T>
bool tc_apply(sma_ctx*, Prob<T>&, const T*, int64_t, T*, int64_t, int64_t, int, int) {
  return false;
}
template <>
bool tc_apply<float>(sma_ctx* h, Prob<float>& P, const float* X, int64_t ldx, float* Yd,
                     int64_t ldyd, int64_t yrows, int nrhs, int nt) {
  if (!h->tc_ok || ldyd != yrows || P.m > 256 || nt <= 0) return false;
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, ell = P.ell, q = P.q;
  const int64_t K = (int64_t)n * nt, Kp = tc_pad_k(K);
  const int64_t rowsZ = (int64_t)ell * nrhs;
  if (rowsZ > 0x7fffffff) return false;
  const size_t zneed = (size_t)2 * rowsZ * Kp, dneed = (size_t)2 * m * Kp;
  if (!P.tcmx) {
    if (h->mem.alloc(&P.tcmx, 4) != SMA_OK || h->mem.alloc(&P.tcsc, 8) != SMA_OK) return false;
    if (cudaMemsetAsync(P.tcmx, 0, 4 * sizeof(unsigned), st) != cudaSuccess) return false;
  }
  const uint16_t* zold = P.Zp;
  if (grow(h, &P.Zp, &P.Zp_elems, zneed) != SMA_OK) return false;
  if (P.Zp != zold) P.Zp_K = -1;   // a new buffer: its K padding is not zero yet
  if (grow(h, &P.Dp, &P.Dp_elems, dneed) != SMA_OK) return false;
  if (P.Zp_K != K) {  // zero the K padding once per shape
    if (cudaMemsetAsync(P.Zp, 0, P.Zp_elems * sizeof(uint16_t), st) != cudaSuccess) return false;
    P.Zp_K = K;
  }
  if (!P.dp_valid || P.Dp_K != K) {
    if (P.Dp_K != K &&
        cudaMemsetAsync(P.Dp, 0, P.Dp_elems * sizeof(uint16_t), st) != cudaSuccess)
      return false;
    h->launches += 3;
    if (tc_absmax(P.D, m, K, m, P.tcmx + 3, st) != cudaSuccess ||
        tc_f16_scales(P.tcmx, P.tcsc, st) != cudaSuccess ||
        tc_split2_transpose_batched(P.D, 1, m, m, (int)K, Kp, 1, 0, 0, (int64_t)m * Kp,
                                    P.tcsc + 2, P.Dp, st) != cudaSuccess)
      return false;
    P.Dp_K = K;
    P.dp_valid = true;
  }
  // Z^T planes: element (c, a) of batch (j, s) at (a + ell s) Kp + c + n j,
  // from X_s[c, b] (c + n b + ldx s) and C_j[a, b] (a + ell b + ell q j)
  const int64_t Kq = tc_pad_k(q);
  const int64_t rowsX = (int64_t)n * nrhs, rowsC = (int64_t)ell * nt;
  if (rowsX > 0x7fffffff || rowsC > 0x7fffffff || nrhs > 65535 || nt > 65535) return false;
  const int64_t xshape = rowsX * Kq;
  if (P.Xq_shape != xshape) {  // zero the K padding (b >= q) once per shape
    if (grow(h, &P.Xq, &P.Xq_elems, (size_t)2 * rowsX * Kq) != SMA_OK) return false;
    if (cudaMemsetAsync(P.Xq, 0, (size_t)2 * rowsX * Kq * sizeof(uint16_t), st) != cudaSuccess)
      return false;
    P.Xq_shape = xshape;
  }
  if (!P.cq_valid) {
    if (grow(h, &P.Cq, &P.Cq_elems, (size_t)2 * rowsC * Kq) != SMA_OK) return false;
    if (cudaMemsetAsync(P.Cq, 0, (size_t)2 * rowsC * Kq * sizeof(uint16_t), st) != cudaSuccess)
      return false;
    h->launches += 4;
    if (tc_absmax(P.C, (int64_t)ell * q, nt, (int64_t)ell * q, P.tcmx + 1, st) != cudaSuccess ||
        tc_rowl1max(P.C, ell, q, nt, P.tcmx + 2, st) != cudaSuccess ||
        tc_f16_scales(P.tcmx, P.tcsc, st) != cudaSuccess ||
        tc_split2_transpose_batched(P.C, 1, ell, ell, q, Kq, nt, (int64_t)ell * q,
                                    (int64_t)ell * Kq, rowsC * Kq, P.tcsc + 1, P.Cq, st) !=
            cudaSuccess)
      return false;
    P.cq_valid = true;
  }
  // the right-hand sides' scale, then every factor of this product
  h->launches += 2;
  if (tc_absmax(X, (int64_t)n * q, nrhs, ldx, P.tcmx, st) != cudaSuccess ||
      tc_f16_scales(P.tcmx, P.tcsc, st) != cudaSuccess)
    return false;
  ++h->launches;
  if (tc_split2_transpose_batched(X, 1, n, n, q, Kq, nrhs, ldx, (int64_t)n * Kq, rowsX * Kq,
                                  P.tcsc, P.Xq, st) != cudaSuccess)
    return false;
  ++h->launches;
  if (tc_mid_planes_f16(P.Xq, (int)rowsX, P.Cq, (int)rowsC, Kq, P.Zp, Kp, rowsZ * Kp, n, ell,
                        P.tcsc + 4, P.status, st) != cudaSuccess)
    return false;
  ++h->launches;
  if (tc_gemm_planes_f16(P.Zp, P.Dp, (int)rowsZ, m, Kp, Yd, m, P.tcsc + 5, P.status, st) !=
      cudaSuccess)
    return false;
  return true;
}

// The fp32 products of the block-low-rank and SPD matvecs, C = A B with A a
// factor of the compressed form (W^T, the structured core, U, L^T, L) and B
// the right-hand sides or an intermediate, on tcgen05 in the fp16 two-piece
// form of the Kronecker-sum matvec when they are large: A's scaled planes are
// built once per compression and cached (keyed by pointer, shape and
// strides), B's each call; the output scale 1 / (s_A s_B) is applied in the
// GEMM's epilogue.  A batch over nb2 is folded into the columns when B's and
// C's batches continue their columns.  Other shapes, and the fp64 path, take
// the CUDA-core product.
template <typename T>
sma_status contract_apply(sma_ctx* h, Prob<T>&, const GemmParams<T>& g) {
  SMA_K(contract<T>(h, g));
  return SMA_OK;
}
template <>
sma_status contract_apply<float>(sma_ctx* h, Prob<float>& P, const GemmParams<float>& g) {
  cudaStream_t st = h->st;
  int64_t N = g.N;
  bool ok = h->tc_ok && !g.dM && !g.dN && !g.dK && !g.dKoff && !g.c_off && !g.Cs &&
            g.kchunk == 0 && g.alpha == 1.f && g.beta == 0.f && g.nb1 == 1 &&
            (g.c_rs == 1 || g.c_cs == 1);
  if (ok && g.nb2 > 1) {
    ok = g.a_b2 == 0 && g.b_b2 == (int64_t)g.N * g.b_cs && g.c_b2 == (int64_t)g.N * g.c_cs;
    N = (int64_t)g.N * g.nb2;
  }
  ok = ok && g.M >= 128 && N >= 128 && g.K >= 64 && N <= 0x7fffffff &&
       (double)g.M * (double)N * (double)g.K >= 268435456.0 && (N + 255) / 256 <= 65535;
  if (!ok) {
    SMA_K(contract<float>(h, g));
    return SMA_OK;
  }
  const int M = g.M, K = g.K;
  const int64_t Kp = tc_pad_k(K);
  // A: the cached factor planes
  Prob<float>::TcOperand* op = nullptr;
  for (auto& o : P.tca)
    if (o.src == g.A && o.M == M && o.K == K && o.rs == g.a_rs && o.cs == g.a_cs) op = &o;
  if (!op) {
    P.tca.emplace_back();
    op = &P.tca.back();
    op->src = g.A; op->M = M; op->K = K; op->rs = g.a_rs; op->cs = g.a_cs;
  }
  if (!op->valid) {
    if (!op->mx) {
      SMA_TRY(h->mem.alloc(&op->mx, 1));
      SMA_TRY(h->mem.alloc(&op->s, 1));
    }
    SMA_TRY(grow(h, &op->planes, &op->elems, (size_t)2 * M * Kp));
    op->Kp = Kp;
    if (Kp > K)   // the K padding of both planes
      SMA_CK(cudaMemset2DAsync(op->planes + K, Kp * sizeof(uint16_t), 0,
                               (Kp - K) * sizeof(uint16_t), (size_t)2 * M, st));
    h->launches += 3;
    SMA_CK(tc_absmax_strided(g.A, M, K, g.a_rs, g.a_cs, op->mx, st));
    SMA_CK(tc_f16_scale1(op->mx, op->s, st));
    SMA_CK(tc_split2_transpose_batched(g.A, g.a_rs, g.a_cs, M, K, Kp, 1, 0, 0, (int64_t)M * Kp,
                                       op->s, op->planes, st));
    op->valid = true;
  }
  // B (element (j, k) at B[k b_rs + j b_cs]) each call
  if (!h->tcb_mx) {
    SMA_TRY(h->mem.alloc(&h->tcb_mx, 1));
    SMA_TRY(h->mem.alloc(&h->tcb_sc, 2));
  }
  SMA_TRY(grow(h, &h->tcb, &h->tcb_elems, (size_t)2 * N * Kp));
  if (Kp > K)
    SMA_CK(cudaMemset2DAsync(h->tcb + K, Kp * sizeof(uint16_t), 0, (Kp - K) * sizeof(uint16_t),
                             (size_t)2 * N, st));
  h->launches += 4;
  SMA_CK(tc_absmax_strided(g.B, N, K, g.b_cs, g.b_rs, h->tcb_mx, st));
  SMA_CK(tc_f16_scale_out(op->mx, h->tcb_mx, h->tcb_sc, st));
  SMA_CK(tc_split2_transpose_batched(g.B, g.b_cs, g.b_rs, (int)N, K, Kp, 1, 0, 0, N * Kp,
                                     h->tcb_sc, h->tcb, st));
  const bool col = g.c_rs == 1;
  SMA_CK(tc_gemm_planes_f16(op->planes, h->tcb, M, (int)N, Kp, g.C, col ? g.c_cs : g.c_rs,
                            h->tcb_sc + 1, P.status, st, col));
  return SMA_OK;
}

// Section 7.4 matvec y = sum_j G_j (C1_j1 (x) C2_j2 (x) C3_j3) x for volumes
// x (level-3 index fastest), as four strided batched GEMMs:
//   S1  U3x[(a3 + l3 j3), (b2, b1)]         = sum_b3 C3_j3[a3, b3] x[b3, b2, b1]
//   S2  V[a3 + l3 (j1 + k1 j2), (b2, b1)]   = sum_j3 G[j1, j2, j3] U3x[(a3 + l3 j3), (b2, b1)]
//   S3  W[(a3 + l3 j1), b1, a2]             = sum_{j2, b2} C2_j2[a2, b2] V[...]
//   S4  y[a3, a2, a1]                       = sum_{j1, b1} C1_j1[a1, b1] W[...]
// with C3 stacked ((l3 k3) x q3) and C1, C2 interleaved (l_t x (k_t q_t),
// column j + k_t b) so that every contraction runs over one stride.
template <typename T>
sma_status apply_multilevel(sma_ctx* h, Prob<T>& P, const T* X, int64_t ldx, T* Y, int64_t ldy,
                            int nv) {
  cudaStream_t st = h->st;
  if (P.h_iscal[0] < 0) {
    SMA_CK(cudaStreamSynchronize(st));
    SMA_CK(cudaMemcpy(P.h_iscal, P.iscal, sizeof(P.h_iscal), cudaMemcpyDeviceToHost));
  }
  const int k1 = P.h_iscal[2], k2 = P.h_iscal[3], k3 = P.h_iscal[4];
  const int l1 = P.lell[0], l2 = P.lell[1], l3 = P.lell[2];
  const int q1 = P.lq[0], q2 = P.lq[1], q3 = P.lq[2];
  const int p1 = P.lp[0], p2 = P.lp[1], p3 = P.lp[2];
  if (k1 <= 0 || k2 <= 0 || k3 <= 0) {
    SMA_CK(cudaMemset2DAsync(Y, ldy * sizeof(T), 0, (size_t)l1 * l2 * l3 * sizeof(T), nv, st));
    return SMA_OK;
  }
  if (!P.ml_valid) {
    if (!P.C1i) {
      SMA_TRY(h->mem.alloc(&P.C1i, (size_t)l1 * q1 * p1));
      SMA_TRY(h->mem.alloc(&P.C2i, (size_t)l2 * q2 * p2));
      SMA_TRY(h->mem.alloc(&P.C3st, (size_t)l3 * q3 * p3));
    }
    SMA_K(struct_strided<T>(P.d_lmap[2], P.d_lisq[2], l3, q3, P.Uml[2], p3, k3, 1,
                            (int64_t)l3 * k3, l3, P.C3st, st));
    SMA_K(struct_strided<T>(P.d_lmap[1], P.d_lisq[1], l2, q2, P.Uml[1], p2, k2, 1,
                            (int64_t)l2 * k2, l2, P.C2i, st));
    SMA_K(struct_strided<T>(P.d_lmap[0], P.d_lisq[0], l1, q1, P.Uml[0], p1, k1, 1,
                            (int64_t)l1 * k1, l1, P.C1i, st));
    for (int j3 = 0; j3 < k3; ++j3)
      SMA_CK(cudaMemcpy2DAsync(P.Gcmp + (size_t)k1 * k2 * j3, k1 * sizeof(T),
                               P.Gc + (size_t)p1 * p2 * j3, p1 * sizeof(T), k1 * sizeof(T), k2,
                               cudaMemcpyDeviceToDevice, st));
    P.ml_valid = true;
  }
  {  // the factors' structured form, when its plane fits in shared memory
    MlApply<T> mp;
    for (int t = 0; t < 3; ++t) {
      mp.l[t] = P.lell[t]; mp.q[t] = P.lq[t]; mp.p[t] = P.lp[t]; mp.nnz[t] = P.lnnz[t];
      mp.ptr[t] = P.d_lptr[t]; mp.col[t] = P.d_lcol[t]; mp.kk[t] = P.d_lkk[t];
      mp.isq[t] = P.d_lisq[t]; mp.U[t] = P.Uml[t];
    }
    mp.r[0] = k1; mp.r[1] = k2; mp.r[2] = k3;
    mp.G = P.Gc; mp.c1 = P.mlc1; mp.c2 = P.mlc2; mp.b = P.mlcb;
    if (ml_apply_smem(mp) <= (size_t)h->max_smem) {
      SMA_TRY(grow(h, &P.Wml, &P.Wml_elems, (size_t)l3 * l2 * k1 * q1 * nv));
      h->launches += P.ml_cvalid ? 1 : 2;
      SMA_K(ml_apply<T>(mp, !P.ml_cvalid, X, ldx, P.Wml, Y, ldy, nv, st));
      P.ml_cvalid = true;
      return SMA_OK;
    }
  }
  const int64_t n21 = (int64_t)q2 * q1;
  SMA_TRY(grow(h, &P.U3x, &P.U3x_elems, (size_t)l3 * k3 * n21 * nv));
  SMA_TRY(grow(h, &P.Vml, &P.Vml_elems, (size_t)l3 * k1 * k2 * n21 * nv));
  SMA_TRY(grow(h, &P.Wml, &P.Wml_elems, (size_t)l3 * k1 * q1 * l2 * nv));
  {  // S1
    GemmParams<T> g;
    g.M = l3 * k3; g.N = (int)n21; g.K = q3;
    g.A = P.C3st; g.a_rs = 1; g.a_cs = (int64_t)l3 * k3;
    g.B = X; g.b_rs = 1; g.b_cs = q3; g.b_b2 = ldx;
    g.C = P.U3x; g.c_rs = 1; g.c_cs = (int64_t)l3 * k3; g.c_b2 = (int64_t)l3 * k3 * n21;
    g.nb2 = nv;
    SMA_K(contract<T>(h, g));
  }
  if (k3 <= 16) {  // S2: the core over j3 for every (a3, column), coalesced over a3
    SMA_K(ml_core<T>(P.Gcmp, k1 * k2, k3, P.U3x, l3, n21 * nv, P.Vml, st));
  } else {  // S2 (batched over a3)
    GemmParams<T> g;
    g.M = k1 * k2; g.N = (int)(n21 * nv); g.K = k3;
    g.A = P.Gcmp; g.a_rs = 1; g.a_cs = (int64_t)k1 * k2;
    g.B = P.U3x; g.b_rs = l3; g.b_cs = (int64_t)l3 * k3; g.b_b1 = 1;
    g.C = P.Vml; g.c_rs = l3; g.c_cs = (int64_t)l3 * k1 * k2; g.c_b1 = 1;
    g.nb1 = l3;
    SMA_K(contract<T>(h, g));
  }
  {  // S3 (batched over b1, volume)
    GemmParams<T> g;
    g.M = l3 * k1; g.N = l2; g.K = k2 * q2;
    g.A = P.Vml; g.a_rs = 1; g.a_cs = (int64_t)l3 * k1;
    g.a_b1 = (int64_t)l3 * k1 * k2 * q2; g.a_b2 = (int64_t)l3 * k1 * k2 * n21;
    g.B = P.C2i; g.b_rs = l2; g.b_cs = 1;
    g.C = P.Wml; g.c_rs = 1; g.c_cs = (int64_t)l3 * k1 * q1;
    g.c_b1 = (int64_t)l3 * k1; g.c_b2 = (int64_t)l3 * k1 * q1 * l2;
    g.nb1 = q1; g.nb2 = nv;
    SMA_K(contract<T>(h, g));
  }
  {  // S4 (batched over a2, volume)
    GemmParams<T> g;
    g.M = l3; g.N = l1; g.K = k1 * q1;
    g.A = P.Wml; g.a_rs = 1; g.a_cs = l3;
    g.a_b1 = (int64_t)l3 * k1 * q1; g.a_b2 = (int64_t)l3 * k1 * q1 * l2;
    g.B = P.C1i; g.b_rs = l1; g.b_cs = 1;
    g.C = Y; g.c_rs = 1; g.c_cs = (int64_t)l3 * l2; g.c_b1 = l3; g.c_b2 = ldy;
    g.nb1 = l2; g.nb2 = nv;
    SMA_K(contract<T>(h, g));
  }
  return SMA_OK;
}

template <typename T>
sma_status apply_core(sma_ctx* h, Prob<T>& P, const T* X, int64_t ldx, T* Yd, int64_t ldyd,
                      int nrhs);
template <typename T>
sma_status spd_apply(sma_ctx* h, Prob<T>& P, const T* X, int64_t ldx, T* Yd, int64_t ldyd,
                     int nrhs);

template <typename T>
sma_status apply_one(sma_ctx* h, Prob<T>& P, const void* Xin, int64_t ldx, void* Yout,
                     int64_t ldy, int nrhs) {
  if (!P.compressed) return SMA_ERR_STATE;
  if (nrhs <= 0 || !Xin || !Yout) return SMA_ERR_ARG;
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, ell = P.ell, q = P.q;
  const int64_t xrows = (int64_t)q * n, yrows = (int64_t)ell * m;
  if (ldx < xrows || ldy < yrows) return SMA_ERR_ARG;
  const T* X = static_cast<const T*>(Xin);
  T* Y = static_cast<T*>(Yout);
  const bool xhost = !is_device_ptr(Xin), yhost = !is_device_ptr(Yout);
  if (xhost) {
    SMA_TRY(grow(h, &P.Xs, &P.Xs_elems, (size_t)xrows * nrhs));
    SMA_CK(cudaMemcpy2DAsync(P.Xs, xrows * sizeof(T), X, ldx * sizeof(T), xrows * sizeof(T), nrhs,
                             cudaMemcpyHostToDevice, st));
    X = P.Xs;
    ldx = xrows;
  }
  T* Yd = Y;
  int64_t ldyd = ldy;
  if (yhost) {
    SMA_TRY(grow(h, &P.Ys, &P.Ys_elems, (size_t)yrows * nrhs));
    Yd = P.Ys;
    ldyd = yrows;
  }
  stage_begin(h, SMA_STAGE_APPLY);
  if (P.spd) SMA_TRY(spd_apply(h, P, X, ldx, Yd, ldyd, nrhs));
  else SMA_TRY(apply_core(h, P, X, ldx, Yd, ldyd, nrhs));
  stage_end(h);
  if (yhost) {
    SMA_CK(cudaMemcpy2DAsync(Y, ldy * sizeof(T), Yd, yrows * sizeof(T), yrows * sizeof(T), nrhs,
                             cudaMemcpyDeviceToHost, st));
    SMA_CK(cudaStreamSynchronize(st));
  }
  return SMA_OK;
}

// Step 4 on device buffers: Y (ell m x nrhs, ld ldyd) = A_hat X (q n x nrhs,
// ld ldx) in the problem's factored form.
template <typename T>
sma_status apply_core(sma_ctx* h, Prob<T>& P, const T* X, int64_t ldx, T* Yd, int64_t ldyd,
                      int nrhs) {
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, ell = P.ell, q = P.q;
  const int64_t yrows = (int64_t)ell * m;
  const sma_decomp d = h->opt.decomp;
  if (d == SMA_HOSVD_MULTILEVEL && !P.ml2) {
    SMA_TRY(apply_multilevel(h, P, X, ldx, Yd, ldyd, nrhs));
  } else if (d == SMA_TSVDM || d == SMA_TUCKER_BLOCKMODE || d == SMA_CP_ALS || P.ml2) {
    // Kronecker sum Y = sum_j D_j X C_j^T (Section 2.2 vec identity).
    if (P.h_iscal[0] < 0) {
      SMA_CK(cudaStreamSynchronize(st));
      SMA_CK(cudaMemcpy(P.h_iscal, P.iscal, sizeof(P.h_iscal), cudaMemcpyDeviceToHost));
    }
    // t-SVDM: one term per slice (rank-0 slices have D_i = 0);
    // Tucker-1: the r2 retained block-mode columns.
    const int nt = d == SMA_TSVDM ? P.nterms_max : (P.ml2 ? P.h_iscal[1] : P.h_iscal[2]);
    if (nt <= 0) {
      if (ldyd == yrows) SMA_CK(cudaMemsetAsync(Yd, 0, sizeof(T) * (size_t)yrows * nrhs, st));
      else SMA_CK(cudaMemset2DAsync(Yd, ldyd * sizeof(T), 0, yrows * sizeof(T), nrhs, st));
      return SMA_OK;
    }
    const int64_t ldZ = (int64_t)n * nt;
    if (tc_apply(h, P, X, ldx, Yd, ldyd, yrows, nrhs, nt)) return SMA_OK;
    SMA_TRY(grow(h, &P.Z, &P.Z_elems, (size_t)ldZ * ell * nrhs));
    // Z[c + n j, a + ell s] = sum_b X_s[c, b] C_j[a, b]
    GemmParams<T> g;
    g.M = n; g.N = ell; g.K = q;
    g.A = X; g.a_rs = 1; g.a_cs = n; g.a_b2 = ldx;
    g.B = P.C; g.b_rs = ell; g.b_cs = 1; g.b_b1 = (int64_t)ell * q;
    g.C = P.Z; g.c_rs = 1; g.c_cs = ldZ; g.c_b1 = n; g.c_b2 = ldZ * ell;
    g.nb1 = nt; g.nb2 = nrhs;
    SMA_K(gemm<T>(g, st));
    // Y = [D_1 | ... | D_nt] Z   (m x (ell nrhs), K = n nt)
    GemmParams<T> g2;
    g2.M = m; g2.K = (int)ldZ;
    g2.A = P.D; g2.a_rs = 1; g2.a_cs = m;
    g2.B = P.Z; g2.b_rs = 1; g2.b_cs = ldZ;
    if (ldyd == yrows) {
      g2.N = ell * nrhs;
      g2.C = Yd; g2.c_rs = 1; g2.c_cs = m;
    } else {
      g2.N = ell; g2.nb2 = nrhs; g2.b_b2 = ldZ * ell;
      g2.C = Yd; g2.c_rs = 1; g2.c_cs = m; g2.c_b2 = ldyd;
    }
    SMA_K(contract<T>(h, g2));
  } else {
    // block low rank Y = (I (x) U) struct_E(F_k) (I (x) W^T) X
    const int r1max = P.r1max, r3max = P.r3max;
    const T* Wf = d == SMA_TUCKER_ROWCOL ? P.F2 : P.F1;
    SMA_TRY(grow(h, &P.Z, &P.Z_elems, (size_t)q * r3max * nrhs));
    SMA_TRY(grow(h, &P.Z2, &P.Z2_elems, (size_t)ell * r1max * nrhs));
    // Z[:, b + q s] = W^T X_s[:, b]   (r3max x q nrhs, zero rows beyond r3)
    GemmParams<T> g;
    g.M = r3max; g.N = q; g.K = n;
    g.A = Wf; g.a_rs = n; g.a_cs = 1;
    g.B = X; g.b_rs = 1; g.b_cs = n; g.b_b2 = ldx;
    g.C = P.Z; g.c_rs = 1; g.c_cs = r3max; g.c_b2 = (int64_t)r3max * q;
    g.nb2 = nrhs;
    SMA_TRY(contract_apply<T>(h, P, g));
    // Z2 = mid Z   ((ell r1max) x nrhs)
    GemmParams<T> g2;
    g2.M = ell * r1max; g2.N = nrhs; g2.K = q * r3max;
    g2.A = P.mid; g2.a_rs = 1; g2.a_cs = (int64_t)ell * r1max;
    g2.B = P.Z; g2.b_rs = 1; g2.b_cs = (int64_t)q * r3max;
    g2.C = P.Z2; g2.c_rs = 1; g2.c_cs = (int64_t)ell * r1max;
    SMA_TRY(contract_apply<T>(h, P, g2));
    // Y_s[:, a] = U Z2_s[:, a]
    GemmParams<T> g3;
    g3.M = m; g3.N = ell; g3.K = r1max;
    g3.A = P.F1; g3.a_rs = 1; g3.a_cs = m;
    g3.B = P.Z2; g3.b_rs = 1; g3.b_cs = r1max; g3.b_b2 = (int64_t)ell * r1max;
    g3.C = Yd; g3.c_rs = 1; g3.c_cs = m; g3.c_b2 = ldyd;
    g3.nb2 = nrhs;
    SMA_TRY(contract_apply<T>(h, P, g3));
  }
  return SMA_OK;
}

// Section 5.2: T_hat X = (I (x) L)(X' + A_hat X') with X' = (I (x) L^T) X.
template <typename T>
sma_status spd_apply(sma_ctx* h, Prob<T>& P, const T* X, int64_t ldx, T* Yd, int64_t ldyd,
                     int nrhs) {
  cudaStream_t st = h->st;
  const int m = P.m, ell = P.ell;
  const int64_t rows = (int64_t)ell * m;
  SMA_TRY(grow(h, &P.Sx, &P.Sx_elems, (size_t)rows * nrhs));
  SMA_TRY(grow(h, &P.Sy, &P.Sy_elems, (size_t)rows * nrhs));
  // X'[:, b + ell s] = L^T X_s[:, b]  (one product over all columns when X is contiguous)
  GemmParams<T> g;
  g.M = m; g.K = m;
  g.A = P.Lc; g.a_rs = m; g.a_cs = 1;
  g.B = X; g.b_rs = 1; g.b_cs = m;
  g.C = P.Sx; g.c_rs = 1; g.c_cs = m;
  if (ldx == rows) {
    g.N = (int)(ell * (int64_t)nrhs);
  } else {
    g.N = ell; g.b_b2 = ldx; g.c_b2 = rows; g.nb2 = nrhs;
  }
  SMA_TRY(contract_apply<T>(h, P, g));
  SMA_TRY(apply_core(h, P, P.Sx, rows, P.Sy, rows, nrhs));
  SMA_K(add_into<T>(P.Sx, rows, P.Sy, rows, rows, nrhs, st));
  // Y_s[:, a] = L Y'_s[:, a]
  GemmParams<T> g2;
  g2.M = m; g2.K = m;
  g2.A = P.Lc; g2.a_rs = 1; g2.a_cs = m;
  g2.B = P.Sy; g2.b_rs = 1; g2.b_cs = m;
  g2.C = Yd; g2.c_rs = 1; g2.c_cs = m;
  if (ldyd == rows) {
    g2.N = (int)(ell * (int64_t)nrhs);
  } else {
    g2.N = ell; g2.b_b2 = rows; g2.c_b2 = ldyd; g2.nb2 = nrhs;
  }
  SMA_TRY(contract_apply<T>(h, P, g2));
  return SMA_OK;
}

// The approximation tensor T (m x n x p) in P.Tt from the factors.
template <typename T>
sma_status make_T(sma_ctx* h, Prob<T>& P) {
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n, p = P.p;
  const int64_t mn = (int64_t)m * n;
  const sma_decomp d = h->opt.decomp;
  if (d == SMA_HOSVD_MULTILEVEL && !P.ml2) {
    const int p1 = P.lp[0], p2 = P.lp[1], p3 = P.lp[2];
    {  // T1 = G_(3) U3^T as (p1 p2) x p3, K = k3
      GemmParams<T> g;
      g.M = p1 * p2; g.N = p3; g.K = p3; g.dK = P.iscal + 4; g.dstride = 0;
      g.A = P.Gc; g.a_rs = 1; g.a_cs = (int64_t)p1 * p2;
      g.B = P.Uml[2]; g.b_rs = p3; g.b_cs = 1;
      g.C = P.T1; g.c_rs = 1; g.c_cs = (int64_t)p1 * p2;
      SMA_K(gemm<T>(g, st));
    }
    {  // T2[:, :, i3] = T1[:, :, i3] U2^T, K = k2
      GemmParams<T> g;
      g.M = p1; g.N = p2; g.K = p2; g.dK = P.iscal + 3; g.dstride = 0;
      g.A = P.T1; g.a_rs = 1; g.a_cs = p1; g.a_b1 = (int64_t)p1 * p2;
      g.B = P.Uml[1]; g.b_rs = p2; g.b_cs = 1;
      g.C = P.T2; g.c_rs = 1; g.c_cs = p1; g.c_b1 = (int64_t)p1 * p2;
      g.nb1 = p3;
      SMA_K(gemm<T>(g, st));
    }
    {  // T = U1 T2_(1), K = k1
      GemmParams<T> g;
      g.M = p1; g.N = p2 * p3; g.K = p1; g.dK = P.iscal + 2; g.dstride = 0;
      g.A = P.Uml[0]; g.a_rs = 1; g.a_cs = p1;
      g.B = P.T2; g.b_rs = 1; g.b_cs = p1;
      g.C = P.Tt; g.c_rs = 1; g.c_cs = p1;
      SMA_K(gemm<T>(g, st));
    }
    return SMA_OK;
  }
  if (d == SMA_TSVDM) {
    // T = Dtrunc x3 M^T: T_mat = D_mat M
    GemmParams<T> g;
    g.M = (int)mn; g.N = p; g.K = p;
    g.A = P.D; g.a_rs = 1; g.a_cs = mn;
    g.B = P.Mt; g.b_rs = 1; g.b_cs = p;
    g.C = P.Tt; g.c_rs = 1; g.c_cs = mn;
    SMA_K(gemm<T>(g, st));
  } else if (d == SMA_TUCKER_BLOCKMODE || d == SMA_CP_ALS || P.ml2) {
    // T = G x3 V: T_mat = G_mat V^T (CP: G_mat = [vec(Xf_j Zf_j^T)], V = Yf;
    // two levels: the D_t and the coefficient vectors, iscal[1] terms)
    GemmParams<T> g;
    g.M = (int)mn; g.N = p; g.K = p; g.dK = P.ml2 ? P.iscal + 1 : P.iscal + 2; g.dstride = 0;
    g.A = P.D; g.a_rs = 1; g.a_cs = mn;
    g.B = P.F1; g.b_rs = p; g.b_cs = 1;
    g.C = P.Tt; g.c_rs = 1; g.c_cs = mn;
    SMA_K(gemm<T>(g, st));
  } else {
    const T* Wf = d == SMA_TUCKER_ROWCOL ? P.F2 : P.F1;
    const int* r1 = P.iscal + 2;
    const int* r3 = d == SMA_TUCKER_ROWCOL ? P.iscal + 3 : P.iscal + 2;
    // tmp_k = U core_k  (m x r3), T_k = tmp_k W^T
    GemmParams<T> g;
    g.M = m; g.N = P.r3max; g.K = P.r1max; g.dN = r3; g.dK = r1; g.dstride = 0;
    g.A = P.F1; g.a_rs = 1; g.a_cs = m;
    g.B = P.core; g.b_rs = 1; g.b_cs = P.r1max; g.b_b1 = (int64_t)P.r1max * P.r3max;
    g.C = P.tmp; g.c_rs = 1; g.c_cs = m; g.c_b1 = (int64_t)m * P.r3max;
    g.nb1 = p;
    SMA_K(gemm<T>(g, st));
    GemmParams<T> g2;
    g2.M = m; g2.N = n; g2.K = P.r3max; g2.dK = r3; g2.dstride = 0;
    g2.A = P.tmp; g2.a_rs = 1; g2.a_cs = m; g2.a_b1 = (int64_t)m * P.r3max;
    g2.B = Wf; g2.b_rs = n; g2.b_cs = 1;
    g2.C = P.Tt; g2.c_rs = 1; g2.c_cs = m; g2.c_b1 = mn;
    g2.nb1 = p;
    SMA_K(gemm<T>(g2, st));
  }
  return SMA_OK;
}

// Section 5.2: T_hat = (I (x) L)(I + M_E[T])(I (x) L^T), densely, through
// two temporary (ell m)^2 buffers.
template <typename T>
sma_status spd_reconstruct(sma_ctx* h, Prob<T>& P, void* Ahat, int64_t ld) {
  cudaStream_t st = h->st;
  const int m = P.m, ell = P.ell;
  const int64_t rows = (int64_t)ell * m;
  SMA_TRY(make_T(h, P));
  T* dst = static_cast<T*>(Ahat);
  const bool host = !is_device_ptr(Ahat);
  T* W = nullptr;
  if (cudaMalloc(&W, 2 * (size_t)rows * rows * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return SMA_ERR_ALLOC;
  }
  T* W1 = W;
  T* W2 = W + (size_t)rows * rows;
  T* out = host ? W1 : dst;
  const int64_t ldo = host ? rows : ld;
  auto run = [&]() -> cudaError_t {
    cudaError_t e;
    ++h->launches;
    if ((e = scatter_ME<T>(P.d_map, P.d_isq, ell, ell, m, m, P.Tt, W1, rows, st)) != cudaSuccess)
      return e;
    ++h->launches;
    if ((e = add_identity<T>(W1, rows, rows, st)) != cudaSuccess) return e;
    // W2 = (I (x) L) W1: block row a of W1 times L
    GemmParams<T> g;
    g.M = m; g.N = (int)rows; g.K = m;
    g.A = P.Lc; g.a_rs = 1; g.a_cs = m;
    g.B = W1; g.b_rs = 1; g.b_cs = rows; g.b_b1 = m;
    g.C = W2; g.c_rs = 1; g.c_cs = rows; g.c_b1 = m;
    g.nb1 = ell;
    ++h->launches;
    if ((e = gemm<T>(g, st)) != cudaSuccess) return e;
    // out = W2 (I (x) L^T): block column b of W2 times L^T
    GemmParams<T> g2;
    g2.M = (int)rows; g2.N = m; g2.K = m;
    g2.A = W2; g2.a_rs = 1; g2.a_cs = rows; g2.a_b1 = (int64_t)m * rows;
    g2.B = P.Lc; g2.b_rs = m; g2.b_cs = 1;
    g2.C = out; g2.c_rs = 1; g2.c_cs = ldo; g2.c_b1 = (int64_t)m * ldo;
    g2.nb1 = ell;
    ++h->launches;
    if ((e = gemm<T>(g2, st)) != cudaSuccess) return e;
    if (host)
      e = cudaMemcpy2DAsync(dst, ld * sizeof(T), W1, rows * sizeof(T), rows * sizeof(T), rows,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  };
  const cudaError_t e = run();
  if (e != cudaSuccess) cudaStreamSynchronize(st);
  cudaFree(W);
  SMA_CK(e);
  return SMA_OK;
}

template <typename T>
sma_status reconstruct_one(sma_ctx* h, Prob<T>& P, void* Ahat, int64_t ld) {
  if (!P.compressed) return SMA_ERR_STATE;
  if (P.spd) {
    if (!Ahat || ld < (int64_t)P.ell * P.m) return SMA_ERR_ARG;
    return spd_reconstruct(h, P, Ahat, ld);
  }
  cudaStream_t st = h->st;
  const int m = P.m, n = P.n;
  if (!Ahat || ld < (int64_t)P.ell * m) return SMA_ERR_ARG;
  SMA_TRY(make_T(h, P));
  T* dst = static_cast<T*>(Ahat);
  const bool host = !is_device_ptr(Ahat);
  const int64_t rows = (int64_t)P.ell * m, cols = (int64_t)P.q * n;
  T* tmpA = nullptr;
  if (host) {
    if (cudaMalloc(&tmpA, rows * cols * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return SMA_ERR_ALLOC;
    }
  }
  ++h->launches;
  cudaError_t e;
  if (P.L == 3) {
    MlMaps mp;
    for (int t = 0; t < 3; ++t) {
      mp.map[t] = P.d_lmap[t];
      mp.isq[t] = P.d_lisq[t];
      mp.ell[t] = P.lell[t];
      mp.q[t] = P.lq[t];
      mp.p[t] = P.lp[t];
    }
    e = ml_scatter<T>(mp, P.Tt, host ? tmpA : dst, host ? rows : ld, st);
  } else {
    e = scatter_ME<T>(P.d_map, P.d_isq, P.ell, P.q, m, n, P.Tt, host ? tmpA : dst,
                      host ? rows : ld, st);
  }
  if (e == cudaSuccess && host) {
    e = cudaMemcpy2DAsync(dst, ld * sizeof(T), tmpA, rows * sizeof(T), rows * sizeof(T), cols,
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (tmpA) cudaFree(tmpA);
  SMA_CK(e);
  return SMA_OK;
}

template <typename T>
sma_status export_one(sma_ctx* h, Prob<T>& P, int which, void* dst, int64_t count,
                      int64_t* avail) {
  const void* src = nullptr;
  int64_t n = 0;
  size_t es = sizeof(T);
  const int64_t mnp = (int64_t)P.m * P.n * P.p;
  switch (which) {
    case 0: src = P.X; n = mnp; break;
    case 1: src = P.Xh; n = P.Xh ? mnp : 0; break;
    case 2:
      if (h->opt.decomp == SMA_HOSVD_MULTILEVEL) { src = P.gsig; n = (int64_t)P.gdim * (P.ml2 ? 4 : 3); }
      else if (h->opt.decomp == SMA_TSVDM) { src = P.sigma; n = (int64_t)P.rc * P.p; }
      else if (h->opt.decomp == SMA_CP_ALS) { src = nullptr; n = 0; }
      else {
        src = P.gsig;
        n = h->opt.decomp == SMA_TUCKER_BLOCKMODE ? (P.sk > 0 ? P.sk * P.sk : P.p) : P.m;
      }
      es = sizeof(double);
      break;
    case 3: src = P.Tt; n = mnp; break;
    case 4:
      if (P.ml2) { src = P.F1; n = (int64_t)P.p * P.p; }
      else if (h->opt.decomp == SMA_HOSVD_MULTILEVEL) { src = P.Uml[0]; n = (int64_t)P.lp[0] * P.lp[0]; }
      else if (h->opt.decomp == SMA_TUCKER_BLOCKMODE || h->opt.decomp == SMA_CP_ALS) {
        src = P.F1;
        n = (int64_t)P.p * P.p;
      }
      else if (h->opt.decomp != SMA_TSVDM) { src = P.F1; n = (int64_t)P.m * P.m; }
      break;
    case 5:
      if (P.spd) { src = P.Lc; n = (int64_t)P.m * P.m; }
      break;
    case 6:
      if (P.cp_r > 0) { src = P.cXf; n = (int64_t)P.m * P.cp_r; }
      break;
    case 7:
      if (P.cp_r > 0) { src = P.cZf; n = (int64_t)P.n * P.cp_r; }
      break;
    default: return SMA_ERR_ARG;
  }
  if (avail) *avail = n;
  if (count <= 0) return SMA_OK;
  if (!src || !dst || count > n) return SMA_ERR_ARG;
  SMA_CK(cudaStreamSynchronize(h->st));
  SMA_CK(cudaMemcpy(dst, src, count * es, cudaMemcpyDefault));
  return SMA_OK;
}

template <typename T>
sma_status ranks_one(sma_ctx* h, Prob<T>& P, int32_t* out, int32_t* count) {
  SMA_CK(cudaStreamSynchronize(h->st));
  if (h->opt.decomp == SMA_TSVDM) {
    SMA_CK(cudaMemcpy(out, P.ranks, P.p * sizeof(int), cudaMemcpyDeviceToHost));
    *count = P.p;
  } else {
    int isc[8];
    SMA_CK(cudaMemcpy(isc, P.iscal, sizeof(isc), cudaMemcpyDeviceToHost));
    const sma_decomp d = h->opt.decomp;
    const int c = P.ml2 ? 4
                        : (d == SMA_TUCKER_BLOCKMODE || d == SMA_CP_ALS)
                              ? 1
                              : (d == SMA_HOSVD_MULTILEVEL ? 3 : 2);
    const bool shared = d == SMA_TUCKER_SHARED_U || d == SMA_TUCKER_SPD;
    for (int i = 0; i < c; ++i) out[i] = shared ? isc[2] : isc[2 + i];
    *count = c;
  }
  return SMA_OK;
}

}  // namespace

// Group the slices of all t-SVDM problems by slice size; upload one
// descriptor array per size and allocate its block-mode workspace.
template <typename T>
sma_status build_bins(sma_ctx* h) {
  auto& ps = probs<T>(h);
  auto& bs = bins<T>(h);
  std::vector<std::vector<SliceDesc<T>>> host;
  for (auto& P : ps) {
    size_t bi = 0;
    // the Jacobi input: the slice, or R1^T (rc x rc) with the QR preconditioning
    const int jm = P.qr ? P.rc : P.m, jn = P.qr ? P.rc : P.n;
    for (; bi < bs.size(); ++bi)
      if (bs[bi].m == jm && bs[bi].n == jn) break;
    if (bi == bs.size()) {
      SvdBin<T> b;
      b.m = jm;
      b.n = jn;
      b.jp = P.jp;
      bs.push_back(b);
      host.emplace_back();
    }
    const int64_t jmn = (int64_t)jm * jn, urc = (int64_t)P.jp.mm * P.rc,
                  vrc = (int64_t)P.rc * P.rc;
    const T* jsrc = P.qr ? qr_jacobi_input(P) : P.Xh;
    for (int k = 0; k < P.p; ++k)
      host[bi].push_back(SliceDesc<T>{jsrc + k * jmn, P.U + k * urc, P.V + k * vrc,
                                      P.sigma + (int64_t)k * P.rc, P.sweeps + k, P.status});
  }
  // the per-slice rebuild and report of the problems without QR, batched by
  // bin when a slice's W and V fit in shared memory
  std::vector<std::vector<PostDesc<T>>> post(bs.size());
  for (auto& P : ps) {
    if (P.qr || ps.size() < 2) continue;
    const size_t smem = sizeof(T) * ((size_t)P.jp.mm * P.rc + (size_t)P.rc * P.rc + P.rc);
    if (smem > (size_t)h->max_smem) continue;
    size_t bi = 0;
    for (; bi < bs.size(); ++bi)
      if (bs[bi].m == P.m && bs[bi].n == P.n) break;
    if (bi == bs.size()) continue;
    auto& b = bs[bi];
    if (!post[bi].empty() &&
        (b.pm != P.m || b.pn != P.n || b.pmm != P.jp.mm || b.prc != P.rc || b.ptrans != P.trans))
      continue;
    b.pm = P.m; b.pn = P.n; b.pmm = P.jp.mm; b.prc = P.rc; b.ptrans = P.trans;
    const int64_t mn = (int64_t)P.m * P.n, urc = (int64_t)P.jp.mm * P.rc,
                  vrc = (int64_t)P.rc * P.rc;
    for (int k = 0; k < P.p; ++k)
      post[bi].push_back(PostDesc<T>{P.Xh + k * mn, P.D + k * mn, P.U + k * urc, P.V + k * vrc,
                                     P.sigma + (int64_t)k * P.rc, P.ranks + k, P.orth + k});
    P.post_batched = true;
  }
  for (size_t bi = 0; bi < bs.size(); ++bi) {
    auto& b = bs[bi];
    if (!post[bi].empty()) {
      b.post_count = (int)post[bi].size();
      SMA_TRY(h->mem.alloc(&b.post, post[bi].size()));
      SMA_CK(cudaMemcpy(b.post, post[bi].data(), post[bi].size() * sizeof(PostDesc<T>),
                        cudaMemcpyHostToDevice));
    }
    b.count = (int)host[bi].size();
    SMA_TRY(h->mem.alloc(&b.desc, host[bi].size()));
    SMA_CK(cudaMemcpy(b.desc, host[bi].data(), host[bi].size() * sizeof(SliceDesc<T>),
                      cudaMemcpyHostToDevice));
    if (b.jp.block_mode)
      SMA_TRY(h->mem.alloc(&b.W, (size_t)(b.jp.mm + b.jp.rc) * b.jp.rc * b.count));
  }
  std::vector<TruncDesc> td;
  for (auto& P : ps)
    td.push_back(TruncDesc{P.sigma, P.rc, P.p, P.stats, P.ranks, P.off, P.stats + 1, P.iscal,
                           P.suf});
  SMA_TRY(h->mem.alloc(&h->tdesc, td.size()));
  SMA_CK(cudaMemcpy(h->tdesc, td.data(), td.size() * sizeof(TruncDesc), cudaMemcpyHostToDevice));
  return SMA_OK;
}

// Shared state of the Gram eigen-solves: the split-K partial products hold
// nsplit * rows^2 doubles with nsplit <= 2 nsm / tiles + 1 and tiles >=
// rows^2 / 4096, so 2 nsm 4096 + rows^2 bounds every Gram of the handle.
static sma_status setup_gram_shared(sma_ctx* h) {
  int gmax = 1;
  for (auto& P : h->p64) gmax = P.gdim > gmax ? P.gdim : gmax;
  for (auto& P : h->p32) gmax = P.gdim > gmax ? P.gdim : gmax;
  h->gpart_elems = (size_t)2 * h->nsm * 4096 + (size_t)gmax * gmax;
  SMA_TRY(h->mem.alloc(&h->gpart, h->gpart_elems));
  const int sweeps = h->opt.max_sweeps > 0 ? h->opt.max_sweeps : 30;
  SMA_TRY(h->mem.alloc(&h->coop_bar, 1));
  SMA_TRY(h->mem.alloc(&h->coop_rot, (size_t)sweeps));
  SMA_TRY(h->mem.alloc(&h->coop_abort, 1));
  return SMA_OK;
}

// ===========================================================================
// exported C ABI
// ===========================================================================
extern "C" {

const char* sma_version(void) { return "sma 0.1 (sm_103a)"; }

const char* sma_status_string(sma_status s) {
  switch (s) {
    case SMA_OK: return "ok";
    case SMA_ERR_ARG: return "invalid argument";
    case SMA_ERR_STRUCT: return "invalid structure map";
    case SMA_ERR_CUDA: return "CUDA error";
    case SMA_ERR_ALLOC: return "device allocation failed";
    case SMA_ERR_NOCONVERGE: return "Jacobi sweep limit reached";
    case SMA_ERR_TIMEOUT: return "device wait timed out";
    case SMA_ERR_NONFINITE: return "non-finite value";
    case SMA_ERR_STATE: return "call out of order";
    case SMA_ERR_UNSUPPORTED: return "unsupported option";
    case SMA_ERR_NOT_SPD: return "diagonal block not positive definite";
  }
  return "unknown status";
}

sma_status sma_create(sma_handle* out, const sma_problem* prob, int32_t nprob,
                      const sma_options* opt) {
  if (!out) return SMA_ERR_ARG;
  *out = nullptr;
  if (!prob || !opt || nprob < 1) return SMA_ERR_ARG;
  if (opt->prec != SMA_FP64 && opt->prec != SMA_MIXED) return SMA_ERR_ARG;
  if ((int)opt->decomp < 0 || opt->decomp > SMA_CP_ALS) return SMA_ERR_ARG;
  if (opt->decomp == SMA_CP_ALS) {
    // CP: a rank the small solves take, iterations, both initial factors, one (m, n)
    if (opt->fixed_rank < 1 || opt->fixed_rank > kCpMaxRank || opt->cp_iters < 1 ||
        !opt->cp_init_x || !opt->cp_init_z)
      return SMA_ERR_ARG;
    for (int i = 1; i < nprob; ++i)
      if (prob[i].m != prob[0].m || prob[i].n != prob[0].n) return SMA_ERR_ARG;
  }
  if ((int)opt->mkind < 0 || opt->mkind > SMA_M_USER) return SMA_ERR_ARG;
  if (opt->layout != SMA_INPUT_DENSE && opt->layout != SMA_INPUT_BLOCKS) return SMA_ERR_ARG;
  if (opt->fixed_rank < 0 || !(opt->rel_tol >= 0.0)) return SMA_ERR_ARG;
  if ((int)opt->precondition < 0 || opt->precondition > SMA_PRECOND_QRCP2) return SMA_ERR_ARG;
  if (opt->autotune < 0 || opt->autotune > 1) return SMA_ERR_ARG;
  if (opt->sketch_cols < 0) return SMA_ERR_ARG;
  if (opt->sketch_cols > 0) {
    // Section 6.3's randomized factor: block-index mode, a fixed rank the
    // sketch can hold, both maps, one (m, n) for all problems
    if (opt->decomp != SMA_TUCKER_BLOCKMODE || !opt->sketch_omega || !opt->sketch_psi)
      return SMA_ERR_ARG;
    if (opt->fixed_rank < 1 || (int64_t)opt->fixed_rank > (int64_t)opt->sketch_cols * opt->sketch_cols)
      return SMA_ERR_ARG;
    for (int i = 1; i < nprob; ++i)
      if (prob[i].m != prob[0].m || prob[i].n != prob[0].n) return SMA_ERR_ARG;
  }
  // host-side validation of every problem before any CUDA call
  for (int i = 0; i < nprob; ++i) {
    std::vector<int64_t> eta;
    std::vector<int> ra, rb;
    if (opt->decomp == SMA_HOSVD_MULTILEVEL) {
      std::vector<int64_t> leta[3];
      SMA_TRY(validate_levels(prob[i], leta));
      if (prob[i].levels == 3 && opt->layout != SMA_INPUT_BLOCKS) return SMA_ERR_ARG;
      continue;
    }
    SMA_TRY(validate_problem(prob[i], eta, ra, rb));
    if (opt->decomp == SMA_TUCKER_SHARED_U && prob[i].m != prob[i].n) return SMA_ERR_ARG;
    if (opt->decomp == SMA_TUCKER_SPD) {
      int k0 = -1;
      std::vector<int32_t> inner;
      SMA_TRY(spd_split(prob[i], &k0, inner));
    }
    if (opt->decomp == SMA_TSVDM && opt->mkind == SMA_M_USER && !opt->M_user) return SMA_ERR_ARG;
  }
  std::unique_ptr<sma_ctx> h(new (std::nothrow) sma_ctx());
  if (!h) return SMA_ERR_ALLOC;
  h->opt = *opt;
  h->st = static_cast<cudaStream_t>(opt->stream);
  h->prof = opt->profile != 0;
  h->nprob = nprob;
  int dev = 0;
  SMA_CK(cudaGetDevice(&dev));
  SMA_CK(cudaDeviceGetAttribute(&h->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  int major = 0, minor = 0;
  SMA_CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  SMA_CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
  h->tc_ok = (opt->prec == SMA_MIXED) && tc_gemm_available(major, minor);
  SMA_CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev));
  SMA_TRY(h->mem.alloc(&h->status_pool, (size_t)nprob));
  if (opt->prec == SMA_FP64) {
    h->p64.resize(nprob);
    for (int i = 0; i < nprob; ++i) SMA_TRY(setup_problem(h.get(), h->p64[i], prob[i]));
    if (opt->decomp == SMA_TSVDM && nprob > 1) SMA_TRY(build_bins<double>(h.get()));
  } else {
    h->p32.resize(nprob);
    for (int i = 0; i < nprob; ++i) SMA_TRY(setup_problem(h.get(), h->p32[i], prob[i]));
    if (opt->decomp == SMA_TSVDM && nprob > 1) SMA_TRY(build_bins<float>(h.get()));
  }
  if (opt->decomp != SMA_TSVDM && opt->decomp != SMA_CP_ALS) SMA_TRY(setup_gram_shared(h.get()));
  if (opt->decomp == SMA_TSVDM && nprob > 1) {
    SMA_CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
    const int na = std::min(nprob, (int)sma_ctx::kAux);
    for (int k = 0; k < na; ++k) {
      SMA_CK(cudaStreamCreateWithFlags(&h->aux[k], cudaStreamNonBlocking));
      const cudaError_t e = cudaEventCreateWithFlags(&h->join_ev[k], cudaEventDisableTiming);
      if (e != cudaSuccess) {
        cudaStreamDestroy(h->aux[k]);
        h->aux[k] = nullptr;
        SMA_CK(e);
      }
      h->naux = k + 1;
    }
  }
  *out = h.release();
  return SMA_OK;
}

sma_status sma_compress(sma_handle h, const void* const* A, const int64_t* lda, sma_result* res) {
  if (!h || !A || !lda) return SMA_ERR_ARG;
  if (h->opt.prec == SMA_FP64) return compress_all<double>(h, A, lda, res);
  return compress_all<float>(h, A, lda, res);
}

sma_status sma_get_result(sma_handle h, int32_t i, sma_result* res) {
  if (!h || !res || i < 0 || i >= h->nprob) return SMA_ERR_ARG;
  if (h->opt.prec == SMA_FP64) {
    if (!h->p64[i].compressed) return SMA_ERR_STATE;
    return read_result(h, h->p64[i], res);
  }
  if (!h->p32[i].compressed) return SMA_ERR_STATE;
  return read_result(h, h->p32[i], res);
}

sma_status sma_get_ranks(sma_handle h, int32_t i, int32_t* ranks, int32_t* count) {
  if (!h || !ranks || !count || i < 0 || i >= h->nprob) return SMA_ERR_ARG;
  if (h->opt.prec == SMA_FP64) return ranks_one(h, h->p64[i], ranks, count);
  return ranks_one(h, h->p32[i], ranks, count);
}

sma_status sma_reconstruct(sma_handle h, int32_t i, void* Ahat, int64_t ld) {
  if (!h || i < 0 || i >= h->nprob) return SMA_ERR_ARG;
  if (h->opt.prec == SMA_FP64) return reconstruct_one(h, h->p64[i], Ahat, ld);
  return reconstruct_one(h, h->p32[i], Ahat, ld);
}

sma_status sma_apply(sma_handle h, int32_t i, const void* X, int64_t ldx, void* Y, int64_t ldy,
                     int32_t nrhs) {
  if (!h || i < 0 || i >= h->nprob) return SMA_ERR_ARG;
  if (h->opt.prec == SMA_FP64) return apply_one(h, h->p64[i], X, ldx, Y, ldy, nrhs);
  return apply_one(h, h->p32[i], X, ldx, Y, ldy, nrhs);
}

sma_status sma_export(sma_handle h, int32_t i, int32_t which, void* dst, int64_t count,
                      int64_t* avail) {
  if (!h || i < 0 || i >= h->nprob) return SMA_ERR_ARG;
  if (h->opt.prec == SMA_FP64) return export_one(h, h->p64[i], which, dst, count, avail);
  return export_one(h, h->p32[i], which, dst, count, avail);
}

sma_status sma_profile(sma_handle h, double* ms, int64_t* calls, int64_t* launches,
                       int32_t reset) {
  if (!h) return SMA_ERR_ARG;
  if (!h->prof) return SMA_ERR_STATE;
  SMA_CK(cudaStreamSynchronize(h->st));
  for (auto& pe : h->pend) {
    float t = 0.f;
    SMA_CK(cudaEventElapsedTime(&t, pe.a, pe.b));
    h->acc_ms[pe.stage] += t;
    h->acc_calls[pe.stage] += 1;
    h->ev_free.push_back(pe.a);
    h->ev_free.push_back(pe.b);
  }
  h->pend.clear();
  for (int s = 0; s < SMA_STAGE_COUNT; ++s) {
    if (ms) ms[s] = h->acc_ms[s];
    if (calls) calls[s] = h->acc_calls[s];
  }
  if (launches) *launches = h->launches;
  if (reset) {
    for (int s = 0; s < SMA_STAGE_COUNT; ++s) {
      h->acc_ms[s] = 0.0;
      h->acc_calls[s] = 0;
    }
    h->launches = 0;
  }
  return SMA_OK;
}

sma_status sma_destroy(sma_handle h) {
  if (!h) return SMA_ERR_ARG;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  delete h;
  return SMA_OK;
}

}  // extern "C"
