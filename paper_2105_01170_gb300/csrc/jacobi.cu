// One-sided (Hestenes) Jacobi SVD of a batch of frontal slices, one CTA per
// slice.
//
// The t-SVDM needs the SVD of every transformed frontal slice Xhat_i.  For an
// mm x rc working matrix W (the slice, transposed when it is wider than
// tall), pairs of columns are rotated until every pair is orthogonal to
// working precision: W V = W_inf with V orthogonal, sigma_j = ||W_inf[:,j]||,
// U = W_inf Sigma^-1 are the left singular vectors and V the right ones.  V is
// accumulated by applying every rotation to the stacked column [w_j; v_j]
// (length mm + rc, dot products over the first mm rows only), so that the
// truncated slice W_r V_r^T keeps the backward stability of one-sided Jacobi
// whatever the convergence tolerance.
//
// Layout on the GPU.  When the whole slice fits in shared memory it is
// loaded once and swept there (round-robin "circle" ordering: c-1 rounds of
// c/2 disjoint pairs, one group of g threads per pair).  Larger slices
// (e.g. 256 x 256 in fp32, 256 KB) use block Jacobi: the columns are split
// into nb >= 3 blocks, the slice lives in an L2-resident workspace, and each
// sweep visits every block pair (I, J) with both blocks staged in shared
// memory; the pairs inside a block are rotated on the block's first visit of
// the sweep and the I x J cross pairs on every visit, so one sweep rotates
// each column pair exactly once.
//
// Precision.  Dot products and rotations run in T (fp32 on the mixed path,
// fp64 on the fp64 path); the rotation angle and the convergence test are
// evaluated in fp64 on both paths; the final column norms are accumulated in
// fp64.  Rotation (Rutishauser form):
//   zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1/sqrt(1+t^2), s = c t, w_a' = c w_a - s w_b, w_b' = s w_a + c w_b,
// applied when |gamma| > tol sqrt(alpha beta); the caller sets tol (4 sqrt(mm) eps(T)).
#include "common.cuh"
#include "kernels.cuh"

namespace sma {
namespace {

struct Pair { int a, b; };

// Circle-method round robin on c (even) players: round t, pair k.
__device__ __forceinline__ Pair rr_pair(int k, int t, int c) {
  const int sb = c - 1 - k;
  Pair pr;
  pr.a = (k == 0) ? 0 : 1 + (k - 1 + t) % (c - 1);
  pr.b = 1 + (sb - 1 + t) % (c - 1);
  return pr;
}

// Rotate the columns at shared-memory slots a and b (group of g lanes, all
// lanes of the warp must call this together).  Returns true if rotated.
template <typename T>
__device__ __forceinline__ bool rotate_pair(T* S, int ldS, int a, int b, bool active,
                                            int mm, int len, int lane, int g, double tol) {
  T al = T(0), be = T(0), ga = T(0);
  T* x = S + (int64_t)(active ? a : 0) * ldS;
  T* y = S + (int64_t)(active ? b : 0) * ldS;
  if (active) {
    for (int r = lane; r < mm; r += g) {
      const T xv = x[r], yv = y[r];
      al = fma(xv, xv, al);
      be = fma(yv, yv, be);
      ga = fma(xv, yv, ga);
    }
  }
  for (int o = g >> 1; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  if (!active) return false;
  const double dal = (double)al, dbe = (double)be, dga = (double)ga;
  if (!(fabs(dga) > tol * sqrt(dal * dbe))) return false;
  const double zeta = (dbe - dal) / (2.0 * dga);
  const double t = (fabs(zeta) > 1e150) ? 0.5 / zeta
                                        : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double cs = 1.0 / sqrt(1.0 + t * t);
  const T c = (T)cs, s = (T)(cs * t);
  for (int r = lane; r < len; r += g) {
    const T xv = x[r], yv = y[r];
    x[r] = c * xv - s * yv;
    y[r] = s * xv + c * yv;
  }
  return true;
}

template <typename T>
__device__ __forceinline__ T load_work(const T* src, int m, int trans, int mm, int r, int c) {
  // stacked column c: rows [0, mm) the working matrix (the slice, m x n with
  // ld m, or its transpose), rows [mm, mm + rc) the identity (V_0 = I)
  if (r >= mm) return (r - mm == c) ? T(1) : T(0);
  return trans ? src[c + (int64_t)r * m] : src[r + (int64_t)c * m];
}

template <typename T>
__global__ void __launch_bounds__(1024) jacobi_kernel(const JacobiParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = blockIdx.x;
  const int tid = threadIdx.x, NTh = blockDim.x;
  const int mm = P.mm, rc = P.rc, ldS = P.ldS, g = P.g;
  const int len = mm + rc;  // stacked column [w; v]
  const int lane = tid % g, gid = tid / g, ngroups = NTh / g;
  const T* src = P.src + (int64_t)s * P.src_bs;
  const bool in_smem = rc <= 2 * P.bcols;
  const int ncols_smem = in_smem ? rc : 2 * P.bcols;
  T* S = reinterpret_cast<T*>(smem_raw);
  const int p2 = P.sort_n;  // power of two >= rc
  const size_t sig_off = ((size_t)ncols_smem * ldS * sizeof(T) + 15) & ~(size_t)15;
  double* sig = reinterpret_cast<double*>(smem_raw + sig_off);
  int* idx = reinterpret_cast<int*>(sig + p2);
  T* W = P.W ? P.W + (int64_t)s * P.W_bs : nullptr;

  int sweeps_used = 0;
  bool converged = false;
  if (in_smem) {
    const int tot = len * rc;
    for (int e = tid; e < tot; e += NTh) {
      int r, c;
      if (P.trans) { c = e % rc; r = e / rc; } else { r = e % len; c = e / len; }
      S[(int64_t)c * ldS + r] = load_work(src, P.m, P.trans, mm, r, c);
    }
    __syncthreads();
    const int c_even = rc + (rc & 1);
    const int npairs = c_even / 2;
    for (int sw = 0; sw < P.max_sweeps && rc > 1; ++sw) {
      bool rot = false;
      for (int t = 0; t < c_even - 1; ++t) {
        for (int base = 0; base < npairs; base += ngroups) {
          const int k = base + gid;
          Pair pr = rr_pair(k < npairs ? k : 0, t, c_even);
          const bool act = (k < npairs) && pr.a < rc && pr.b < rc;
          rot |= rotate_pair(S, ldS, pr.a, pr.b, act, mm, len, lane, g, P.tol);
        }
        __syncthreads();
      }
      sweeps_used = sw + 1;
      if (!__syncthreads_or(rot)) { converged = true; break; }
    }
    if (rc <= 1) converged = true;
  } else {
    // block mode: stacked working copy in global memory (len x rc)
    const int tot = len * rc;
    for (int e = tid; e < tot; e += NTh) {
      int r, c;
      if (P.trans) { c = e % rc; r = e / rc; } else { r = e % len; c = e / len; }
      W[r + (int64_t)c * len] = load_work(src, P.m, P.trans, mm, r, c);
    }
    __syncthreads();
    const int bc = P.bcols;
    const int nb = (rc + bc - 1) / bc;
    for (int sw = 0; sw < P.max_sweeps; ++sw) {
      bool rot = false;
      for (int I = 0; I < nb; ++I) {
        for (int J = I + 1; J < nb; ++J) {
          const int bI = min(bc, rc - I * bc), bJ = min(bc, rc - J * bc);
          // stage blocks I -> slots [0, bI), J -> slots [bc, bc + bJ)
          for (int e = tid; e < len * bI; e += NTh) {
            const int r = e % len, c = e / len;
            S[(int64_t)c * ldS + r] = W[r + (int64_t)(I * bc + c) * len];
          }
          for (int e = tid; e < len * bJ; e += NTh) {
            const int r = e % len, c = e / len;
            S[(int64_t)(bc + c) * ldS + r] = W[r + (int64_t)(J * bc + c) * len];
          }
          __syncthreads();
          // pairs inside a block on the block's first visit of this sweep
          const bool doI = (I == 0 && J == 1);
          const bool doJ = (I == 0);
          if (doI || doJ) {
            const int cI = doI ? bI + (bI & 1) : 0;
            const int cJ = doJ ? bJ + (bJ & 1) : 0;
            const int pI = cI / 2, pJ = cJ / 2;
            const int rounds = max(cI, cJ) - 1;
            for (int t = 0; t < rounds; ++t) {
              const int np = pI + pJ;
              for (int base = 0; base < np; base += ngroups) {
                const int k = base + gid;
                bool act = false;
                int a = 0, b = 0;
                if (k < pI) {
                  if (t < cI - 1) {
                    Pair pr = rr_pair(k, t, cI);
                    act = pr.a < bI && pr.b < bI;
                    a = pr.a; b = pr.b;
                  }
                } else if (k < np) {
                  if (t < cJ - 1) {
                    Pair pr = rr_pair(k - pI, t, cJ);
                    act = pr.a < bJ && pr.b < bJ;
                    a = bc + pr.a; b = bc + pr.b;
                  }
                }
                rot |= rotate_pair(S, ldS, a, b, act, mm, len, lane, g, P.tol);
              }
              __syncthreads();
            }
          }
          // cross pairs I x J
          for (int t = 0; t < bc; ++t) {
            for (int base = 0; base < bc; base += ngroups) {
              const int k = base + gid;
              const int j = (k + t) % bc;
              const bool act = (k < bc) && k < bI && j < bJ;
              rot |= rotate_pair(S, ldS, k, bc + j, act, mm, len, lane, g, P.tol);
            }
            __syncthreads();
          }
          for (int e = tid; e < len * bI; e += NTh) {
            const int r = e % len, c = e / len;
            W[r + (int64_t)(I * bc + c) * len] = S[(int64_t)c * ldS + r];
          }
          for (int e = tid; e < len * bJ; e += NTh) {
            const int r = e % len, c = e / len;
            W[r + (int64_t)(J * bc + c) * len] = S[(int64_t)(bc + c) * ldS + r];
          }
          __syncthreads();
        }
      }
      sweeps_used = sw + 1;
      if (!__syncthreads_or(rot)) { converged = true; break; }
    }
  }

  // column norms (fp64 accumulation)
  const int warp = tid >> 5, wl = tid & 31, nwarps = NTh >> 5;
  for (int c = warp; c < p2; c += nwarps) {
    double acc = 0.0;
    if (c < rc) {
      for (int r = wl; r < mm; r += 32) {
        const double v = in_smem ? (double)S[(int64_t)c * ldS + r] : (double)W[r + (int64_t)c * len];
        acc = fma(v, v, acc);
      }
    }
    acc = warp_sum(acc);
    if (wl == 0) {
      sig[c] = (c < rc) ? sqrt(acc) : -1.0;
      idx[c] = c;
    }
  }
  __syncthreads();
  // bitonic sort, descending by sigma, ties by ascending column
  for (int k = 2; k <= p2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < p2; i += NTh) {
        const int l = i ^ j;
        if (l > i) {
          const double si = sig[i], sl = sig[l];
          const int ii = idx[i], il = idx[l];
          // "i before l" in final order when (si > sl) or (si == sl and ii < il)
          const bool i_first = (si > sl) || (si == sl && ii < il);
          const bool up = ((i & k) == 0);
          if (up ? !i_first : i_first) {
            sig[i] = sl; sig[l] = si;
            idx[i] = il; idx[l] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
  // outputs: sorted sigma, the sorted columns W (= U Sigma) and V
  double* so = P.sigma + (int64_t)s * rc;
  for (int j = tid; j < rc; j += NTh) {
    so[j] = sig[j];
    if (!isfinite(sig[j])) atomicOr(P.status, SMA_STATUS_BIT(SMA_ERR_NONFINITE));
  }
  T* Wo = P.U + (int64_t)s * P.U_bs;
  T* Vo = P.V + (int64_t)s * P.V_bs;
  for (int e = tid; e < len * rc; e += NTh) {
    const int r = e % len, j = e / len;
    const int c = idx[j];
    const T v = in_smem ? S[(int64_t)c * ldS + r] : W[r + (int64_t)c * len];
    if (r < mm) Wo[r + (int64_t)j * mm] = v;
    else Vo[(r - mm) + (int64_t)j * rc] = v;
  }
  if (tid == 0) {
    if (P.sweeps) P.sweeps[s] = sweeps_used;
    if (!converged) atomicOr(P.status, SMA_STATUS_BIT(SMA_ERR_NOCONVERGE));
  }
}

}  // namespace

template <typename T>
JacobiPlan jacobi_plan(int m, int n, int max_smem) {
  JacobiPlan pl;
  pl.trans = (m < n) ? 1 : 0;
  pl.mm = pl.trans ? n : m;
  pl.rc = pl.trans ? m : n;
  pl.ldS = pl.mm + pl.rc + 1;
  int p2 = 1;
  while (p2 < pl.rc) p2 <<= 1;
  pl.sort_n = p2;
  const size_t sort_bytes = (size_t)p2 * (sizeof(double) + sizeof(int)) + 16;
  const size_t col_bytes = (size_t)pl.ldS * sizeof(T);
  const size_t full = (size_t)pl.rc * col_bytes + sort_bytes;
  if (full <= (size_t)max_smem) {
    pl.bcols = (pl.rc + 1) / 2 > 0 ? (pl.rc + 1) / 2 : 1;
    pl.smem = full;
  } else {
    const int bmax = (int)(((size_t)max_smem - sort_bytes) / (2 * col_bytes));
    const int nb = (pl.rc + bmax - 1) / bmax < 3 ? 3 : (pl.rc + bmax - 1) / bmax;
    pl.bcols = (pl.rc + nb - 1) / nb;
    pl.smem = 2 * (size_t)pl.bcols * col_bytes + sort_bytes;
  }
  const bool in_smem = pl.rc <= 2 * pl.bcols;
  const int maxpairs = in_smem ? (pl.rc + 1) / 2 : pl.bcols;
  // threads: one group of g lanes per pair of a round, about 16 rows per lane
  int gd = 1;
  while (gd < 32 && gd * 16 < pl.mm + pl.rc) gd <<= 1;
  int nt = 32;
  while (nt < 1024 && nt < maxpairs * gd) nt <<= 1;
  int gp = 1;
  while (gp * 2 <= 32 && gp * 2 * (maxpairs > 0 ? maxpairs : 1) <= nt) gp <<= 1;
  pl.threads = nt;
  pl.g = gp;
  pl.block_mode = in_smem ? 0 : 1;
  return pl;
}

template <typename T>
cudaError_t jacobi_svd(const JacobiParams<T>& P, int nslices, int threads, size_t smem,
                       cudaStream_t st) {
  if (nslices <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  jacobi_kernel<T><<<nslices, threads, smem, st>>>(P);
  return cudaGetLastError();
}

template JacobiPlan jacobi_plan<float>(int, int, int);
template JacobiPlan jacobi_plan<double>(int, int, int);
template cudaError_t jacobi_svd<float>(const JacobiParams<float>&, int, int, size_t, cudaStream_t);
template cudaError_t jacobi_svd<double>(const JacobiParams<double>&, int, int, size_t, cudaStream_t);

}  // namespace sma
