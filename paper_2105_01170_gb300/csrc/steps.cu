// Bandwidth-bound steps of the path: the struct_E gather (Section 3,
// matrix-to-tensor map), the global truncation rule, the construction of the
// structured Kronecker factors C_j = struct_E(v_j) (Theorem 'tuckerkron'),
// the tensor-to-matrix scatter M_E used for validation, and reports.
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace sma {
namespace {

constexpr int GATHER_THREADS = 256;
constexpr int GATHER_MAX_CTAS = 152 * 8;

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

// x = RN32(RN64(a w)) -- the product rounded to double, then to float, as the
// fp64 reference computes it -- from fp32 arithmetic (fp64 only in rare
// cases).  w = wh + wl + d with wh = RN32(w), wl = RN32(w - wh), |d| <=
// 2^-48 |w|.  a wh = p + e exactly (e by FMA); f = RN32(a wl + e); then
// r = RN32(p + f) and the residual t = (p - r) + f (p - r is exact) place
// a w within about 2^-46 |a w| of r + t.  When |t| stays below half an ulp
// of r by more than 2^-40 |r|, both a w and its double rounding lie strictly
// inside r's rounding interval, so r is the reference value.  When w is
// itself a float (wl = 0, e.g. an integer sqrt(eta)) a w = p + e exactly, its
// double rounding is exact, and r = RN32(p + e) is the reference value ties
// included.  Otherwise (a tie within reach, r a power of two, r tiny or not
// finite) the fp64 product decides.
__device__ __forceinline__ float scale_exact(float a, float wh, float wl, double w) {
  const float p = a * wh;
  const float e = fmaf(a, wh, -p);
  const float f = fmaf(a, wl, e);
  const float r = p + f;
  const float t = (p - r) + f;
  const float ar = fabsf(r);
  const unsigned bits = __float_as_uint(ar);
  const float half_ulp = __uint_as_float((bits & 0x7f800000u) - (24u << 23));
  const bool safe = ar > 0x1p-100f && ar < 0x1p+100f && (bits & 0x007fffffu) != 0u &&
                    fabsf(t) < half_ulp - ar * 0x1p-40f;
  if (safe || a == 0.f || wl == 0.f) return r;
  return (float)((double)a * w);
}

// s + (hi, lo) as a float-float sum (Knuth's two-sum for the high part; the
// low part collects the rounding errors and the exact square remainders).
__device__ __forceinline__ void ff_add_square(float r, float& hi, float& lo) {
  const float sq = r * r;
  const float esq = fmaf(r, r, -sq);
  const float t = hi + sq;
  const float bv = t - hi;
  const float err = (hi - (t - bv)) + (sq - bv);
  hi = t;
  lo += err + esq;
}

__device__ __forceinline__ float4 scale_acc(float4 a, float wh, float wl, double w, float& hi,
                                            float& lo) {
  const float4 x = make_float4(scale_exact(a.x, wh, wl, w), scale_exact(a.y, wh, wl, w),
                               scale_exact(a.z, wh, wl, w), scale_exact(a.w, wh, wl, w));
  ff_add_square(x.x, hi, lo);
  ff_add_square(x.y, hi, lo);
  ff_add_square(x.z, hi, lo);
  ff_add_square(x.w, hi, lo);
  return x;
}
__device__ __forceinline__ double2 scale_acc(double2 a, float, float, double w, double& acc,
                                             double&) {
  const double x = a.x * w, y = a.y * w;
  acc = fma(x, x, fma(y, y, acc));
  return make_double2(x, y);
}

// Division by a value fixed for the launch: shift and mask for powers of two.
struct Div32 {
  unsigned d, shift;
  bool pow2;
  __host__ __device__ Div32(unsigned d_) : d(d_), shift(0), pow2((d_ & (d_ - 1)) == 0) {
    while ((1u << shift) < d_) ++shift;
  }
  __device__ __forceinline__ unsigned div(unsigned x) const { return pow2 ? x >> shift : x / d; }
};

// The gather by 16-byte vectors: column c of slice k of X is X[:, c, k] =
// w[k] A[rep_off[k] + c lda + (0..m-1)].  The vectors of all columns are
// numbered consecutively (column-major), and each thread loads U of them
// (a grid stride apart) before it stores any, so U 16-byte loads per thread
// are in flight; a warp's loads cover consecutive vectors, which are
// consecutive addresses within a column whatever m is.  Used when every
// column starts on a 16-byte boundary (m and lda multiples of the vector
// width, aligned bases) and the item count fits 32 bits; otherwise
// elementwise with the same numbering.  The fp32 scaling is the fp64
// reference's value (scale_exact) and ||X||^2 is summed per thread as a
// float-float pair, so the loop runs on the fp32 pipe; the per-CTA partial
// sums are fp64.
template <typename T, int U>
__device__ __forceinline__ void gather_body(const T* __restrict__ A, int64_t lda,
                                            const int64_t* __restrict__ rep_off,
                                            const double* __restrict__ w,
                                            const float2* __restrict__ wf, int m, int n, int p,
                                            T* __restrict__ X, double* __restrict__ partial,
                                            unsigned bid, unsigned nblk) {
  using V = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::n;
  using Acc = typename std::conditional<std::is_same<T, float>::value, float, double>::type;
  __shared__ double red[32];
  const int64_t total_v = (int64_t)n * p * (m / VN);
  const bool vec_ok = (m % VN == 0) && (lda % VN == 0) &&
                      ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                      ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && total_v < (1ll << 31);
  Acc hi = Acc(0), lo = Acc(0);
  if (vec_ok) {
    const unsigned mv = (unsigned)(m / VN), total = (unsigned)total_v;
    const Div32 dmv(mv), dn((unsigned)n);
    const unsigned stride = nblk * blockDim.x;
    for (unsigned e0 = bid * blockDim.x + threadIdx.x; e0 < total; e0 += stride * U) {
      V v[U];
      int kk[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const unsigned e = e0 + u * stride;
        const unsigned ee = e < total ? e : 0u;
        const unsigned col = dmv.div(ee);
        const unsigned q = ee - col * mv;
        const unsigned k = dn.div(col), c = col - k * (unsigned)n;
        kk[u] = (int)k;
        if (e < total)
          v[u] = __ldg(reinterpret_cast<const V*>(A + rep_off[k] + (int64_t)c * lda +
                                                  (int64_t)q * VN));
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const unsigned e = e0 + u * stride;
        if (e < total) {
          const float2 ws = wf[kk[u]];
          reinterpret_cast<V*>(X)[e] = scale_acc(v[u], ws.x, ws.y, w[kk[u]], hi, lo);
        }
      }
    }
  } else {
    const int64_t total = (int64_t)n * p * m;
    const int64_t stride = (int64_t)nblk * blockDim.x;
    for (int64_t e = bid * (int64_t)blockDim.x + threadIdx.x; e < total; e += stride) {
      const int64_t col = e / m;
      const int r = (int)(e - col * m);
      const int k = (int)(col / n), c = (int)(col - (int64_t)k * n);
      const T a = __ldg(A + rep_off[k] + (int64_t)c * lda + r);
      T x;
      if constexpr (std::is_same<T, float>::value) {
        const float2 ws = wf[k];
        x = scale_exact(a, ws.x, ws.y, w[k]);
        ff_add_square(x, hi, lo);
      } else {
        x = a * w[k];
        hi = fma(x, x, hi);
      }
      X[e] = x;
    }
  }
  double acc = (double)hi + (double)lo;
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partial[bid] = acc;
}

template <typename T, int U>
__global__ void __launch_bounds__(GATHER_THREADS)
gather_vec_kernel(const T* __restrict__ A, int64_t lda, const int64_t* __restrict__ rep_off,
                  const double* __restrict__ w, const float2* __restrict__ wf, int m, int n,
                  int p, T* __restrict__ X, double* __restrict__ partial) {
  gather_body<T, U>(A, lda, rep_off, w, wf, m, n, p, X, partial, blockIdx.x, gridDim.x);
}

// The gathers of many problems in one launch: CTA b works for the problem
// whose CTA range [part0, part0 + nparts) holds it (a binary search over the
// descriptors' part0, which ascend).
template <typename T, int U>
__global__ void __launch_bounds__(GATHER_THREADS)
gather_batched_kernel(const GatherDesc* __restrict__ d, int nprob) {
  int lo = 0, hi = nprob - 1;
  const int b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d[mid].part0 <= b) lo = mid; else hi = mid - 1;
  }
  const GatherDesc g = d[lo];
  gather_body<T, U>(static_cast<const T*>(g.A), g.lda, g.rep_off, g.w,
                    reinterpret_cast<const float2*>(g.wf), g.m, g.n, g.p, static_cast<T*>(g.X),
                    g.partial, (unsigned)(b - g.part0), (unsigned)g.nparts);
}

// ||X_i||^2 of each problem from its partial sums (one CTA per problem).
__global__ void finish_norm_batched_kernel(const GatherDesc* __restrict__ d) {
  __shared__ double red[32];
  const GatherDesc g = d[blockIdx.x];
  double acc = 0.0;
  for (int i = threadIdx.x; i < g.nparts; i += blockDim.x) acc += g.partial[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *g.norm2 = acc;
}

// per-CTA fp64 sums of (X - T)^2
template <typename T>
__global__ void __launch_bounds__(GATHER_THREADS)
residual_kernel(const T* __restrict__ X, const T* __restrict__ Tt, int64_t count,
                double* __restrict__ partial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double d = Tt ? (double)X[e] - (double)Tt[e] : (double)X[e];
    acc = fma(d, d, acc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void finish_norm_kernel(const double* partial, int nparts, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partial[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *out = acc;
}

// ---------------------------------------------------------------------------
// Global truncation (one CTA).  sigma is rc x p, descending per slice.
// Tolerance rule: discard the longest prefix of all values taken in
// ascending order (ties: higher slice first, then higher index) whose energy
// sum stays <= budget.  F(v) = energy of all values <= v is monotone; the
// largest attained value v* with F(v*) <= budget is found by bisection over
// the bit patterns of non-negative doubles, then ties at the next value are
// split in the order above.
// ---------------------------------------------------------------------------
constexpr int TR_THREADS = 1024;

__device__ __forceinline__ int count_greater(const double* s, int rc, double v) {
  // number of leading entries (descending array) strictly greater than v
  int lo = 0, hi = rc;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s[mid] > v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// truncate_block for at most 32 slices, by warp 0 alone: the same sums in
// the same order (a block sum over one busy warp adds only zeros after the
// warp's own butterfly), so the same ranks bit for bit, without the block
// barriers of the 70 bisection passes (the Gram truncations have p = 1).
__device__ __forceinline__ void truncate_warp(const double* __restrict__ sigma, int rc, int p,
                                              const double* normX2, double rel_tol,
                                              int fixed_rank, int* ranks, int* off, double* err2,
                                              int* iscal, double* suf, int energies) {
  const int lane = threadIdx.x & 31;
  const int i = lane;   // this lane's slice (p <= 32)
  const bool own = i < p;
  const double* s = sigma + (int64_t)i * rc;
  double* E = suf + (int64_t)i * (rc + 1);
  if (own) {
    double acc = 0.0;
    E[rc] = 0.0;
    for (int j = rc - 1; j >= 0; --j) {
      acc += energies ? fmax(s[j], 0.0) : s[j] * s[j];
      E[j] = acc;
    }
  }
  __syncwarp();
  if (fixed_rank > 0) {
    double disc = 0.0;
    if (own) {
      const int r = min(fixed_rank, rc);
      ranks[i] = r;
      disc = E[r];
    }
    disc = warp_sum(disc);
    if (lane == 0) *err2 = disc;
  } else {
    const double budget = rel_tol * rel_tol * (*normX2);
    const double mx = warp_max(own ? s[0] : 0.0);
    unsigned long long lo = 0ull, hi = (unsigned long long)__double_as_longlong(mx);
    for (int it = 0; it < 70 && lo < hi; ++it) {
      const unsigned long long mid = lo + (hi - lo + 1) / 2;
      const double v = __longlong_as_double((long long)mid);
      double F = own ? E[count_greater(s, rc, v)] : 0.0;
      F = warp_sum(F);   // identical in every lane
      if (F <= budget) lo = mid; else hi = mid - 1;
    }
    const double vstar = __longlong_as_double((long long)lo);
    double F = 0.0, vnext = INFINITY;
    if (own) {
      const int cg = count_greater(s, rc, vstar);
      ranks[i] = cg;
      F = E[cg];
      if (cg > 0) vnext = s[cg - 1];
    }
    F = warp_sum(F);
    vnext = -warp_max(-vnext);
    __syncwarp();
    if (lane == 0) {
      double disc = F;
      if (isfinite(vnext) && vnext > 0.0) {
        const double e = energies ? vnext : vnext * vnext;
        for (int q = p - 1; q >= 0; --q) {
          const double* sq = sigma + (int64_t)q * rc;
          int r = ranks[q];
          while (r > 0 && sq[r - 1] == vnext && disc + e <= budget) {
            disc += e;
            --r;
          }
          ranks[q] = r;
          if (!(disc + e <= budget)) break;
        }
      }
      *err2 = disc;
    }
  }
  __syncwarp();
  if (lane == 0) {
    int acc = 0, nz = 0;
    for (int q = 0; q < p; ++q) {
      off[q] = acc;
      acc += ranks[q];
      nz += ranks[q] > 0;
    }
    off[p] = acc;
    iscal[0] = acc;
    iscal[1] = nz;
  }
}

__device__ __forceinline__ void truncate_block(const double* __restrict__ sigma, int rc, int p,
                                               const double* normX2, double rel_tol,
                                               int fixed_rank, int* ranks, int* off, double* err2,
                                               int* iscal, double* suf, int energies) {
  if (p <= 32) {   // (block-uniform) one warp does it all
    if (threadIdx.x < 32)
      truncate_warp(sigma, rc, p, normX2, rel_tol, fixed_rank, ranks, off, err2, iscal, suf,
                    energies);
    return;
  }
  __shared__ double red[32];
  __shared__ unsigned long long s_lo, s_hi;
  const int tid = threadIdx.x;
  // suffix energies E_i[j] = sum_{j' >= j} sigma_ij'^2, E_i[rc] = 0
  for (int i = tid; i < p; i += blockDim.x) {
    const double* s = sigma + (int64_t)i * rc;
    double* E = suf + (int64_t)i * (rc + 1);
    double acc = 0.0;
    E[rc] = 0.0;
    for (int j = rc - 1; j >= 0; --j) {
      acc += energies ? fmax(s[j], 0.0) : s[j] * s[j];
      E[j] = acc;
    }
  }
  __syncthreads();
  if (fixed_rank > 0) {
    double disc = 0.0;
    for (int i = tid; i < p; i += blockDim.x) {
      const int r = min(fixed_rank, rc);
      ranks[i] = r;
      disc += suf[(int64_t)i * (rc + 1) + r];
    }
    disc = block_sum(disc, red);
    if (tid == 0) *err2 = disc;
  } else {
    const double budget = rel_tol * rel_tol * (*normX2);
    // largest sigma overall (bisection upper bound)
    double mx = 0.0;
    for (int i = tid; i < p; i += blockDim.x) mx = fmax(mx, sigma[(int64_t)i * rc]);
    __shared__ double smax[32];
    {
      double v = warp_max(mx);
      if ((tid & 31) == 0) smax[tid >> 5] = v;
      __syncthreads();
      if (tid < 32) {
        double t = (tid < (int)(blockDim.x >> 5)) ? smax[tid] : 0.0;
        t = warp_max(t);
        if (tid == 0) smax[0] = t;
      }
      __syncthreads();
      mx = smax[0];
      __syncthreads();
    }
    if (tid == 0) {
      s_lo = 0ull;  // F(0) = 0 <= budget (all sigma >= 0)
      s_hi = (unsigned long long)__double_as_longlong(mx);
    }
    __syncthreads();
    // invariant: F(lo) <= budget; find the largest bits in [lo, hi] with F <= budget
    for (int it = 0; it < 70; ++it) {
      const unsigned long long lo = s_lo, hi = s_hi;
      if (lo >= hi) break;
      const unsigned long long mid = lo + (hi - lo + 1) / 2;
      const double v = __longlong_as_double((long long)mid);
      double F = 0.0;
      for (int i = tid; i < p; i += blockDim.x) {
        const double* s = sigma + (int64_t)i * rc;
        F += suf[(int64_t)i * (rc + 1) + count_greater(s, rc, v)];
      }
      F = block_sum(F, red);
      if (tid == 0) {
        if (F <= budget) s_lo = mid; else s_hi = mid - 1;
      }
      __syncthreads();
    }
    const double vstar = __longlong_as_double((long long)s_lo);
    // ranks before tie handling, F(v*), next larger value
    double F = 0.0, vnext = INFINITY;
    for (int i = tid; i < p; i += blockDim.x) {
      const double* s = sigma + (int64_t)i * rc;
      const int cg = count_greater(s, rc, vstar);
      ranks[i] = cg;
      F += suf[(int64_t)i * (rc + 1) + cg];
      if (cg > 0) vnext = fmin(vnext, s[cg - 1]);
    }
    F = block_sum(F, red);
    {
      double v = -warp_max(-vnext);
      if ((tid & 31) == 0) smax[tid >> 5] = v;
      __syncthreads();
      if (tid < 32) {
        double t = (tid < (int)(blockDim.x >> 5)) ? smax[tid] : INFINITY;
        t = -warp_max(-t);
        if (tid == 0) smax[0] = t;
      }
      __syncthreads();
      vnext = smax[0];
      __syncthreads();
    }
    if (tid == 0) {
      double disc = F;
      if (isfinite(vnext) && vnext > 0.0) {
        // tied values at vnext, split from the highest slice down
        const double e = energies ? vnext : vnext * vnext;
        for (int i = p - 1; i >= 0; --i) {
          const double* s = sigma + (int64_t)i * rc;
          int r = ranks[i];
          while (r > 0 && s[r - 1] == vnext && disc + e <= budget) {
            disc += e;
            --r;
          }
          ranks[i] = r;
          if (!(disc + e <= budget)) break;
        }
      }
      *err2 = disc;
    }
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0, nz = 0;
    for (int i = 0; i < p; ++i) {
      off[i] = acc;
      acc += ranks[i];
      nz += ranks[i] > 0;
    }
    off[p] = acc;
    iscal[0] = acc;
    iscal[1] = nz;
  }
}

__global__ void __launch_bounds__(TR_THREADS)
truncate_kernel(const double* __restrict__ sigma, int rc, int p, const double* normX2,
                double rel_tol, int fixed_rank, int* ranks, int* off, double* err2,
                int* iscal, double* suf, int energies) {
  truncate_block(sigma, rc, p, normX2, rel_tol, fixed_rank, ranks, off, err2, iscal, suf,
                 energies);
}

// one CTA per problem
__global__ void __launch_bounds__(TR_THREADS)
truncate_batched_kernel(const TruncDesc* __restrict__ d, double rel_tol, int fixed_rank) {
  const TruncDesc t = d[blockIdx.x];
  truncate_block(t.sigma, t.rc, t.p, t.normX2, rel_tol, fixed_rank, t.ranks, t.off, t.err2,
                 t.iscal, t.suf, 0);
}

template <typename T>
__global__ void struct_terms_kernel(const int* __restrict__ map, const double* __restrict__ isq,
                                    int ell, int q, const T* __restrict__ coef, int64_t cs_i,
                                    int64_t cs_k, int nterms, const int* nterms_dev,
                                    T* __restrict__ C) {
  const int nt = nterms_dev ? min(nterms, *nterms_dev) : nterms;
  const int64_t per = (int64_t)ell * q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * nterms;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / per);
    const int pos = (int)(e - (int64_t)i * per);
    const int k = map[pos];
    T v = T(0);
    if (i < nt && k >= 0) v = (T)((double)coef[i * cs_i + k * cs_k] * isq[k]);
    C[e] = v;
  }
}

// The same terms written only at the map's nonzero positions nzpos[e] (block
// index k = nzk[e]); the other positions of C stay as the caller zeroed them.
template <typename T>
__global__ void struct_terms_nz_kernel(const int* __restrict__ nzpos, const int* __restrict__ nzk,
                                       int nnz, const double* __restrict__ isq, int ell, int q,
                                       const T* __restrict__ coef, int64_t cs_i, int64_t cs_k,
                                       int nterms, const int* nterms_dev, T* __restrict__ C) {
  const int nt = nterms_dev ? min(nterms, *nterms_dev) : nterms;
  const int64_t per = (int64_t)ell * q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)nnz * nterms;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / nnz);
    const int z = (int)(e - (int64_t)i * nnz);
    const int k = nzk[z];
    const T v = (i < nt) ? (T)((double)coef[i * cs_i + k * cs_k] * isq[k]) : T(0);
    C[(int64_t)i * per + nzpos[z]] = v;
  }
}

template <typename T>
__global__ void scatter_kernel(const int* __restrict__ map, const double* __restrict__ isq,
                               int ell, int q, int m, int n, const T* __restrict__ Tt,
                               T* __restrict__ Ahat, int64_t ld) {
  const int64_t rows = (int64_t)ell * m, cols = (int64_t)q * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / rows, row = e - col * rows;
    const int a = (int)(row / m), r = (int)(row - (int64_t)a * m);
    const int b = (int)(col / n), c = (int)(col - (int64_t)b * n);
    const int k = map[a + ell * b];
    T v = T(0);
    if (k >= 0) v = (T)((double)Tt[r + (int64_t)m * c + (int64_t)m * n * k] * isq[k]);
    Ahat[row + col * ld] = v;
  }
}

template <typename T>
__global__ void orth_kernel(const T* __restrict__ Gm, int rc, const int* __restrict__ ranks,
                            const double* __restrict__ scale, double* out, int use_inv) {
  // G[a, b] / (s_a s_b) - delta_ab with the reciprocals 1 / s_a staged once
  // per slice; the per-element products run in the element type (fp32 on the
  // mixed path, whose factors carry fp32 accuracy; fp64 arithmetic is slow on
  // this part); 0 where s_a = 0 (or below the fp32 range)
  extern __shared__ double inv_raw[];
  T* inv = reinterpret_cast<T*>(inv_raw);
  __shared__ double red[32];
  const int i = blockIdx.x;
  const int r = ranks ? ranks[i] : rc;
  const T* G = Gm + (int64_t)i * rc * rc;
  const double* sc = scale ? scale + (int64_t)i * rc : nullptr;
  const double smin = sizeof(T) == 4 ? 1e-30 : 0.0;
  if (sc && use_inv) {
    for (int a = threadIdx.x; a < r; a += blockDim.x)
      inv[a] = sc[a] > smin ? (T)(1.0 / sc[a]) : T(0);
    __syncthreads();
  }
  T mxt = T(0);
  double mxd = 0.0;
  // rows a along the lanes, columns b over the warps (coalesced, no division)
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int b = threadIdx.x >> 5; b < r; b += nwarp) {
    for (int a = lane; a < r; a += 32) {
      if (sc && use_inv) {
        const T ia = inv[a], ib = inv[b];
        const T g = (ia > T(0) && ib > T(0)) ? G[a + (int64_t)b * rc] * ia * ib
                                             : (a == b ? T(1) : T(0));
        mxt = fmax(mxt, fabs(g - (a == b ? T(1) : T(0))));
      } else {
        double g = (double)G[a + (int64_t)b * rc];
        if (sc) g = (sc[a] > 0 && sc[b] > 0) ? g / (sc[a] * sc[b]) : (a == b ? 1.0 : 0.0);
        mxd = fmax(mxd, fabs(g - (a == b ? 1.0 : 0.0)));
      }
    }
  }
  double mx = fmax(mxd, (double)mxt);
  // block max via shared memory
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    t = warp_max(t);
    if (threadIdx.x == 0) out[i] = t;
  }
}

// The defect of the retained columns straight from the factor: for slice i,
// max over a, b < r_i of |(W^T W)[a, b] / (s_a s_b) - delta_ab| with W the
// K x rc column block of the slice (ld ldw).  One CTA per 64 x 64 tile
// (a-tile <= b-tile) of the leading r_i x r_i block: the two column tiles
// pass through shared memory 32 rows at a time, each thread accumulates a
// 4 x 4 block of the tile in registers (in T: fp32 on the mixed path, as the
// products of the unfused form), and the epilogue scales, takes the largest
// deviation and merges it into out[i] by an integer max on the bits (the
// deviations are non-negative doubles, which order like their bit patterns).
// No Gram is written.  out must be zero on entry.
constexpr int OG_TILE = 64;
constexpr int OG_KC = 32;
constexpr int OG_LD = OG_TILE + 4;   // row stride of a staged tile (16-byte rows)

template <typename T>
__device__ __forceinline__ void og_load4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const double2 q0 = *reinterpret_cast<const double2*>(p);
    const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
    orth_gram_kernel(const T* __restrict__ Wall, int ldw, int64_t w_bs, int K, int rc,
                     const int* __restrict__ ranks, const double* __restrict__ sigma,
                     unsigned long long* __restrict__ out) {
  __shared__ __align__(16) T As[OG_KC][OG_LD];
  __shared__ __align__(16) T Bs[OG_KC][OG_LD];
  __shared__ T inv_a[OG_TILE], inv_b[OG_TILE];
  __shared__ double red[8];
  const int i = blockIdx.y;
  const int r = ranks ? min(max(ranks[i], 0), rc) : rc;
  const int nt = (rc + OG_TILE - 1) / OG_TILE;
  int t = blockIdx.x, ta = 0;
  while (ta < nt && t >= nt - ta) {
    t -= nt - ta;
    ++ta;
  }
  const int tb = ta + t;
  const int a0 = ta * OG_TILE, b0 = tb * OG_TILE;
  if (ta >= nt || b0 >= r) return;   // (uniform over the CTA)
  const T* W = Wall + (int64_t)i * w_bs;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const double smin = sizeof(T) == 4 ? 1e-30 : 0.0;
  if (tid < 2 * OG_TILE) {
    // reciprocal scales in the element type (fp64 arithmetic is slow on this
    // part; the mixed path's factors carry fp32 accuracy)
    const int c = (tid < OG_TILE ? a0 : b0) + (tid & (OG_TILE - 1));
    const T sv = (c < r && sigma) ? (T)sigma[(int64_t)i * rc + c] : T(1);
    const T iv = (c < r) ? (sigma ? (sv > (T)smin ? T(1) / sv : T(0)) : T(1)) : T(0);
    if (tid < OG_TILE) inv_a[tid] = iv;
    else inv_b[tid - OG_TILE] = iv;
  }
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
  // rows k0.. of the two column tiles (32 consecutive rows of a column per
  // 32 consecutive threads), the next chunk loaded into registers while the
  // current one is multiplied
  constexpr int OG_PER = 2 * OG_KC * OG_TILE / 256;
  T pre[OG_PER];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < OG_PER; ++u) {
      const int e = tid + 256 * u;
      const int kk = e % OG_KC, cc = (e / OG_KC) % OG_TILE, which = e / (OG_KC * OG_TILE);
      const int c = (which ? b0 : a0) + cc, row = k0 + kk;
      pre[u] = (c < r && row < K) ? W[row + (int64_t)c * ldw] : T(0);
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < K; k0 += OG_KC) {
    __syncthreads();   // the previous chunk is consumed
#pragma unroll
    for (int u = 0; u < OG_PER; ++u) {
      const int e = tid + 256 * u;
      const int kk = e % OG_KC, cc = (e / OG_KC) % OG_TILE, which = e / (OG_KC * OG_TILE);
      if (which) Bs[kk][cc] = pre[u];
      else As[kk][cc] = pre[u];
    }
    __syncthreads();
    if (k0 + OG_KC < K) fetch(k0 + OG_KC);
#pragma unroll 8
    for (int kk = 0; kk < OG_KC; ++kk) {
      T a[4], b[4];
      og_load4(&As[kk][4 * tx], a);
      og_load4(&Bs[kk][4 * ty], b);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
  }
  // scaled deviations (0 outside the retained block; the identity's entry
  // where a scale is zero or below the working range)
  T mxt = T(0);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int la = 4 * tx + u, lb = 4 * ty + v;
      const int a = a0 + la, b = b0 + lb;
      if (a < r && b < r) {
        const T ia = inv_a[la], ib = inv_b[lb];
        const T dl = (a == b) ? T(1) : T(0);
        const T g = (ia > T(0) && ib > T(0)) ? acc[u][v] * ia * ib : dl;
        mxt = fmax(mxt, fabs(g - dl));
      }
    }
  double mx = warp_max((double)mxt);
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  if (tid < 32) {
    double v = tid < 8 ? red[tid] : 0.0;
    v = warp_max(v);
    if (tid == 0) atomicMax(out + i, (unsigned long long)__double_as_longlong(v));
  }
}

// dst[i0 + n0 (i1 + n1 i2)] = src[i0 s0 + i1 s1 + i2 s2]: an unfolding laid
// out contiguously (one GEMM then forms its Gram instead of one per slice)
__global__ void permute3_kernel(const double* __restrict__ src, int64_t s0, int64_t s1, int64_t s2,
                                int n0, int n1, int n2, double* __restrict__ dst) {
  const int64_t total = (int64_t)n0 * n1 * n2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(e % n0);
    const int64_t r = e / n0;
    const int i1 = (int)(r % n1), i2 = (int)(r / n1);
    dst[e] = src[i0 * s0 + i1 * s1 + i2 * s2];
  }
}

template <typename TD, typename TS>
__global__ void convert_kernel(const TS* __restrict__ s, TD* __restrict__ d, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (TD)s[e];
}

// ---- multilevel (Section 7.2): X[i1 + p1 (i2 + p2 i3)] = w1 w2 w3 a[...] ----
template <typename T>
__global__ void ml_gather_kernel(const T* __restrict__ a, const double* __restrict__ w1,
                                 const double* __restrict__ w2, const double* __restrict__ w3,
                                 int p1, int p2, int p3, T* __restrict__ X,
                                 double* __restrict__ partial) {
  __shared__ double red[32];
  const int64_t total = (int64_t)p1 * p2 * p3;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i1 = (int)(e % p1);
    const int i2 = (int)((e / p1) % p2);
    const int i3 = (int)(e / ((int64_t)p1 * p2));
    const T v = (T)((double)a[e] * (w1[i1] * w2[i2] * w3[i3]));
    X[e] = v;
    acc = fma((double)v, (double)v, acc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// out[a s_a + b s_b + j s_j] = coef[k + p j] / sqrt(eta_k), k = map(a, b)
// (0 where map(a, b) < 0), for j < nterms: struct_E of coefficient columns in
// an arbitrary (stacked / interleaved) layout.
template <typename T>
__global__ void struct_strided_kernel(const int* __restrict__ map, const double* __restrict__ isq,
                                      int ell, int q, const T* __restrict__ coef, int p,
                                      int nterms, int64_t s_a, int64_t s_b, int64_t s_j,
                                      T* __restrict__ out) {
  const int64_t per = (int64_t)ell * q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * nterms;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / per);
    const int pos = (int)(e - (int64_t)j * per);
    const int a = pos % ell, b = pos / ell;
    const int k = map[pos];
    out[a * s_a + b * s_b + j * s_j] = (k >= 0) ? (T)((double)coef[k + (int64_t)p * j] * isq[k]) : T(0);
  }
}

// dense A_hat of a three-level structured matrix (m = n = 1) from the
// approximation tensor T (p1 x p2 x p3): entry ((a1,a2,a3), (b1,b2,b3)),
// row index a3 + l3 (a2 + l2 a1), column b3 + q3 (b2 + q2 b1).
template <typename T>
__global__ void ml_scatter_kernel(MlMaps mp, const T* __restrict__ Tt, T* __restrict__ Ahat,
                                  int64_t ld) {
  const int64_t rows = (int64_t)mp.ell[0] * mp.ell[1] * mp.ell[2];
  const int64_t cols = (int64_t)mp.q[0] * mp.q[1] * mp.q[2];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / rows, row = e - col * rows;
    const int a3 = (int)(row % mp.ell[2]), a2 = (int)((row / mp.ell[2]) % mp.ell[1]),
              a1 = (int)(row / ((int64_t)mp.ell[2] * mp.ell[1]));
    const int b3 = (int)(col % mp.q[2]), b2 = (int)((col / mp.q[2]) % mp.q[1]),
              b1 = (int)(col / ((int64_t)mp.q[2] * mp.q[1]));
    const int k1 = mp.map[0][a1 + mp.ell[0] * b1];
    const int k2 = mp.map[1][a2 + mp.ell[1] * b2];
    const int k3 = mp.map[2][a3 + mp.ell[2] * b3];
    T v = T(0);
    if (k1 >= 0 && k2 >= 0 && k3 >= 0)
      v = (T)((double)Tt[k1 + (int64_t)mp.p[0] * (k2 + (int64_t)mp.p[1] * k3)] * mp.isq[0][k1] *
              mp.isq[1][k2] * mp.isq[2][k3]);
    Ahat[row + col * ld] = v;
  }
}

inline unsigned grid_for(int64_t work, int threads, int64_t cap = 152 * 32) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

int gather_parts(int m, int n, int p) {
  const int64_t total = (int64_t)m * n * p;
  int64_t g = (total + GATHER_THREADS * 4 - 1) / (GATHER_THREADS * 4);
  if (g < 1) g = 1;
  if (g > GATHER_MAX_CTAS) g = GATHER_MAX_CTAS;
  return (int)g;
}

template <typename TS, typename T>
cudaError_t gather(const TS* A, int64_t lda, const int64_t* rep_off, const double* w,
                   const float* wf, int m, int n, int p, T* X, double* partial, cudaStream_t st) {
  const int g = gather_parts(m, n, p);
  static_assert(std::is_same<TS, T>::value, "the gather keeps the input's element type");
  gather_vec_kernel<T, 4><<<g, GATHER_THREADS, 0, st>>>(A, lda, rep_off, w,
                                                         reinterpret_cast<const float2*>(wf), m, n,
                                                         p, X, partial);
  return cudaGetLastError();
}

template <typename T>
cudaError_t gather_batched(const GatherDesc* d, int nprob, int total_parts, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  gather_batched_kernel<T, 4><<<total_parts, GATHER_THREADS, 0, st>>>(d, nprob);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finish_norm_batched_kernel<<<nprob, 256, 0, st>>>(d);
  return cudaGetLastError();
}
template cudaError_t gather_batched<float>(const GatherDesc*, int, int, cudaStream_t);
template cudaError_t gather_batched<double>(const GatherDesc*, int, int, cudaStream_t);

template <typename T>
cudaError_t residual_norm2(const T* X, const T* Tt, int64_t count, double* partial, int nparts,
                           double* out, cudaStream_t st) {
  residual_kernel<T><<<nparts, GATHER_THREADS, 0, st>>>(X, Tt, count, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finish_norm_kernel<<<1, 1024, 0, st>>>(partial, nparts, out);
  return cudaGetLastError();
}
template cudaError_t residual_norm2<float>(const float*, const float*, int64_t, double*, int,
                                           double*, cudaStream_t);
template cudaError_t residual_norm2<double>(const double*, const double*, int64_t, double*, int,
                                            double*, cudaStream_t);

// out[k] = trace of slice k of an m x n x p tensor (fp64 sum over the
// min(m, n) diagonal entries), one warp per slice.
template <typename T>
__global__ void slice_traces_kernel(const T* __restrict__ src, int m, int n, int p,
                                    double* __restrict__ out) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= p) return;
  const int d = m < n ? m : n;
  const T* s = src + (int64_t)warp * m * n;
  double acc = 0.0;
  for (int j = lane; j < d; j += 32) acc += (double)s[j + (int64_t)j * m];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[warp] = acc;
}

// y = a x + b y elementwise (fp64).
__global__ void axpby_kernel(double a, const double* __restrict__ x, double b,
                             double* __restrict__ y, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = fma(a, x[e], b * y[e]);
}

cudaError_t axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  axpby_kernel<<<blocks, 256, 0, st>>>(a, x, b, y, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t slice_traces(const T* src, int m, int n, int p, double* out, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (int)(((int64_t)p * 32 + threads - 1) / threads);
  slice_traces_kernel<T><<<blocks, threads, 0, st>>>(src, m, n, p, out);
  return cudaGetLastError();
}
template cudaError_t slice_traces<float>(const float*, int, int, int, double*, cudaStream_t);
template cudaError_t slice_traces<double>(const double*, int, int, int, double*, cudaStream_t);

__global__ void sum_slabs_kernel(const double* __restrict__ part, int nslab, int64_t count,
                                 double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < nslab; ++s) acc += part[e + s * count];
    out[e] = acc;
  }
}

// Terms of the two-level Kronecker sum: t = j1 + k1 j2 < k1 k2 copies the core
// slice G[:, j1, j2] (mn entries; G is mn x p1 x p2) to Gt[:, t] and writes
// the coefficient vector V[i1 + p1 i2, t] = Y1[i1, j1] Y2[i2, j2]; terms
// t >= k1 k2 (up to p1 p2) are zero; *nterms = k1 k2.  One CTA per term.
template <typename T>
__global__ void ml2_terms_kernel(const T* __restrict__ G, int mn, int p1, int p2,
                                 const T* __restrict__ Y1, const T* __restrict__ Y2,
                                 const int* __restrict__ k1p, const int* __restrict__ k2p,
                                 T* __restrict__ Gt, T* __restrict__ V, int* __restrict__ nterms) {
  const int t = blockIdx.x, p = p1 * p2;
  const int k1 = *k1p, k2 = *k2p;
  const bool live = k1 > 0 && t < k1 * k2;
  const int j1 = live ? t % k1 : 0, j2 = live ? t / k1 : 0;
  const T* g = G + ((int64_t)j1 + (int64_t)p1 * j2) * mn;
  for (int e = threadIdx.x; e < mn; e += blockDim.x) Gt[(int64_t)t * mn + e] = live ? g[e] : T(0);
  for (int k = threadIdx.x; k < p; k += blockDim.x) {
    const int i1 = k % p1, i2 = k / p1;
    V[k + (int64_t)t * p] = live ? Y1[i1 + (int64_t)j1 * p1] * Y2[i2 + (int64_t)j2 * p2] : T(0);
  }
  if (t == 0 && threadIdx.x == 0) *nterms = k1 * k2;
}

// Core step of the three-level matvec: for every column c and a3,
// V[a3 + l3 j12 + l3 k12 c] = sum_j3 G[j12 + k12 j3] U[a3 + l3 j3 + l3 k3 c]
// (j12 < k12, j3 < k3 <= 16); threads run over a3 fastest, so both sides are
// coalesced.  G (k12 x k3) is staged in shared memory.
template <typename T>
__global__ void ml_core_kernel(const T* __restrict__ G, int k12, int k3, const T* __restrict__ U,
                               int l3, int64_t ncol, T* __restrict__ V) {
  extern __shared__ unsigned char sm_raw[];
  T* Gs = reinterpret_cast<T*>(sm_raw);
  for (int e = threadIdx.x; e < k12 * k3; e += blockDim.x) Gs[e] = G[e];
  __syncthreads();
  const int64_t total = (int64_t)l3 * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a3 = (int)(e % l3);
    const int64_t c = e / l3;
    T u[16];
#pragma unroll
    for (int j3 = 0; j3 < 16; ++j3)
      u[j3] = j3 < k3 ? U[a3 + (int64_t)l3 * j3 + (int64_t)l3 * k3 * c] : T(0);
    T* v = V + a3 + (int64_t)l3 * k12 * c;
    for (int j12 = 0; j12 < k12; ++j12) {
      T acc = T(0);
#pragma unroll
      for (int j3 = 0; j3 < 16; ++j3)
        if (j3 < k3) acc = fma(Gs[j12 + k12 * j3], u[j3], acc);
      v[(int64_t)l3 * j12] = acc;
    }
  }
}

template <typename T>
cudaError_t ml_core(const T* G, int k12, int k3, const T* U, int l3, int64_t ncol, T* V,
                    cudaStream_t st) {
  if (k3 < 1 || k3 > 16 || k12 < 1 || l3 < 1) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)l3 * ncol;
  int64_t grid = (total + 255) / 256;
  if (grid > 152 * 32) grid = 152 * 32;
  ml_core_kernel<T><<<(int)grid, 256, (size_t)k12 * k3 * sizeof(T), st>>>(G, k12, k3, U, l3, ncol,
                                                                          V);
  return cudaGetLastError();
}
template cudaError_t ml_core<float>(const float*, int, int, const float*, int, int64_t, float*,
                                    cudaStream_t);
template cudaError_t ml_core<double>(const double*, int, int, const double*, int, int64_t,
                                     double*, cudaStream_t);

// V[:, j] /= sqrt(ev[j]) for j < *r (zero column where ev[j] <= 0).
__global__ void scale_cols_rsqrt_kernel(double* V, int64_t ld, int rows, const double* ev,
                                        const int* r) {
  const int j = blockIdx.x;
  if (j >= *r) return;
  const double e = ev[j];
  const double f = e > 0.0 ? 1.0 / sqrt(e) : 0.0;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) V[i + j * ld] *= f;
}

template <typename T>
cudaError_t ml2_terms(const T* G, int mn, int p1, int p2, const T* Y1, const T* Y2, const int* k1,
                      const int* k2, T* Gt, T* V, int* nterms, cudaStream_t st) {
  const int p = p1 * p2;
  if (p <= 0 || p > 65535 * 1024) return cudaErrorInvalidValue;
  ml2_terms_kernel<T><<<p, 256, 0, st>>>(G, mn, p1, p2, Y1, Y2, k1, k2, Gt, V, nterms);
  return cudaGetLastError();
}
template cudaError_t ml2_terms<float>(const float*, int, int, int, const float*, const float*,
                                      const int*, const int*, float*, float*, int*, cudaStream_t);
template cudaError_t ml2_terms<double>(const double*, int, int, int, const double*, const double*,
                                       const int*, const int*, double*, double*, int*,
                                       cudaStream_t);

cudaError_t scale_cols_rsqrt(double* V, int64_t ld, int rows, const double* ev, const int* r,
                             cudaStream_t st) {
  // one CTA per possible column; columns at or past *r return at once
  const int cols = (int)(ld < 65535 ? ld : 65535);
  scale_cols_rsqrt_kernel<<<cols, 256, 0, st>>>(V, ld, rows, ev, r);
  return cudaGetLastError();
}

cudaError_t sum_slabs(const double* part, int nslab, int64_t count, double* out, cudaStream_t st) {
  int64_t grid = (count + 255) / 256;
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  sum_slabs_kernel<<<(int)grid, 256, 0, st>>>(part, nslab, count, out);
  return cudaGetLastError();
}

cudaError_t finish_norm(const double* partial, int nparts, double* out, cudaStream_t st) {
  finish_norm_kernel<<<1, 1024, 0, st>>>(partial, nparts, out);
  return cudaGetLastError();
}

cudaError_t truncate_ranks_batched(const TruncDesc* d, int nprob, double rel_tol, int fixed_rank,
                                   cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  truncate_batched_kernel<<<nprob, TR_THREADS, 0, st>>>(d, rel_tol, fixed_rank);
  return cudaGetLastError();
}

cudaError_t truncate_ranks(const double* sigma, int rc, int p, const double* normX2,
                           double rel_tol, int fixed_rank, int* ranks, int* off, double* err2,
                           int* iscal, double* scratch, cudaStream_t st, int energies) {
  truncate_kernel<<<1, TR_THREADS, 0, st>>>(sigma, rc, p, normX2, rel_tol, fixed_rank, ranks,
                                            off, err2, iscal, scratch, energies);
  return cudaGetLastError();
}

template <typename T>
cudaError_t build_struct_terms_nz(const int* nzpos, const int* nzk, int nnz, const double* isq,
                                  int ell, int q, const T* coef, int64_t cs_i, int64_t cs_k,
                                  int nterms, const int* nterms_dev, T* C, cudaStream_t st) {
  const int64_t work = (int64_t)nnz * nterms;
  if (work <= 0) return cudaSuccess;
  struct_terms_nz_kernel<T><<<grid_for(work, 256), 256, 0, st>>>(nzpos, nzk, nnz, isq, ell, q,
                                                                   coef, cs_i, cs_k, nterms,
                                                                   nterms_dev, C);
  return cudaGetLastError();
}
template cudaError_t build_struct_terms_nz<float>(const int*, const int*, int, const double*, int,
                                                  int, const float*, int64_t, int64_t, int,
                                                  const int*, float*, cudaStream_t);
template cudaError_t build_struct_terms_nz<double>(const int*, const int*, int, const double*, int,
                                                   int, const double*, int64_t, int64_t, int,
                                                   const int*, double*, cudaStream_t);

template <typename T>
cudaError_t build_struct_terms(const int* map, const double* isq, int ell, int q, const T* coef,
                               int64_t cs_i, int64_t cs_k, int nterms, const int* nterms_dev,
                               T* C, cudaStream_t st) {
  const int64_t work = (int64_t)ell * q * nterms;
  if (work <= 0) return cudaSuccess;
  struct_terms_kernel<T><<<grid_for(work, 256), 256, 0, st>>>(map, isq, ell, q, coef, cs_i,
                                                                cs_k, nterms, nterms_dev, C);
  return cudaGetLastError();
}

template <typename T>
cudaError_t scatter_ME(const int* map, const double* isq, int ell, int q, int m, int n,
                       const T* Tt, T* Ahat, int64_t ld, cudaStream_t st) {
  const int64_t work = (int64_t)ell * m * q * n;
  scatter_kernel<T><<<grid_for(work, 256), 256, 0, st>>>(map, isq, ell, q, m, n, Tt, Ahat, ld);
  return cudaGetLastError();
}

template <typename T>
cudaError_t orth_gram_defect(const T* W, int ldw, int64_t w_bs, int K, int rc, int p,
                             const int* ranks, const double* scale, double* out,
                             cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * (size_t)p, st);
  if (e != cudaSuccess) return e;
  if (rc <= 0) return cudaSuccess;
  const int nt = (rc + OG_TILE - 1) / OG_TILE;
  const dim3 grid(nt * (nt + 1) / 2, p);
  orth_gram_kernel<T><<<grid, 256, 0, st>>>(W, ldw, w_bs, K, rc, ranks, scale,
                                            reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError();
}

template <typename T>
cudaError_t orth_defect(const T* Gm, int rc, int p, const int* ranks, const double* scale,
                        double* out, cudaStream_t st) {
  if (p <= 0) return cudaSuccess;
  const int use_inv = (scale && rc <= 6144) ? 1 : 0;   // reciprocals fit in 48 KB
  orth_kernel<T><<<p, 512, use_inv ? (size_t)rc * sizeof(double) : 0, st>>>(Gm, rc, ranks, scale,
                                                                             out, use_inv);
  return cudaGetLastError();
}

namespace {
// One CTA per slice.  W's and V's discarded columns (and W's retained ones,
// for the defect) are staged in shared memory when they fit; the rebuild
// reads Xhat and writes D once, column by column.
template <typename T>
__global__ void __launch_bounds__(256, 4)
slice_post_kernel(const PostDesc<T>* __restrict__ desc, int m, int n, int mm, int rc, int trans) {
  extern __shared__ __align__(16) unsigned char post_raw[];
  T* Ws = reinterpret_cast<T*>(post_raw);     // mm x rc
  T* Vs = Ws + (size_t)mm * rc;                // rc x rc
  T* inv = Vs + (size_t)rc * rc;               // rc: 1 / sigma_a (0 where sigma_a is 0)
  __shared__ double red[32];
  const PostDesc<T> d = desc[blockIdx.x];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int r = min(max(*d.rank, 0), rc);
  if (sizeof(T) == 4 && (mm * rc) % 4 == 0 && (rc * rc) % 4 == 0) {
    // 16-byte loads (each slice's W and V start on 16-byte boundaries then)
    const float4* w4 = reinterpret_cast<const float4*>(d.W);
    const float4* v4 = reinterpret_cast<const float4*>(d.V);
    float4* ws4 = reinterpret_cast<float4*>(Ws);
    float4* vs4 = reinterpret_cast<float4*>(Vs);
    for (int e = tid; e < (mm * rc) / 4; e += nth) ws4[e] = w4[e];
    for (int e = tid; e < (rc * rc) / 4; e += nth) vs4[e] = v4[e];
  } else {
    for (int e = tid; e < mm * rc; e += nth) Ws[e] = d.W[e];
    for (int e = tid; e < rc * rc; e += nth) Vs[e] = d.V[e];
  }
  const double smin = sizeof(T) == 4 ? 1e-30 : 0.0;
  for (int a = tid; a < r; a += nth) inv[a] = d.sigma[a] > smin ? (T)(1.0 / d.sigma[a]) : T(0);
  __syncthreads();
  // D = Xhat - sum_{j >= r} (left_j)(right_j)^T; left = W (trans: V), right = V (W)
  const T* Lf = trans ? Vs : Ws;
  const T* Rf = trans ? Ws : Vs;
  const int ldl = trans ? rc : mm, ldr = trans ? mm : rc;
  // by 4 x 4 tiles of D (each element's multiply-adds in the same order as
  // one element at a time; 8 shared loads per 16 products)
  const int mt = (m + 3) >> 2, ntl = (n + 3) >> 2;
  for (int e = tid; e < mt * ntl; e += nth) {
    const int i0 = 4 * (e % mt), c0 = 4 * (e / mt);
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        acc[u][v] = (i0 + u < m && c0 + v < n) ? d.Xh[(i0 + u) + (int64_t)m * (c0 + v)] : T(0);
    for (int j = r; j < rc; ++j) {
      T lv[4], rv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        lv[u] = i0 + u < m ? Lf[i0 + u + (int64_t)ldl * j] : T(0);
        rv[u] = c0 + u < n ? Rf[c0 + u + (int64_t)ldr * j] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(-lv[u], rv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (i0 + u < m && c0 + v < n) d.D[(i0 + u) + (int64_t)m * (c0 + v)] = acc[u][v];
  }
  // max |w_a . w_b / (sigma_a sigma_b) - delta_ab| over a <= b < r, by 4 x 4
  // tiles of the Gram (each thread one tile pair at a time: 8 shared loads
  // per 16 products); the scaling by the staged reciprocals in the element
  // type (as orth_kernel)
  T mxt = T(0);
  const int nt = (r + 3) >> 2;
  for (int e = tid; e < nt * nt; e += nth) {
    const int ta = e % nt, tb = e / nt;
    if (ta > tb) continue;
    T g[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) g[u][v] = T(0);
    const int a0 = 4 * ta, b0 = 4 * tb;
    for (int i = 0; i < mm; ++i) {
      T wa[4], wb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        wa[u] = a0 + u < r ? Ws[i + (int64_t)mm * (a0 + u)] : T(0);
        wb[u] = b0 + u < r ? Ws[i + (int64_t)mm * (b0 + u)] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) g[u][v] = fma(wa[u], wb[v], g[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int a = a0 + u, b = b0 + v;
        if (a >= r || b >= r || a > b) continue;
        const T ia = inv[a], ib = inv[b];
        const T gn = (ia > T(0) && ib > T(0)) ? g[u][v] * ia * ib : (a == b ? T(1) : T(0));
        mxt = fmax(mxt, fabs(gn - (a == b ? T(1) : T(0))));
      }
  }
  double mx = warp_max((double)mxt);
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  if (tid < 32) {
    double t = tid < (nth >> 5) ? red[tid] : 0.0;
    t = warp_max(t);
    if (tid == 0) *d.orth = t;
  }
}
}  // namespace

template <typename T>
cudaError_t slice_post(const PostDesc<T>* d, int count, int m, int n, int mm, int rc, int trans,
                       cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = sizeof(T) * ((size_t)mm * rc + (size_t)rc * rc + rc);
  cudaError_t e = cudaFuncSetAttribute(slice_post_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the largest shared-memory carveout, so that several CTAs fit per SM
  e = cudaFuncSetAttribute(slice_post_kernel<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           100);
  if (e != cudaSuccess) return e;
  // about one 4 x 4 tile of the slice per thread: small slices take small CTAs
  int threads = 32;
  while (threads < 256 && threads * 16 < m * n) threads <<= 1;
  slice_post_kernel<T><<<count, threads, smem, st>>>(d, m, n, mm, rc, trans);
  return cudaGetLastError();
}
template cudaError_t slice_post<float>(const PostDesc<float>*, int, int, int, int, int, int,
                                       cudaStream_t);
template cudaError_t slice_post<double>(const PostDesc<double>*, int, int, int, int, int, int,
                                        cudaStream_t);

cudaError_t permute3(const double* src, int64_t s0, int64_t s1, int64_t s2, int n0, int n1, int n2,
                     double* dst, cudaStream_t st) {
  const int64_t work = (int64_t)n0 * n1 * n2;
  if (work <= 0) return cudaSuccess;
  permute3_kernel<<<grid_for(work, 256), 256, 0, st>>>(src, s0, s1, s2, n0, n1, n2, dst);
  return cudaGetLastError();
}

template <typename TD, typename TS>
cudaError_t convert(const TS* src, TD* dst, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  convert_kernel<TD, TS><<<grid_for(count, 256), 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t ml_gather(const T* a, const double* w1, const double* w2, const double* w3, int p1,
                      int p2, int p3, T* X, double* partial, int nparts, cudaStream_t st) {
  ml_gather_kernel<T><<<nparts, GATHER_THREADS, 0, st>>>(a, w1, w2, w3, p1, p2, p3, X, partial);
  return cudaGetLastError();
}
template <typename T>
cudaError_t struct_strided(const int* map, const double* isq, int ell, int q, const T* coef, int p,
                           int nterms, int64_t s_a, int64_t s_b, int64_t s_j, T* out,
                           cudaStream_t st) {
  const int64_t work = (int64_t)ell * q * nterms;
  if (work <= 0) return cudaSuccess;
  struct_strided_kernel<T><<<grid_for(work, 256), 256, 0, st>>>(map, isq, ell, q, coef, p, nterms,
                                                                  s_a, s_b, s_j, out);
  return cudaGetLastError();
}
template <typename T>
cudaError_t ml_scatter(const MlMaps& mp, const T* Tt, T* Ahat, int64_t ld, cudaStream_t st) {
  const int64_t work = (int64_t)mp.ell[0] * mp.ell[1] * mp.ell[2] * mp.q[0] * mp.q[1] * mp.q[2];
  ml_scatter_kernel<T><<<grid_for(work, 256), 256, 0, st>>>(mp, Tt, Ahat, ld);
  return cudaGetLastError();
}
template cudaError_t ml_gather<float>(const float*, const double*, const double*, const double*, int,
                                      int, int, float*, double*, int, cudaStream_t);
template cudaError_t ml_gather<double>(const double*, const double*, const double*, const double*,
                                       int, int, int, double*, double*, int, cudaStream_t);
template cudaError_t struct_strided<float>(const int*, const double*, int, int, const float*, int,
                                           int, int64_t, int64_t, int64_t, float*, cudaStream_t);
template cudaError_t struct_strided<double>(const int*, const double*, int, int, const double*,
                                            int, int, int64_t, int64_t, int64_t, double*,
                                            cudaStream_t);
template cudaError_t ml_scatter<float>(const MlMaps&, const float*, float*, int64_t, cudaStream_t);
template cudaError_t ml_scatter<double>(const MlMaps&, const double*, double*, int64_t,
                                        cudaStream_t);

template cudaError_t gather<double, double>(const double*, int64_t, const int64_t*, const double*,
                                            const float*, int, int, int, double*, double*,
                                            cudaStream_t);
template cudaError_t gather<float, float>(const float*, int64_t, const int64_t*, const double*,
                                          const float*, int, int, int, float*, double*,
                                          cudaStream_t);
template cudaError_t build_struct_terms<float>(const int*, const double*, int, int, const float*,
                                               int64_t, int64_t, int, const int*, float*,
                                               cudaStream_t);
template cudaError_t build_struct_terms<double>(const int*, const double*, int, int,
                                                const double*, int64_t, int64_t, int, const int*,
                                                double*, cudaStream_t);
template cudaError_t scatter_ME<float>(const int*, const double*, int, int, int, int,
                                       const float*, float*, int64_t, cudaStream_t);
template cudaError_t scatter_ME<double>(const int*, const double*, int, int, int, int,
                                        const double*, double*, int64_t, cudaStream_t);
template cudaError_t orth_gram_defect<float>(const float*, int, int64_t, int, int, int,
                                            const int*, const double*, double*, cudaStream_t);
template cudaError_t orth_gram_defect<double>(const double*, int, int64_t, int, int, int,
                                             const int*, const double*, double*, cudaStream_t);
template cudaError_t orth_defect<float>(const float*, int, int, const int*, const double*,
                                        double*, cudaStream_t);
template cudaError_t orth_defect<double>(const double*, int, int, const int*, const double*,
                                         double*, cudaStream_t);
template cudaError_t convert<float, double>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t convert<double, float>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t convert<float, float>(const float*, float*, int64_t, cudaStream_t);
template cudaError_t convert<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace sma
