// QR preconditioning of the per-slice one-sided Jacobi SVD.
//
// One-sided Jacobi converges in markedly fewer sweeps on the transposed
// triangular factor of a column-pivoted QR than on the slice itself (the
// preconditioning of Drmac and Veselic, "New fast and accurate Jacobi SVD
// algorithm", 2008): with  B P = Q1 R1  (B the mm x rc working matrix),
// Jacobi on R1^T gives R1^T = W V^T, hence
//     B = (Q1 V) (P W)^T,
// with the singular values the column norms of W.  qrcp_kernel factors every
// slice (Householder reflectors, LAPACK-style storage: R on and above the
// diagonal, the reflector tails below, tau separately) and writes R1^T as the
// Jacobi input; qr_finish forms P W_d (a row scatter) and Q1 [V_d; 0] for
// the columns d = rho_i..rc-1 that the truncation discards, which is all the
// truncated rebuild  Xhat_i - (Q1 V_d)(P W_d)^T  needs.
//
// A second QR, of R1^T (R1^T P2 = Q2 R2, the Jacobi then run on R2^T =
// W V^T), brings the Jacobi input closer to diagonal again and saves further
// sweeps (the second step of the same preconditioning): then
//     B = (Q1 P2 W)(P Q2 V)^T,
// and the rebuild takes L_d = Q1 [P2 W_d; 0] and Rt_d = P Q2 V_d.  The second
// QR needs no pivoting (P2 = I): qr_blocked_kernel, by panels.
//
// One CTA per slice.  The active columns live in shared memory as far as it
// holds them; pivoting swaps column pointers, never data.  Columns that do not
// fit go to a global overflow; the columns with the largest norms are placed
// there, since the pivoting retires them first.  The partial column norms are
// recomputed exactly after every step from the updated column (it is in
// registers anyway), so no downdating formula is involved.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace sma {
namespace {

constexpr int QR_THREADS = 768;
constexpr int QR_RPL = 8;   // rows per lane held in registers by the column update
static_assert(32 * QR_RPL == kQrWarpRows, "register rebuild covers kQrWarpRows rows");

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <typename T>
__device__ __forceinline__ T load_slice(const T* src, int m, int trans, int r, int c) {
  return trans ? src[c + (int64_t)r * m] : src[r + (int64_t)c * m];
}

// block-wide max of v (NaN ignored); every thread gets it; red holds >= 32
template <typename T>
__device__ __forceinline__ T block_max(T v, T* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < nw ? red[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

// block-wide argmax over nrm[k..rc) (ties: smallest index); all threads get it
template <typename T>
__device__ __forceinline__ int block_argmax(const T* nrm, int k, int rc, T* rv, int* ri) {
  T best = T(-1);
  int bi = k;
  for (int j = k + threadIdx.x; j < rc; j += blockDim.x)
    if (nrm[j] > best) {
      best = nrm[j];
      bi = j;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    rv[w] = best;
    ri[w] = bi;
  }
  __syncthreads();
  if (w == 0) {
    best = threadIdx.x < (unsigned)nw ? rv[threadIdx.x] : T(-1);
    bi = threadIdx.x < (unsigned)nw ? ri[threadIdx.x] : k;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (threadIdx.x == 0) ri[32] = bi;
  }
  __syncthreads();
  return ri[32];
}

// x <- (I - tau v v^T) x on rows k..mm-1 of one column, by one warp (v[k] = 1,
// v zero above k).  With NORM, returns to every lane ||nsc x[k+1..mm)||^2 of
// the updated column (nsc a power of two that keeps the squares in range).
template <typename T, bool NORM>
__device__ __forceinline__ T reflect_col(T* x, const T* v, T tau, int k, int mm, int lane,
                                         T nsc) {
  T a = T(0);
  if (mm - k <= 32 * QR_RPL) {
    T xr[QR_RPL];
    T w = T(0);
#pragma unroll
    for (int i = 0; i < QR_RPL; ++i) {
      const int r = k + lane + 32 * i;
      xr[i] = r < mm ? x[r] : T(0);
    }
#pragma unroll
    for (int i = 0; i < QR_RPL; ++i) {
      const int r = k + lane + 32 * i;
      if (r < mm) w = fma(v[r], xr[i], w);
    }
    w = warp_sum(w);
    const T tw = tau * w;
#pragma unroll
    for (int i = 0; i < QR_RPL; ++i) {
      const int r = k + lane + 32 * i;
      if (r < mm) {
        const T y = fma(-tw, v[r], xr[i]);
        x[r] = y;
        if (NORM && r > k) {
          const T ys = y * nsc;
          a = fma(ys, ys, a);
        }
      }
    }
  } else {
    T w = T(0);
    for (int r = k + lane; r < mm; r += 32) w = fma(v[r], x[r], w);
    w = warp_sum(w);
    const T tw = tau * w;
    for (int r = k + lane; r < mm; r += 32) {
      const T y = fma(-tw, v[r], x[r]);
      x[r] = y;
      if (NORM && r > k) {
        const T ys = y * nsc;
        a = fma(ys, ys, a);
      }
    }
  }
  if (NORM) a = warp_sum(a);
  return a;
}

// block-wide sum of v in T; every thread gets it; red holds >= 32
template <typename T>
__device__ __forceinline__ T block_sum_t(T v, T* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < nw ? red[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[32] = v;
  }
  __syncthreads();
  return red[32];
}

// x_c <- (I - tau v v^T) x_c on rows k..mm-1 for the NC columns with act[c]
// (one warp, interleaved for latency); lane 0 gets the updated row-k entry
// of each column in yk[c].
template <typename T, int NC>
__device__ __forceinline__ void reflect_n(T* const (&x)[NC], const bool (&act)[NC], const T* v,
                                          T tau, int k, int mm, int lane, T (&yk)[NC]) {
  if (mm - k <= 32 * QR_RPL) {
    T xr[NC][QR_RPL];
    T w[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      w[c] = T(0);
#pragma unroll
      for (int i = 0; i < QR_RPL; ++i) {
        const int r = k + lane + 32 * i;
        xr[c][i] = (act[c] && r < mm) ? x[c][r] : T(0);
      }
    }
#pragma unroll
    for (int i = 0; i < QR_RPL; ++i) {
      const int r = k + lane + 32 * i;
      if (r < mm) {
        const T vr = v[r];
#pragma unroll
        for (int c = 0; c < NC; ++c) w[c] = fma(vr, xr[c][i], w[c]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < NC; ++c) w[c] += __shfl_xor_sync(0xffffffffu, w[c], o);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T tw = tau * w[c];
#pragma unroll
      for (int i = 0; i < QR_RPL; ++i) {
        const int r = k + lane + 32 * i;
        if (act[c] && r < mm) {
          const T y = fma(-tw, v[r], xr[c][i]);
          x[c][r] = y;
          if (i == 0) yk[c] = y;
        }
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      T w = T(0);
      for (int r = k + lane; r < mm; r += 32) w = fma(v[r], x[c][r], w);
      w = warp_sum(w);
      const T tw = tau * w;
      for (int r = k + lane; r < mm; r += 32) {
        const T y = fma(-tw, v[r], x[c][r]);
        x[c][r] = y;
        if (r == k) yk[c] = y;
      }
    }
  }
}

// reflect_n for fp32 columns with mm % 4 == 0 and mm <= 4 * 64 rows: lane l
// holds the float4 rows q = k / 4 + l + 32 i (i < 2), so one instruction moves
// four rows.  The rows [4 (k / 4), k) above the reflector are included with
// v = 0 there (the caller clears them), which leaves them unchanged.
template <int NC>
__device__ __forceinline__ void reflect_n4(float* const (&x)[NC], const bool (&act)[NC],
                                           const float* v, float tau, int k, int mm, int lane,
                                           float (&yk)[NC]) {
  const int q0 = k >> 2, mq = mm >> 2;
  const float4* v4 = reinterpret_cast<const float4*>(v);
  float4 xr[NC][2];
  float w[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    w[c] = 0.f;
    const float4* x4 = reinterpret_cast<const float4*>(x[c]);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int q = q0 + lane + 32 * i;
      xr[c][i] = (act[c] && q < mq) ? x4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  float4 vr[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int q = q0 + lane + 32 * i;
    vr[i] = q < mq ? v4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      w[c] = fmaf(vr[i].x, xr[c][i].x, fmaf(vr[i].y, xr[c][i].y,
             fmaf(vr[i].z, xr[c][i].z, fmaf(vr[i].w, xr[c][i].w, w[c]))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] += __shfl_xor_sync(0xffffffffu, w[c], o);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const float tw = tau * w[c];
    float4* x4 = reinterpret_cast<float4*>(x[c]);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int q = q0 + lane + 32 * i;
      if (act[c] && q < mq) {
        const float4 y = make_float4(fmaf(-tw, vr[i].x, xr[c][i].x), fmaf(-tw, vr[i].y, xr[c][i].y),
                                     fmaf(-tw, vr[i].z, xr[c][i].z), fmaf(-tw, vr[i].w, xr[c][i].w));
        x4[q] = y;
        if (i == 0 && lane == 0) {
          const int e = k & 3;
          yk[c] = e == 0 ? y.x : e == 1 ? y.y : e == 2 ? y.z : y.w;
        }
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(QR_THREADS) qrcp_kernel(const QrParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = blockIdx.x;
  const int mm = P.mm, rc = P.rc;
  const int novf = P.plan.novf;
  const size_t colb = align16((size_t)mm * sizeof(T));
  T* nrm = reinterpret_cast<T*>(smem_raw);                            // [rc] (8-byte slots)
  T* nrm0 = reinterpret_cast<T*>(smem_raw + (size_t)rc * 8);          // [rc] (8-byte slots)
  T** colp = reinterpret_cast<T**>(smem_raw + (size_t)rc * 16);       // [rc]
  int* perm = reinterpret_cast<int*>(colp + rc);                      // [rc]
  int* ipos = perm + rc;                                              // [rc]
  int* gpos = ipos + rc;                                              // [novf]
  unsigned char* p1 = smem_raw + align16((size_t)rc * 36);
  T* v = reinterpret_cast<T*>(p1);                                    // [mm]
  unsigned char* slots = p1 + colb;                                   // [nslot][mm]
  __shared__ T rv[32];
  __shared__ int ri[33];
  __shared__ T redt[33];
  __shared__ T sh_nsc;
  __shared__ int sh_nglob, sh_mig_src, sh_mig_pos;
  const T* src = P.src + (int64_t)s * P.src_bs;
  T* F = P.F + (int64_t)s * P.F_bs;
  T* G = P.G + (int64_t)s * P.G_bs;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nth >> 5;

  // The norms that steer the pivoting are kept in T (fp64 arithmetic is far
  // slower than fp32 on this part) for the entries scaled by nsc = 2^-e,
  // 2^(e-1) <= max |B| < 2^e: an orthogonal update keeps every scaled entry
  // below sqrt(mm), so no square overflows.
  T amax = T(0);
  for (int e = tid; e < mm * rc; e += nth) {
    int r, c;
    if (P.trans) { c = e % rc; r = e / rc; } else { r = e % mm; c = e / mm; }
    amax = fmax(amax, fabs(load_slice(src, P.m, P.trans, r, c)));
  }
  amax = block_max(amax, rv);
  if (tid == 0) {
    const int ex = (amax > T(0) && isfinite(amax)) ? min(max(ilogb(amax), -100), 100) : -1;
    sh_nsc = ldexp(T(1), -ex - 1);
  }
  __syncthreads();
  const T nsc = sh_nsc;
  // column norms of B, then the order by descending norm (ties by index)
  for (int c = warp; c < rc; c += nw) {
    T a = T(0);
    for (int r = lane; r < mm; r += 32) {
      const T x = load_slice(src, P.m, P.trans, r, c) * nsc;
      a = fma(x, x, a);
    }
    a = warp_sum(a);
    if (lane == 0) nrm[c] = a;
  }
  __syncthreads();
  // (a NaN norm counts as -1 so that the order stays total and the ranks a
  // permutation)
  for (int c = tid; c < rc; c += nth) {
    const T nc = nrm[c] == nrm[c] ? nrm[c] : T(-1);
    int rk = 0;
    for (int i = 0; i < rc; ++i) {
      const T ni = nrm[i] == nrm[i] ? nrm[i] : T(-1);
      rk += (ni > nc || (ni == nc && i < c)) ? 1 : 0;
    }
    perm[rk] = c;
    ipos[c] = rk;
  }
  // position j starts with the column of rank j; the first novf positions
  // (largest norms) are stored in the overflow
  for (int j = tid; j < rc; j += nth) {
    colp[j] = j < novf ? G + (int64_t)j * mm
                       : reinterpret_cast<T*>(slots + (size_t)(j - novf) * colb);
    if (j < novf) gpos[j] = j;   // overflow column j sits at position j
  }
  if (tid == 0) sh_nglob = novf;
  __syncthreads();
  for (int e = tid; e < mm * rc; e += nth) {
    int r, c;
    if (P.trans) { c = e % rc; r = e / rc; } else { r = e % mm; c = e / mm; }
    colp[ipos[c]][r] = load_slice(src, P.m, P.trans, r, c);
  }
  __syncthreads();
  for (int j = warp; j < rc; j += nw) {
    const T* cj = colp[j];
    T a = T(0);
    for (int r = lane; r < mm; r += 32) {
      const T x = cj[r] * nsc;
      a = fma(x, x, a);
    }
    a = warp_sum(a);
    if (lane == 0) {
      nrm[j] = a;
      nrm0[j] = a;
    }
  }
  __syncthreads();

  // float4 rows for the reflector applications: fp32, columns of a multiple
  // of 4 rows (16-byte aligned in the slots and in the overflow), at most 256
  const bool vec4 = sizeof(T) == 4 && mm % 4 == 0 && mm <= 256;
  for (int k = 0; k < rc; ++k) {
    // pivot: the remaining column with the largest norm
    const int jp = block_argmax(nrm, k, rc, rv, ri);
    const T* cp = colp[jp];
    // Householder reflector of the pivot column's rows k..mm-1: copy to v,
    // squared norm of its tail on the scaled entries
    T s2 = T(0);
    for (int r = k + tid; r < mm; r += nth) {
      const T x = cp[r];
      v[r] = x;
      if (r > k) {
        const T xs = x * nsc;
        s2 = fma(xs, xs, s2);
      }
    }
    s2 = block_sum_t(s2, redt);
    // every thread forms the same scalars (alpha from the column, which this
    // step does not modify): beta = -sign(alpha) ||x[k:]||, tau = (beta -
    // alpha) / beta, tail scale 1 / (alpha - beta)
    const T alpha_s = cp[k] * nsc;
    T tau = T(0), beta = cp[k], scale = T(1);
    if (s2 != T(0)) {
      const T beta_s = -copysign(sqrt(fma(alpha_s, alpha_s, s2)), alpha_s);
      tau = (beta_s - alpha_s) / beta_s;
      beta = beta_s / nsc;
      scale = nsc / (alpha_s - beta_s);
    }
    // retire the pivot column into F column k: R[0..k, k] and the reflector
    T* Fk = F + (int64_t)k * mm;
    for (int r = tid; r < mm; r += nth) {
      T out;
      if (r < k) {
        out = cp[r];
      } else if (r == k) {
        out = beta;
      } else {
        out = v[r] * scale;
        v[r] = out;
      }
      Fk[r] = out;
    }
    if (tid < 4 && (k & ~3) + tid < k) v[(k & ~3) + tid] = T(0);   // rows above k, float4 form
    if (tid == 0) {
      v[k] = T(1);
      P.tau[(int64_t)s * rc + k] = tau;
      if (jp != k) {   // the column at position k moves to position jp
        T t = nrm[k]; nrm[k] = nrm[jp]; nrm[jp] = t;
        t = nrm0[k]; nrm0[k] = nrm0[jp]; nrm0[jp] = t;
        T* tp = colp[k]; colp[k] = colp[jp]; colp[jp] = tp;
        const int pi = perm[k]; perm[k] = perm[jp]; perm[jp] = pi;
        if (sh_nglob > 0 && tp >= G && tp < G + (int64_t)novf * mm)
          gpos[(tp - G) / mm] = jp;
      }
      // Overflow columns move into shared memory as slots free up: the
      // retired pivot's slot takes one remaining overflow column (copied
      // below), or a retired overflow pivot leaves the overflow itself.
      sh_mig_src = -1;
      if (sh_nglob > 0) {
        T* pk = colp[k];
        if (pk >= G && pk < G + (int64_t)novf * mm) {
          gpos[(pk - G) / mm] = -1;
          --sh_nglob;
        } else {
          for (int g = 0; g < novf; ++g)
            if (gpos[g] > k) {
              sh_mig_src = g;
              sh_mig_pos = gpos[g];
              gpos[g] = -1;
              --sh_nglob;
              break;
            }
        }
      }
    }
    __syncthreads();
    if (sh_mig_src >= 0) {   // (block-uniform) copy the column into the freed slot
      const int g = sh_mig_src, pos = sh_mig_pos;
      T* dst = colp[k];
      const T* srcg = G + (int64_t)g * mm;
      for (int r = tid; r < mm; r += nth) dst[r] = srcg[r];
      __syncthreads();
      if (tid == 0) colp[pos] = dst;
      __syncthreads();
    }
    // apply the reflector to the remaining columns, two per warp at a time;
    // downdate their partial norms (n - y_k^2), recomputed exactly when the
    // downdate has lost most of its digits
    for (int j0 = k + 1 + warp; j0 < rc; j0 += 2 * nw) {
      const int j1 = j0 + nw;
      T* const xs[2] = {colp[j0], colp[j1 < rc ? j1 : j0]};
      const bool act[2] = {true, j1 < rc};
      T yk[2] = {T(0), T(0)};
      if constexpr (sizeof(T) == 4) {
        if (vec4) reflect_n4<2>(xs, act, v, tau, k, mm, lane, yk);
        else reflect_n<T, 2>(xs, act, v, tau, k, mm, lane, yk);
      } else {
        reflect_n<T, 2>(xs, act, v, tau, k, mm, lane, yk);
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!act[c]) continue;
        const int j = c ? j1 : j0;
        T nn = T(0);
        int rec = 0;
        if (lane == 0) {
          const T y = yk[c] * nsc;
          nn = nrm[j] - y * y;
          rec = (nn > T(1e-3) * nrm0[j]) ? 0 : 1;
        }
        rec = __shfl_sync(0xffffffffu, rec, 0);
        if (rec) {
          __syncwarp();
          T a = T(0);
          for (int r = k + 1 + lane; r < mm; r += 32) {
            const T z = xs[c][r] * nsc;
            a = fma(z, z, a);
          }
          a = warp_sum(a);
          if (lane == 0) {
            nrm[j] = a;
            nrm0[j] = a;
          }
        } else if (lane == 0) {
          nrm[j] = nn;
        }
      }
    }
    __syncthreads();
  }
  // Jacobi input R1^T (rc x rc, lower triangular); the permutation
  T* J = P.Jin + (int64_t)s * P.J_bs;
  for (int e = tid; e < rc * rc; e += nth) {
    const int r = e % rc, c = e / rc;
    J[r + (int64_t)c * rc] = (c <= r) ? F[c + (int64_t)r * mm] : T(0);
  }
  for (int j = tid; j < rc; j += nth) P.perm[(int64_t)s * rc + j] = perm[j];
}

// Rt = P W (row j of W to row perm[j]) for all columns; L_d = Q1 [V_d; 0]
// for the discarded columns d = ranks[s]..rc-1, the reflectors applied last
// to first with the next reflector fetched while the current one is applied.
// The first fslot of those columns are built in shared memory.
template <typename T>
__global__ void __launch_bounds__(QR_THREADS) qr_finish_kernel(const QrParams<T> P,
                                                                const int* __restrict__ ranks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = blockIdx.x;
  const int mm = P.mm, rc = P.rc;
  const size_t colb = align16((size_t)mm * sizeof(T));
  unsigned char* slots = smem_raw + 2 * colb;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
  const int* perm = P.perm + (int64_t)s * rc;
  const T* W = P.W + (int64_t)s * P.W_bs;        // rc x rc (Jacobi W of R1^T)
  const T* V = P.V + (int64_t)s * P.V_bs;        // rc x rc
  T* Rt = P.Rt + (int64_t)s * P.Rt_bs;           // rc x rc
  T* L = P.L + (int64_t)s * P.L_bs;              // mm x rc
  const T* F = P.F + (int64_t)s * P.F_bs;
  const T* tau = P.tau + (int64_t)s * rc;
  for (int e = tid; e < rc * rc; e += nth) {
    const int j = e % rc, c = e / rc;
    const int pj = perm[j];
    if ((unsigned)pj < (unsigned)rc) Rt[pj + (int64_t)c * rc] = W[j + (int64_t)c * rc];
  }
  const int d0 = ranks ? min(max(ranks[s], 0), rc) : 0;
  const int nd = rc - d0;
  if (nd == 0) return;
  const int fslot = P.plan.fslot;
  auto col = [&](int t) -> T* {
    return t < fslot ? reinterpret_cast<T*>(slots + (size_t)t * colb)
                     : L + (int64_t)(d0 + t) * mm;
  };
  for (int e = tid; e < mm * nd; e += nth) {
    const int r = e % mm, t = e / mm;
    col(t)[r] = (r < rc) ? V[r + (int64_t)(d0 + t) * rc] : T(0);
  }
  {
    const int k = rc - 1;
    T* v0 = reinterpret_cast<T*>(smem_raw);
    for (int r = k + tid; r < mm; r += nth) v0[r] = (r == k) ? T(1) : F[r + (int64_t)k * mm];
  }
  __syncthreads();
  int cur = 0;
  for (int k = rc - 1; k >= 0; --k) {
    const T* vk = reinterpret_cast<const T*>(smem_raw + (size_t)cur * colb);
    if (k > 0) {
      T* nx = reinterpret_cast<T*>(smem_raw + (size_t)(cur ^ 1) * colb);
      const int k1 = k - 1;
      for (int r = k1 + tid; r < mm; r += nth) nx[r] = (r == k1) ? T(1) : F[r + (int64_t)k1 * mm];
    }
    const T tk = tau[k];
    if (tk != T(0))
      for (int t = warp; t < nd; t += nw) reflect_col<T, false>(col(t), vk, tk, k, mm, lane, T(1));
    __syncthreads();
    cur ^= 1;
  }
  const int ns = min(nd, fslot);
  for (int e = tid; e < mm * ns; e += nth) {
    const int r = e % mm, t = e / mm;
    L[r + (int64_t)(d0 + t) * mm] = col(t)[r];
  }
}

// ---- unpivoted blocked Householder QR of an n x n matrix (n <= 256) -------
// The second QR of the two-step preconditioning needs no pivoting (its input
// R1^T already carries the first QR's ordering), so it runs by panels of
// QB_NB columns: warp 0 factors a panel with the panel's columns in
// registers (lane l: rows l + 32 i) and leaves the reflectors in shared
// memory; then every warp applies them to the trailing columns, QB_NC columns
// at a time in registers, their inner products reduced together.  Two block
// barriers per panel instead of several per column.  Same output as
// qrcp_kernel: F = R on and above the diagonal and the reflector tails below
// (ld n), tau, perm = identity, Jin = R^T.
constexpr int QB_NB = 8;
constexpr int QB_NC = 4;
template <typename T> struct QbThreads { static constexpr int v = 512; };
template <> struct QbThreads<double> { static constexpr int v = 256; };

// entry `row` of a register column (lane row % 32, register row / 32),
// broadcast to the warp
template <typename T>
__device__ __forceinline__ T reg_entry(const T (&x)[QR_RPL], int row) {
  const int ir = row >> 5;
  T a = T(0);
#pragma unroll
  for (int i = 0; i < QR_RPL; ++i)
    if (i == ir) a = x[i];
  return __shfl_sync(0xffffffffu, a, row & 31);
}

// Warp sums of 4 values at once (a reduce-scatter: lane l ends with the full
// sum of value 2 b4 + b3 from bits b4 b3 of l; 10 shuffles in all instead of
// 20), returned to every lane in w.
template <typename T>
__device__ __forceinline__ void warp_sum4(T (&w)[4], int lane) {
  const bool h4 = lane & 16, h3 = lane & 8;
  T u2[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const T send = h4 ? w[i] : w[i + 2];
    const T keep = h4 ? w[i + 2] : w[i];
    u2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  T u = (h3 ? u2[1] : u2[0]) + __shfl_xor_sync(0xffffffffu, h3 ? u2[0] : u2[1], 8);
  u += __shfl_xor_sync(0xffffffffu, u, 4);
  u += __shfl_xor_sync(0xffffffffu, u, 2);
  u += __shfl_xor_sync(0xffffffffu, u, 1);
#pragma unroll
  for (int c = 0; c < 4; ++c) w[c] = __shfl_sync(0xffffffffu, u, 16 * (c >> 1) + 8 * (c & 1));
}

template <typename T>
__global__ void __launch_bounds__(QbThreads<T>::v) qr_blocked_kernel(const QrParams<T> P) {
  __shared__ T Vs[QB_NB][kQrWarpRows];
  __shared__ T ts[QB_NB];
  __shared__ T rv[32];
  __shared__ T sh_nsc;
  const int s = blockIdx.x;
  const int n = P.rc;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
  const T* src = P.src + (int64_t)s * P.src_bs;
  T* F = P.F + (int64_t)s * P.F_bs;
  T* tau = P.tau + (int64_t)s * n;
  // F <- the input; power-of-two scale for the norms as in qrcp_kernel
  T amax = T(0);
  for (int e = tid; e < n * n; e += nth) {
    const int r = e % n, c = e / n;
    const T a = src[r + (int64_t)c * P.m];
    F[e] = a;
    amax = fmax(amax, fabs(a));
  }
  amax = block_max(amax, rv);
  if (tid == 0) {
    const int ex = (amax > T(0) && isfinite(amax)) ? min(max(ilogb(amax), -100), 100) : -1;
    sh_nsc = ldexp(T(1), -ex - 1);
  }
  __syncthreads();
  const T nsc = sh_nsc;
  for (int j0 = 0; j0 < n; j0 += QB_NB) {
    const int nb = min(QB_NB, n - j0);
    const int i0 = j0 >> 5;   // register rows below i0 are above the panel: untouched
    if (warp == 0) {
      T x[QB_NB][QR_RPL];
#pragma unroll
      for (int c = 0; c < QB_NB; ++c)
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) {
          const int r = lane + 32 * i;
          x[c][i] = (c < nb && r < n) ? F[r + (int64_t)(j0 + c) * n] : T(0);
        }
#pragma unroll
      for (int jj = 0; jj < QB_NB; ++jj) {
        if (jj >= nb) break;
        const int j = j0 + jj;
        // reflector of column jj, rows j..n-1: beta = -sign(alpha) ||x[j:]||,
        // tau = (beta - alpha) / beta, tail scale 1 / (alpha - beta)
        T s2 = T(0);
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) {
          const int r = lane + 32 * i;
          if (i >= i0 && r > j && r < n) {
            const T xs = x[jj][i] * nsc;
            s2 = fma(xs, xs, s2);
          }
        }
        s2 = warp_sum(s2);
        const T alpha = reg_entry(x[jj], j);
        const T alpha_s = alpha * nsc;
        T tk = T(0), beta = alpha, scale = T(1);
        if (s2 != T(0)) {
          const T beta_s = -copysign(sqrt(fma(alpha_s, alpha_s, s2)), alpha_s);
          tk = (beta_s - alpha_s) / beta_s;
          beta = beta_s / nsc;
          scale = nsc / (alpha_s - beta_s);
        }
        // column jj becomes [R(0..j, j); v tail]; v = e_j + tail
        T v[QR_RPL];
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) {
          const int r = lane + 32 * i;
          T vi = T(0);
          if (r == j) {
            vi = T(1);
            x[jj][i] = beta;
          } else if (r > j && r < n) {
            vi = x[jj][i] * scale;
            x[jj][i] = vi;
          }
          v[i] = vi;
          Vs[jj][r] = vi;
        }
        if (lane == 0) {
          ts[jj] = tk;
          tau[j] = tk;
        }
        // the panel's later columns
        if (tk != T(0)) {
#pragma unroll
          for (int c = jj + 1; c < QB_NB; ++c) {
            if (c >= nb) break;
            T w = T(0);
#pragma unroll
            for (int i = 0; i < QR_RPL; ++i)
              if (i >= i0) w = fma(v[i], x[c][i], w);
            w = warp_sum(w);
            const T tw = tk * w;
#pragma unroll
            for (int i = 0; i < QR_RPL; ++i)
              if (i >= i0) x[c][i] = fma(-tw, v[i], x[c][i]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < QB_NB; ++c)
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) {
          const int r = lane + 32 * i;
          if (c < nb && i >= i0 && r < n) F[r + (int64_t)(j0 + c) * n] = x[c][i];
        }
    }
    __syncthreads();
    // trailing columns j0 + nb .. n-1: the panel's reflectors, first to last
    for (int t0 = j0 + nb + warp * QB_NC; t0 < n; t0 += nw * QB_NC) {
      const int nc = min(QB_NC, n - t0);
      T x[QB_NC][QR_RPL];
#pragma unroll
      for (int c = 0; c < QB_NC; ++c)
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) {
          const int r = lane + 32 * i;
          x[c][i] = (c < nc && i >= i0 && r < n) ? F[r + (int64_t)(t0 + c) * n] : T(0);
        }
#pragma unroll
      for (int jj = 0; jj < QB_NB; ++jj) {
        if (jj >= nb) break;
        const T tk = ts[jj];
        if (tk == T(0)) continue;
        T v[QR_RPL];
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) v[i] = (i >= i0) ? Vs[jj][lane + 32 * i] : T(0);
        T w[QB_NC];
#pragma unroll
        for (int c = 0; c < QB_NC; ++c) {
          T a = T(0);
#pragma unroll
          for (int i = 0; i < QR_RPL; ++i)
            if (i >= i0) a = fma(v[i], x[c][i], a);
          w[c] = a;
        }
        warp_sum4(w, lane);
#pragma unroll
        for (int c = 0; c < QB_NC; ++c) {
          const T tw = tk * w[c];
#pragma unroll
          for (int i = 0; i < QR_RPL; ++i)
            if (i >= i0) x[c][i] = fma(-tw, v[i], x[c][i]);
        }
      }
#pragma unroll
      for (int c = 0; c < QB_NC; ++c)
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) {
          const int r = lane + 32 * i;
          if (c < nc && i >= i0 && r < n) F[r + (int64_t)(t0 + c) * n] = x[c][i];
        }
    }
    __syncthreads();
  }
  // Jacobi input R^T (lower triangular) and the identity permutation
  T* J = P.Jin + (int64_t)s * P.J_bs;
  for (int e = tid; e < n * n; e += nth) {
    const int r = e % n, c = e / n;
    J[r + (int64_t)c * n] = (c <= r) ? F[c + (int64_t)r * n] : T(0);
  }
  for (int j = tid; j < n; j += nth) P.perm[(int64_t)s * n + j] = j;
}

// ---- rebuild with the columns held in registers (mm <= 32 QR_RPL) ---------
// Each warp keeps NC columns in registers (lane l: rows l + 32 i) and applies
// all rc reflectors to them, last to first.  The reflectors are staged in
// shared memory QfChunk (32 fp32, 16 fp64) at a time by the whole CTA (one
// coalesced pass), so each step reads its reflector at shared-memory latency.

constexpr int QF_THREADS = 512;
template <typename T> struct QfChunk { static constexpr int v = 128 / sizeof(T); };

// Warp sums of NC values (NC = 4: the reduce-scatter of warp_sum4).
template <typename T, int NC>
__device__ __forceinline__ void warp_sum_n(T (&w)[NC], int lane) {
  if constexpr (NC == 4) {
    warp_sum4(w, lane);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < NC; ++c) w[c] += __shfl_xor_sync(0xffffffffu, w[c], o);
  }
}

// x_c <- H_0 H_1 ... H_{rc-1} x_c for every warp's NC register columns
// (reflector k: v = e_k + F[k+1..len, k], ld len, scalar tau[k]); `act`
// says whether the warp holds columns.  Called by every thread of the CTA.
template <typename T, int NC>
__device__ __forceinline__ void apply_q_chunked(T (&x)[NC][QR_RPL], bool act,
                                                const T* __restrict__ F,
                                                const T* __restrict__ tau, int rc, int len,
                                                T (*Fs)[kQrWarpRows], T* ts, int lane) {
  constexpr int CH = QfChunk<T>::v;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int khi = rc - 1; khi >= 0; khi -= CH) {
    const int klo = max(khi - CH + 1, 0), nk = khi - klo + 1;
    __syncthreads();   // the previous chunk is consumed
    for (int e = tid; e < nk * kQrWarpRows; e += nth) {
      const int r = e % kQrWarpRows, kk = e / kQrWarpRows, k = klo + kk;
      Fs[kk][r] = (r > k && r < len) ? F[r + (int64_t)k * len] : (r == k ? T(1) : T(0));
    }
    for (int kk = tid; kk < nk; kk += nth) ts[kk] = tau[klo + kk];
    __syncthreads();
    if (!act) continue;
    for (int kk = nk - 1; kk >= 0; --kk) {
      const T tk = ts[kk];
      if (tk == T(0)) continue;
      T v[QR_RPL];
#pragma unroll
      for (int i = 0; i < QR_RPL; ++i) v[i] = Fs[kk][lane + 32 * i];
      T w[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T a = T(0);
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) a = fma(v[i], x[c][i], a);
        w[c] = a;
      }
      warp_sum_n<T, NC>(w, lane);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T tw = tk * w[c];
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) x[c][i] = fma(-tw, v[i], x[c][i]);
      }
    }
  }
}

// The discarded columns d = ranks[s]..rc-1 of the rebuild factors.
//   One QR (TWO = false):  Rt_d = P1 W_d,  L_d = Q1 [V_d; 0].
//   Two QRs (B P1 = Q1 R1, R1^T P2 = Q2 R2, the Jacobi on R2^T giving
//   R2^T = W V^T, hence B = (Q1 P2 W)(P1 Q2 V)^T):
//                          Rt_d = P1 (Q2 V_d),  L_d = Q1 [P2 W_d; 0].
// P carries the first factorisation and the outputs, P2 the second.
template <typename T, int NC, bool TWO>
__global__ void __launch_bounds__(QF_THREADS, 1)
    qr_finish_warp_kernel(const QrParams<T> P, const QrParams<T> P2, const int* __restrict__ ranks) {
  __shared__ T Fs[QfChunk<T>::v][kQrWarpRows];
  __shared__ T ts[QfChunk<T>::v];
  const int s = blockIdx.x;
  const int mm = P.mm, rc = P.rc;
  const int d0 = ranks ? min(max(ranks[s], 0), rc) : 0;
  const int nd = rc - d0;
  if (nd == 0) return;   // (uniform over the CTA)
  const int tid = threadIdx.x, nth = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
  const int* perm1 = P.perm + (int64_t)s * rc;
  const T* W = P.W + (int64_t)s * P.W_bs + (int64_t)d0 * rc;   // rc x nd
  const T* V = P.V + (int64_t)s * P.V_bs + (int64_t)d0 * rc;   // rc x nd
  T* Rt = P.Rt + (int64_t)s * P.Rt_bs + (int64_t)d0 * rc;      // rc x nd
  T* L = P.L + (int64_t)s * P.L_bs + (int64_t)d0 * mm;         // mm x nd
  if (TWO) {
    // L_d <- [P2 W_d; 0]: row j of W_d to row perm2[j]
    const int* perm2 = P2.perm + (int64_t)s * rc;
    for (int64_t e = tid; e < (int64_t)mm * nd; e += nth) {
      const int r = (int)(e % mm), t = (int)(e / mm);
      if (r < rc) {
        const int pj = perm2[r];
        if ((unsigned)pj < (unsigned)rc) L[pj + (int64_t)t * mm] = W[r + (int64_t)t * rc];
      } else {
        L[r + (int64_t)t * mm] = T(0);
      }
    }
    // (the barrier at the top of the first chunk orders these stores before
    // the loads of L below)
  } else {
    // Rt_d <- P1 W_d
    for (int64_t e = tid; e < (int64_t)rc * nd; e += nth) {
      const int j = (int)(e % rc), t = (int)(e / rc);
      const int pj = perm1[j];
      if ((unsigned)pj < (unsigned)rc) Rt[pj + (int64_t)t * rc] = W[j + (int64_t)t * rc];
    }
  }
  if (TWO) {
    // Rt_d <- P1 (Q2 V_d)
    for (int base = 0; base < nd; base += nw * NC) {
      const int t0 = base + warp * NC;
      const int nc = max(0, min(NC, nd - t0));
      T x[NC][QR_RPL];
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) {
          const int r = lane + 32 * i;
          x[c][i] = (c < nc && r < rc) ? V[r + (int64_t)(t0 + c) * rc] : T(0);
        }
      apply_q_chunked<T, NC>(x, nc > 0, P2.F + (int64_t)s * P2.F_bs, P2.tau + (int64_t)s * rc, rc,
                             rc, Fs, ts, lane);
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int i = 0; i < QR_RPL; ++i) {
          const int r = lane + 32 * i;
          if (c < nc && r < rc) {
            const int pr = perm1[r];
            if ((unsigned)pr < (unsigned)rc) Rt[pr + (int64_t)(t0 + c) * rc] = x[c][i];
          }
        }
    }
  }
  // L_d <- Q1 [V_d; 0] (one QR) or Q1 L_d (two QRs, L_d staged above)
  for (int base = 0; base < nd; base += nw * NC) {
    const int t0 = base + warp * NC;
    const int nc = max(0, min(NC, nd - t0));
    T x[NC][QR_RPL];
    if (TWO) __syncthreads();   // the staging of L_d (first pass) or nothing
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int i = 0; i < QR_RPL; ++i) {
        const int r = lane + 32 * i;
        T val = T(0);
        if (c < nc) {
          if (TWO) val = r < mm ? L[r + (int64_t)(t0 + c) * mm] : T(0);
          else val = r < rc ? V[r + (int64_t)(t0 + c) * rc] : T(0);
        }
        x[c][i] = val;
      }
    apply_q_chunked<T, NC>(x, nc > 0, P.F + (int64_t)s * P.F_bs, P.tau + (int64_t)s * rc, rc, mm,
                           Fs, ts, lane);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int i = 0; i < QR_RPL; ++i) {
        const int r = lane + 32 * i;
        if (c < nc && r < mm) L[r + (int64_t)(t0 + c) * mm] = x[c][i];
      }
  }
}

// ---- fp32 slices of at most 256 x 256 with every column resident ----------
// The factorisations above keep the active columns in shared-memory slots
// (and a global overflow) and let any warp update any column, so every step
// goes through column pointers and the generic load/store path.  Here each of
// the QRR_WARPS warps owns a fixed set of columns for the whole
// factorisation: its first QRR_REG slots in registers, the rest in the warp's
// own shared-memory slots; lane l holds the float4 rows l + 32 i of each.
// A step of the column-pivoted QR takes
//   (1) every warp's largest remaining partial norm (kept by lane j for slot
//       j), one block barrier, the same block-wide argmax in every warp: a
//       max over the norms' bit patterns (non-negative floats order like
//       their bits), ties to the lowest warp and slot;
//   (2) the owner of the pivot column forms the Householder reflector (same
//       scalars as qrcp_kernel), writes it to shared memory, retires the
//       column into F (R above the diagonal, beta, the reflector tail) and
//       moves its last active column into the freed slot, so a warp's active
//       columns are always its first slots; one block barrier;
//   (3) every warp applies the reflector to its active columns, four at a
//       time (their inner products reduced together), and downdates their
//       partial norms from the new row-k entries (exact recompute when the
//       downdate has lost most of its digits).
// Without pivoting (the second QR) the pivot of step k is column k, step (1)
// and its barrier drop out, and the reflector buffer alternates between two
// copies, so one barrier per step remains; slot j holds column
// warp + QRR_WARPS (ns - 1 - j), so the columns retire from the last slot
// down and the register slots stay active longest.  Outputs as qrcp_kernel:
// F, tau, perm (position -> column), Jin = R1^T.
constexpr int QRR_THREADS = 512;
constexpr int QRR_WARPS = QRR_THREADS / 32;
constexpr int QRR_SLOTS = 16;   // columns per warp: rc <= QRR_WARPS * QRR_SLOTS
constexpr int QRR_REG = 4;      // of them in registers
constexpr int QRR_MAX = QRR_WARPS * QRR_SLOTS;

__host__ __device__ constexpr int qrr_nq(int mm) { return ((mm + 3) / 4 + 31) / 32; }

size_t qr_res_smem(int mm, int rc) {
  const size_t mq = (size_t)((mm + 3) / 4);
  const int ns = (rc + QRR_SLOTS - 1) / QRR_SLOTS;
  const int nsm = ns > QRR_REG ? ns - QRR_REG : 0;
  return (2 + (size_t)nsm * QRR_WARPS) * mq * sizeof(float4);
}

__device__ __forceinline__ float f4c(const float4& a, int e) {
  return e == 0 ? a.x : e == 1 ? a.y : e == 2 ? a.z : a.w;
}

__device__ __forceinline__ float dot4f(const float4& a, const float4& b, float acc) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
}

__device__ __forceinline__ float4 axpy4(float s, const float4& v, const float4& x) {
  return make_float4(fmaf(s, v.x, x.x), fmaf(s, v.y, x.y), fmaf(s, v.z, x.z), fmaf(s, v.w, x.w));
}

// sum over the rows r > k held by this lane of (nsc x_r)^2
template <int NQ>
__device__ __forceinline__ float tail_sq(const float4 (&x)[NQ], int k, int mm, int lane,
                                         float nsc) {
  float a = 0.f;
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int r0 = 4 * (lane + 32 * i);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + e;
      if (r > k && r < mm) {
        const float z = f4c(x[i], e) * nsc;
        a = fmaf(z, z, a);
      }
    }
  }
  return a;
}

// The reflector of step k applied to four columns, float4 rows from I0 on
// (rows below 128 I0 are zero in v); the lane holding row k stores the
// updated row-k entries to yk[4].
template <int NQ, int I0>
__device__ __forceinline__ void qrr_apply4(float4 (&x)[4][NQ], const float4 (&vr)[NQ], float tk,
                                           int lane, int klane, int ki, int ke, float* yk) {
  float w[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float a = 0.f;
#pragma unroll
    for (int i = I0; i < NQ; ++i) a = dot4f(vr[i], x[c][i], a);
    w[c] = a;
  }
  warp_sum4(w, lane);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float tw = -tk * w[c];
#pragma unroll
    for (int i = I0; i < NQ; ++i) x[c][i] = axpy4(tw, vr[i], x[c][i]);
  }
  if (lane == klane) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float y = 0.f;
#pragma unroll
      for (int i = 0; i < NQ; ++i)
        if (i == ki) y = f4c(x[c][i], ke);
      yk[c] = y;
    }
  }
}

// the block-wide winner of a max over unsigned keys (0: no candidate) held
// one per lane of each warp: ties to the lowest warp, then the lowest lane;
// returns warp * 32 + lane (the lane part in the winning warp only).  One
// block barrier.
__device__ __forceinline__ int qrr_argmax(unsigned key, unsigned* ck, int warp, int lane) {
  const unsigned m = __reduce_max_sync(0xffffffffu, key);
  const unsigned b = __ballot_sync(0xffffffffu, key == m);
  if (lane == 0) ck[warp] = m;
  __syncthreads();
  const unsigned kw = lane < QRR_WARPS ? ck[lane] : 0u;
  const unsigned mw = __reduce_max_sync(0xffffffffu, kw);
  const int ww = __ffs(__ballot_sync(0xffffffffu, kw == mw)) - 1;
  // the lane within warp ww is known to warp ww (its own ballot), the only
  // warp that needs it
  return ww * 32 + ((warp == ww) ? (__ffs(b) - 1) : 0);
}

template <int NQ, bool PIVOT>
__global__ void __launch_bounds__(QRR_THREADS, 1) qr_res_kernel(const QrParams<float> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned ck[QRR_WARPS];
  __shared__ float yk_s[QRR_WARPS][QRR_SLOTS];
  __shared__ float tau_s[2];
  __shared__ float rv[32];
  __shared__ float sh_nsc;
  const int s = blockIdx.x;
  const int mm = P.mm, rc = P.rc, mq = (mm + 3) >> 2;
  const int ns = (rc + QRR_SLOTS - 1) / QRR_SLOTS;   // slots per warp
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float4* vS = reinterpret_cast<float4*>(smem_raw);   // [2][mq] reflectors
  const int sstr = QRR_WARPS * mq;                    // float4s between a warp's slots
  float4* wS = vS + 2 * mq + warp * mq;               // this warp's slot QRR_REG
  const float* src = P.src + (int64_t)s * P.src_bs;
  float* F = P.F + (int64_t)s * P.F_bs;
  float* yk = yk_s[warp];
  auto slot_ptr = [&](int j) { return wS + (j - QRR_REG) * sstr; };
  // the column initially in slot j (>= rc: absent)
  auto col0 = [&](int j) {
    return PIVOT ? warp + QRR_WARPS * j : warp + QRR_WARPS * (ns - 1 - j);
  };

  // load the columns (B[r, c] = slice[r, c], or slice[c, r] when trans)
  float4 xr[QRR_REG][NQ];
#pragma unroll
  for (int j = 0; j < QRR_REG; ++j)
#pragma unroll
    for (int i = 0; i < NQ; ++i) xr[j][i] = make_float4(0.f, 0.f, 0.f, 0.f);
  float amax = 0.f;
  unsigned act = 0;   // active slots (PIVOT: always the first na)
#pragma unroll
  for (int j = 0; j < QRR_SLOTS; ++j) {
    if (j >= ns) break;
    const int c = col0(j);
    const bool have = c < rc;
    if (have) act |= 1u << j;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      const int q = lane + 32 * i;
      float e4[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 4 * q + e;
        e4[e] = (have && r < mm) ? load_slice(src, P.m, P.trans, r, c) : 0.f;
        amax = fmaxf(amax, fabsf(e4[e]));
      }
      const float4 v4 = make_float4(e4[0], e4[1], e4[2], e4[3]);
      if (j < QRR_REG) {
#pragma unroll
        for (int jj = 0; jj < QRR_REG; ++jj)
          if (jj == j) xr[jj][i] = v4;
      } else if (q < mq) {
        slot_ptr(j)[q] = v4;
      }
    }
  }
  amax = block_max(amax, rv);
  if (tid == 0) {
    const int ex = (amax > 0.f && isfinite(amax)) ? min(max(ilogb(amax), -100), 100) : -1;
    sh_nsc = ldexpf(1.f, -ex - 1);
  }
  __syncthreads();
  const float nsc = sh_nsc;
  // lane j: the column in slot j and its scaled squared partial norm
  int mycol = lane < QRR_SLOTS ? col0(lane) : 0;
  float nrm = 0.f, nrm0 = 0.f;
  if (PIVOT) {
#pragma unroll
    for (int j = 0; j < QRR_SLOTS; ++j) {
      if (j >= ns) break;
      float4 x[NQ];
#pragma unroll
      for (int i = 0; i < NQ; ++i) {
        const int q = lane + 32 * i;
        if (j < QRR_REG) {
#pragma unroll
          for (int jj = 0; jj < QRR_REG; ++jj)
            if (jj == j) x[i] = xr[jj][i];
        } else {
          x[i] = q < mq ? slot_ptr(j)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      const float a = warp_sum(tail_sq<NQ>(x, -1, mm, lane, nsc));
      if (lane == j) nrm = nrm0 = a;
    }
  }

  for (int k = 0; k < rc; ++k) {
    const int buf = k & 1;
    float4* vk = vS + buf * mq;
    // (1) the pivot: warp ow, slot oj
    int ow, oj;
    if (PIVOT) {
      const bool mine = (act >> lane) & 1u;   // (lanes >= QRR_SLOTS: 0)
      const unsigned key = mine ? (nrm > 0.f ? __float_as_uint(nrm) + 1u : 1u) : 0u;
      const int wl = qrr_argmax(key, ck, warp, lane);
      ow = wl >> 5;
      oj = wl & 31;   // valid in warp ow only
    } else {
      ow = k % QRR_WARPS;
      oj = ns - 1 - k / QRR_WARPS;
    }
    // (2) its owner forms the reflector and retires the column
    const int klane = (k >> 2) & 31, ki = k >> 7, ke = k & 3;
    if (ow == warp) {
      float4 x[NQ];
#pragma unroll
      for (int i = 0; i < NQ; ++i) {
        const int q = lane + 32 * i;
        if (oj < QRR_REG) {
          x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int jj = 0; jj < QRR_REG; ++jj)
            if (jj == oj) x[i] = xr[jj][i];
        } else {
          x[i] = q < mq ? slot_ptr(oj)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      const float s2 = warp_sum(tail_sq<NQ>(x, k, mm, lane, nsc));
      float al = 0.f;
#pragma unroll
      for (int i = 0; i < NQ; ++i)
        if (i == ki) al = f4c(x[i], ke);
      const float alpha = __shfl_sync(0xffffffffu, al, klane);
      const float alpha_s = alpha * nsc;
      float tk = 0.f, beta = alpha, scale = 1.f;
      if (s2 != 0.f) {
        const float beta_s = -copysignf(sqrtf(fmaf(alpha_s, alpha_s, s2)), alpha_s);
        tk = (beta_s - alpha_s) / beta_s;
        beta = beta_s / nsc;
        scale = nsc / (alpha_s - beta_s);
      }
      float* Fk = F + (int64_t)k * mm;
#pragma unroll
      for (int i = 0; i < NQ; ++i) {
        const int q = lane + 32 * i;
        float vv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = 4 * q + e;
          const float xv = f4c(x[i], e);
          float out, ve;
          if (r < k) {
            out = xv;
            ve = 0.f;
          } else if (r == k) {
            out = beta;
            ve = 1.f;
          } else {
            out = xv * scale;
            ve = out;
          }
          vv[e] = r < mm ? ve : 0.f;
          if (r < mm) Fk[r] = out;
        }
        if (q < mq) vk[q] = make_float4(vv[0], vv[1], vv[2], vv[3]);
      }
      const int pcol = __shfl_sync(0xffffffffu, mycol, oj);
      if (lane == 0) {
        tau_s[buf] = tk;
        P.tau[(int64_t)s * rc + k] = tk;
        P.perm[(int64_t)s * rc + k] = pcol;
      }
      if (PIVOT) {
        // the last active slot e moves into the freed slot oj
        const int e = 31 - __clz(act);
        if (e != oj) {
          float4 t[NQ];
#pragma unroll
          for (int i = 0; i < NQ; ++i) {
            const int q = lane + 32 * i;
            if (e < QRR_REG) {
              t[i] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int jj = 0; jj < QRR_REG; ++jj)
                if (jj == e) t[i] = xr[jj][i];
            } else {
              t[i] = q < mq ? slot_ptr(e)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (oj < QRR_REG) {
#pragma unroll
              for (int jj = 0; jj < QRR_REG; ++jj)
                if (jj == oj) xr[jj][i] = t[i];
            } else if (q < mq) {
              slot_ptr(oj)[q] = t[i];
            }
          }
          const float ne = __shfl_sync(0xffffffffu, nrm, e);
          const float ne0 = __shfl_sync(0xffffffffu, nrm0, e);
          const int ce = __shfl_sync(0xffffffffu, mycol, e);
          if (lane == oj) {
            nrm = ne;
            nrm0 = ne0;
            mycol = ce;
          }
        }
        act &= ~(1u << e);
      } else {
        act &= ~(1u << oj);
      }
    }
    __syncthreads();
    // (3) every warp: the reflector on its active columns
    if (act != 0u) {
      const float tk = tau_s[buf];
      float4 vr[NQ];
#pragma unroll
      for (int i = 0; i < NQ; ++i) {
        const int q = lane + 32 * i;
        vr[i] = q < mq ? vk[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const bool hi_only = NQ == 2 && k >= 128;
#pragma unroll
      for (int g = 0; g < QRR_SLOTS / 4; ++g) {
        if (((act >> (4 * g)) & 0xfu) == 0u) continue;
        float4 x[4][NQ];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int i = 0; i < NQ; ++i) {
            const int j = 4 * g + c, q = lane + 32 * i;
            if (g == 0) x[c][i] = xr[c][i];
            else x[c][i] = (q < mq && (!hi_only || i > 0)) ? slot_ptr(j)[q]
                                                            : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        if (hi_only) qrr_apply4<NQ, (NQ > 1 ? 1 : 0)>(x, vr, tk, lane, klane, ki, ke, yk + 4 * g);
        else qrr_apply4<NQ, 0>(x, vr, tk, lane, klane, ki, ke, yk + 4 * g);
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int i = 0; i < NQ; ++i) {
            const int j = 4 * g + c, q = lane + 32 * i;
            if (g == 0) xr[c][i] = x[c][i];
            else if (q < mq && (!hi_only || i > 0)) slot_ptr(j)[q] = x[c][i];
          }
      }
    }
    if (PIVOT) {
      __syncwarp();
      // partial norms without row k; exact recompute on cancellation
      const bool mine = (act >> lane) & 1u;
      float nn = 0.f;
      bool rec = false;
      if (mine) {
        const float y = yk[lane] * nsc;
        nn = nrm - y * y;
        rec = !(nn > 1e-3f * nrm0);
      }
      const unsigned rm = __ballot_sync(0xffffffffu, rec);
      if (mine && !rec) nrm = nn;
      if (rm != 0u) {
#pragma unroll
        for (int j = 0; j < QRR_SLOTS; ++j) {
          if (!((rm >> j) & 1u)) continue;
          float4 x[NQ];
#pragma unroll
          for (int i = 0; i < NQ; ++i) {
            const int q = lane + 32 * i;
            if (j < QRR_REG) {
#pragma unroll
              for (int jj = 0; jj < QRR_REG; ++jj)
                if (jj == j) x[i] = xr[jj][i];
            } else {
              x[i] = q < mq ? slot_ptr(j)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
          }
          const float a = warp_sum(tail_sq<NQ>(x, k, mm, lane, nsc));
          if (lane == j) nrm = nrm0 = a;
        }
      }
    }
  }
  __syncthreads();
  // Jacobi input R1^T (rc x rc, lower triangular)
  float* J = P.Jin + (int64_t)s * P.J_bs;
  for (int e = tid; e < rc * rc; e += QRR_THREADS) {
    const int r = e % rc, c = e / rc;
    J[r + (int64_t)c * rc] = (c <= r) ? F[c + (int64_t)r * mm] : 0.f;
  }
}

}  // namespace

template <typename T>
QrPlan qr_plan(int mm, int rc, int max_smem) {
  QrPlan q;
  // leave room for the kernels' static shared memory
  max_smem = max_smem > 1024 ? max_smem - 1024 : 0;
  const size_t colb = align16((size_t)mm * sizeof(T));
  const size_t head = align16((size_t)rc * 36) + colb;
  const size_t avail = (size_t)max_smem > head ? (size_t)max_smem - head : 0;
  q.nslot = (int)std::min<size_t>((size_t)rc, avail / colb);
  q.novf = rc - q.nslot;
  q.smem_qr = head + (size_t)q.nslot * colb;
  const size_t fhead = 2 * colb;
  const size_t favail = (size_t)max_smem > fhead ? (size_t)max_smem - fhead : 0;
  q.fslot = (int)std::min<size_t>((size_t)rc, favail / colb);
  q.smem_fin = fhead + (size_t)q.fslot * colb;
  return q;
}

namespace {
bool qr_res_fits(int mm, int rc) {
  if (mm < 1 || rc < 1 || mm > 4 * 32 * 2 || rc > QRR_MAX || rc > mm) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  return qr_res_smem(mm, rc) + 2048 <= (size_t)optin;
}

template <int NQ, bool PIVOT>
cudaError_t qr_res_launch(const QrParams<float>& P, int nslices, cudaStream_t st) {
  const size_t smem = qr_res_smem(P.mm, P.rc);
  cudaError_t e = cudaFuncSetAttribute(qr_res_kernel<NQ, PIVOT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qr_res_kernel<NQ, PIVOT><<<nslices, QRR_THREADS, smem, st>>>(P);
  return cudaGetLastError();
}

template <bool PIVOT>
cudaError_t qr_res(const QrParams<float>& P, int nslices, cudaStream_t st) {
  return qrr_nq(P.mm) == 1 ? qr_res_launch<1, PIVOT>(P, nslices, st)
                           : qr_res_launch<2, PIVOT>(P, nslices, st);
}
}  // namespace

template <typename T>
cudaError_t qrcp(const QrParams<T>& P, int nslices, cudaStream_t st) {
  if (nslices <= 0) return cudaSuccess;
  if constexpr (std::is_same<T, float>::value)
    if (qr_res_fits(P.mm, P.rc)) return qr_res<true>(P, nslices, st);
  if (P.plan.novf > 0 && !P.G) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(qrcp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)P.plan.smem_qr);
  if (e != cudaSuccess) return e;
  qrcp_kernel<T><<<nslices, QR_THREADS, P.plan.smem_qr, st>>>(P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t qr_blocked(const QrParams<T>& P, int nslices, cudaStream_t st) {
  if (nslices <= 0) return cudaSuccess;
  if (P.rc > kQrWarpRows || P.mm != P.rc || P.rc < 1) return cudaErrorInvalidValue;
  if constexpr (std::is_same<T, float>::value)
    if (qr_res_fits(P.mm, P.rc)) return qr_res<false>(P, nslices, st);
  qr_blocked_kernel<T><<<nslices, QbThreads<T>::v, 0, st>>>(P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t qr_finish(const QrParams<T>& P, const QrParams<T>* P2, const int* ranks, int nslices,
                      cudaStream_t st) {
  if (nslices <= 0) return cudaSuccess;
  if (P.mm <= kQrWarpRows) {
    constexpr int NC = sizeof(T) == 4 ? 4 : 2;
    if (P2) {
      if (P2->mm != P.rc || P2->rc != P.rc) return cudaErrorInvalidValue;
      qr_finish_warp_kernel<T, NC, true><<<nslices, QF_THREADS, 0, st>>>(P, *P2, ranks);
    } else {
      qr_finish_warp_kernel<T, NC, false><<<nslices, QF_THREADS, 0, st>>>(P, P, ranks);
    }
    return cudaGetLastError();
  }
  if (P2) return cudaErrorInvalidValue;   // two QRs only with the register form
  cudaError_t e = cudaFuncSetAttribute(qr_finish_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)P.plan.smem_fin);
  if (e != cudaSuccess) return e;
  qr_finish_kernel<T><<<nslices, QR_THREADS, P.plan.smem_fin, st>>>(P, ranks);
  return cudaGetLastError();
}

template QrPlan qr_plan<float>(int, int, int);
template QrPlan qr_plan<double>(int, int, int);
template cudaError_t qrcp<float>(const QrParams<float>&, int, cudaStream_t);
template cudaError_t qrcp<double>(const QrParams<double>&, int, cudaStream_t);
template cudaError_t qr_blocked<float>(const QrParams<float>&, int, cudaStream_t);
template cudaError_t qr_blocked<double>(const QrParams<double>&, int, cudaStream_t);
template cudaError_t qr_finish<float>(const QrParams<float>&, const QrParams<float>*, const int*,
                                      int, cudaStream_t);
template cudaError_t qr_finish<double>(const QrParams<double>&, const QrParams<double>*,
                                       const int*, int, cudaStream_t);

}  // namespace sma
