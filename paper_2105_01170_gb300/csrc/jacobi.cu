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
// Precision.  Dot products, rotation angles and rotations run in T (fp32 on
// the mixed path, fp64 on the fp64 path); on the mixed path the angle and the
// convergence test of nearly parallel columns (|cos| > 0.99) are evaluated in
// fp64; the final column norms are accumulated in fp64.  Rotation (Rutishauser form):
//   zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1/sqrt(1+t^2), s = c t, w_a' = c w_a - s w_b, w_b' = s w_a + c w_b,
// applied when |gamma| > tol sqrt(alpha beta); the caller sets tol (4 sqrt(mm) eps(T)).
#include <algorithm>
#include <vector>

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

// Rotation angle for the pair with squared norms al, be and inner product
// ga; false when the pair is already orthogonal to tolerance.
__device__ __forceinline__ bool angle_fp64(double al, double be, double ga, double tol,
                                           double floor_, double& c, double& s) {
  if (!(fabs(ga) > tol * sqrt(al) * sqrt(be)) || !(fabs(ga) > floor_)) return false;
  const double zeta = (be - al) / (2.0 * ga);
  const double t = (fabs(zeta) > 1e150) ? 0.5 / zeta
                                        : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  c = 1.0 / sqrt(1.0 + t * t);
  s = c * t;
  return true;
}

// fp64 rotation with the tangent taken in fp32: any
// tangent near the optimal one gives an exact (valid) rotation, which leaves
// the pair orthogonal to about fp32 relative accuracy for the next sweep to
// finish, while (c, s) themselves are orthonormal to fp64 accuracy: c =
// 1/sqrt(1 + t^2) from the fp32 estimate refined by two Newton steps in fp64.
// The threshold is tested without square roots; nearly parallel columns
// (|cos| > 0.99) and values outside the fp32 range take the fp64 angle.
__device__ __forceinline__ bool angle_fp64_fast(double al, double be, double ga, double tol,
                                                double floor_, double& c, double& s) {
  const double g2 = ga * ga, ab = al * be;
  if (!(g2 > tol * tol * ab) || !(fabs(ga) > floor_)) return false;
  const double d = be - al;
  const double ad = fabs(d), ag = fabs(ga);
  if (g2 > 0.9801 * ab || ag > 1e30 || ag < 1e-30 || ad > 1e30 || (ad < 1e-30 && ad != 0.0))
    return angle_fp64(al, be, ga, 0.0, 0.0, c, s);
  const float zeta = __fdividef((float)d, 2.0f * (float)ga);
  const float az = fabsf(zeta);
  float tf;
  if (az > 1e18f) {
    tf = __fdividef(0.5f, zeta);
  } else {
    const float q = fmaf(zeta, zeta, 1.0f);
    tf = copysignf(__fdividef(1.0f, az + q * rsqrtf(q)), zeta);
  }
  const double t = (double)tf;
  const double q = fma(t, t, 1.0);
  double r = (double)rsqrtf((float)q);
  r = r * fma(-0.5 * q, r * r, 1.5);
  r = r * fma(-0.5 * q, r * r, 1.5);
  c = r;
  s = r * t;
  return true;
}

template <typename T> struct Angle;
template <> struct Angle<double> {
  static __device__ __forceinline__ bool get(double al, double be, double ga, double tol,
                                             double floor_, double& c, double& s) {
    return angle_fp64_fast(al, be, ga, tol, floor_, c, s);
  }
};
template <> struct Angle<float> {
  // fp32 angle; fp64 for nearly parallel columns (|cos| > 0.99), where the
  // difference of the squared norms loses most of its fp32 digits
  static __device__ __forceinline__ bool get(float al, float be, float ga, float tol,
                                             float floor_, float& c, float& s) {
    const float nrm = sqrtf(al) * sqrtf(be);
    if (!(fabsf(ga) > tol * nrm) || !(fabsf(ga) > floor_)) return false;
    if (fabsf(ga) > 0.99f * nrm) {
      double cd = 1.0, sd = 0.0;
      angle_fp64(al, be, ga, 0.0, 0.0, cd, sd);
      c = (float)cd;
      s = (float)sd;
      return true;
    }
    // t only has to be close to the optimal tangent (any exact rotation is
    // valid), so the divisions are the fast approximate ones
    const float zeta = __fdividef(be - al, 2.0f * ga);
    const float az = fabsf(zeta);
    const float t = (az > 1e18f) ? __fdividef(0.5f, zeta)
                                 : copysignf(__fdividef(1.0f, az + sqrtf(fmaf(zeta, zeta, 1.0f))), zeta);
    // c = 1/sqrt(1 + t^2) to about half an ulp: q = 1 + t^2 as an unevaluated
    // sum (q_hi + q_lo), one Newton step on rsqrt with the residual formed by
    // fused multiply-adds; s = t c.  (The angle t itself may carry fp32
    // rounding -- any exact rotation is valid -- but (c, s) must be as close
    // to orthogonal as fp32 allows, since each column sees thousands of them.)
    const float u_hi = t * t;
    const float u_lo = fmaf(t, t, -u_hi);
    const float q_hi = 1.0f + u_hi;
    const float q_lo = ((u_hi <= 1.0f) ? ((1.0f - q_hi) + u_hi) : ((u_hi - q_hi) + 1.0f)) + u_lo;
    const float r0 = rsqrtf(q_hi);
    const float a_hi = r0 * r0;
    const float a_lo = fmaf(r0, r0, -a_hi);
    const float e = fmaf(-q_hi, a_hi, 1.0f) - fmaf(q_hi, a_lo, q_lo * a_hi);
    c = fmaf(0.5f * r0, e, r0);
    s = c * t;
    return true;
  }
  // The same rotation as (c, t = s / c), for the scaled-rotation form.
  static __device__ __forceinline__ bool get_ct(float al, float be, float ga, float tol,
                                                float floor_, float& c, float& t) {
    // square roots and reciprocals through the approximate hardware
    // functions: the threshold needs no more, and any tangent is a valid
    // rotation as long as c is computed from it accurately (below)
    al = fmaxf(al, 0.f);
    be = fmaxf(be, 0.f);
    const float nrm = (al * rsqrtf(al)) * (be * rsqrtf(be));   // NaN when a norm is 0
    if (!(fabsf(ga) > tol * nrm) || !(fabsf(ga) > floor_)) return false;
    if (fabsf(ga) > 0.99f * nrm) {
      double cd = 1.0, sd = 0.0;
      angle_fp64(al, be, ga, 0.0, 0.0, cd, sd);
      c = (float)cd;
      t = (float)(sd / cd);
      return true;
    }
    const float zeta = __fdividef(be - al, 2.0f * ga);
    const float az = fabsf(zeta);
    if (az > 1e18f) {
      t = __fdividef(0.5f, zeta);
    } else {
      const float q = fmaf(zeta, zeta, 1.0f);
      t = copysignf(__fdividef(1.0f, az + q * rsqrtf(q)), zeta);
    }
    const float u_hi = t * t;
    const float u_lo = fmaf(t, t, -u_hi);
    const float q_hi = 1.0f + u_hi;
    const float q_lo = ((u_hi <= 1.0f) ? ((1.0f - q_hi) + u_hi) : ((u_hi - q_hi) + 1.0f)) + u_lo;
    const float r0 = rsqrtf(q_hi);
    const float a_hi = r0 * r0;
    const float a_lo = fmaf(r0, r0, -a_hi);
    const float e = fmaf(-q_hi, a_hi, 1.0f) - fmaf(q_hi, a_lo, q_lo * a_hi);
    c = fmaf(0.5f * r0, e, r0);
    return true;
  }
};

// Rows per lane kept in registers between the dot products and the rotation.
template <typename T> struct CacheRows { static constexpr int v = 32; };
template <> struct CacheRows<double> { static constexpr int v = 16; };

// Rotate the stacked columns at shared-memory slots a and b (group of g
// lanes; every lane of the warp must call this together).  Dot products over
// rows [0, mm), rotation over rows [0, len).  Returns true if rotated.
// A pair is left alone when it is orthogonal to the relative tolerance tol or
// when its inner product is below floor_ = eps^2 ||W||_F^2, the rounding
// level of the whole slice (columns that are numerically zero).
template <typename T>
__device__ __forceinline__ bool rotate_pair(T* S, int ldS, int a, int b, bool active,
                                            int mm, int len, int lane, int g, T tol, T floor_) {
  constexpr int NR = CacheRows<T>::v;
  T xr[NR], yr[NR];
  T al = T(0), be = T(0), ga = T(0);
  T* x = S + (int64_t)(active ? a : 0) * ldS;
  T* y = S + (int64_t)(active ? b : 0) * ldS;
  if (active) {
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int r = lane + i * g;
      xr[i] = T(0);
      yr[i] = T(0);
      if (r < mm) {
        xr[i] = x[r];
        yr[i] = y[r];
      }
      al = fma(xr[i], xr[i], al);
      be = fma(yr[i], yr[i], be);
      ga = fma(xr[i], yr[i], ga);
    }
    for (int r = lane + NR * g; r < mm; r += g) {
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
  T c, s;
  if (!Angle<T>::get(al, be, ga, tol, floor_, c, s)) return false;
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    const int r = lane + i * g;
    if (r < mm) {
      x[r] = c * xr[i] - s * yr[i];
      y[r] = s * xr[i] + c * yr[i];
    }
  }
  for (int r = lane + NR * g; r < mm; r += g) {
    const T xv = x[r], yv = y[r];
    x[r] = c * xv - s * yv;
    y[r] = s * xv + c * yv;
  }
  for (int r = mm + lane; r < len; r += g) {
    const T xv = x[r], yv = y[r];
    x[r] = c * xv - s * yv;
    y[r] = s * xv + c * yv;
  }
  return true;
}

// float4 form of rotate_pair: lane l handles rows 4q..4q+3 for q = l + i g;
// columns start on 16-byte boundaries (ldS % 4 == 0, mm % 4 == len % 4 == 0).
template <int VEC>
__device__ __forceinline__ bool rotate_pair4(float* S, int ldS, int a, int b, bool active,
                                             int mm, int len, int lane, int g, float tol,
                                             float floor_) {
  constexpr int NQ = CacheRows<float>::v / 4;
  float4 xr[NQ], yr[NQ];
  float al = 0.f, be = 0.f, ga = 0.f;
  float4* x = reinterpret_cast<float4*>(S + (int64_t)(active ? a : 0) * ldS);
  float4* y = reinterpret_cast<float4*>(S + (int64_t)(active ? b : 0) * ldS);
  const int mq = mm >> 2, lq = len >> 2;
  if (active) {
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      const int q = lane + i * g;
      xr[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      yr[i] = xr[i];
      if (q < mq) {
        xr[i] = x[q];
        yr[i] = y[q];
      }
      al = fmaf(xr[i].x, xr[i].x, fmaf(xr[i].y, xr[i].y, fmaf(xr[i].z, xr[i].z, fmaf(xr[i].w, xr[i].w, al))));
      be = fmaf(yr[i].x, yr[i].x, fmaf(yr[i].y, yr[i].y, fmaf(yr[i].z, yr[i].z, fmaf(yr[i].w, yr[i].w, be))));
      ga = fmaf(xr[i].x, yr[i].x, fmaf(xr[i].y, yr[i].y, fmaf(xr[i].z, yr[i].z, fmaf(xr[i].w, yr[i].w, ga))));
    }
    for (int q = lane + NQ * g; q < mq; q += g) {
      const float4 xv = x[q], yv = y[q];
      al = fmaf(xv.x, xv.x, fmaf(xv.y, xv.y, fmaf(xv.z, xv.z, fmaf(xv.w, xv.w, al))));
      be = fmaf(yv.x, yv.x, fmaf(yv.y, yv.y, fmaf(yv.z, yv.z, fmaf(yv.w, yv.w, be))));
      ga = fmaf(xv.x, yv.x, fmaf(xv.y, yv.y, fmaf(xv.z, yv.z, fmaf(xv.w, yv.w, ga))));
    }
  }
  for (int o = g >> 1; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  if (!active) return false;
  float c, sn;
  if (!Angle<float>::get(al, be, ga, tol, floor_, c, sn)) return false;
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int q = lane + i * g;
    if (q < mq) {
      x[q] = make_float4(c * xr[i].x - sn * yr[i].x, c * xr[i].y - sn * yr[i].y,
                         c * xr[i].z - sn * yr[i].z, c * xr[i].w - sn * yr[i].w);
      y[q] = make_float4(sn * xr[i].x + c * yr[i].x, sn * xr[i].y + c * yr[i].y,
                         sn * xr[i].z + c * yr[i].z, sn * xr[i].w + c * yr[i].w);
    }
  }
  for (int q = lane + NQ * g; q < mq; q += g) {
    const float4 xv = x[q], yv = y[q];
    x[q] = make_float4(c * xv.x - sn * yv.x, c * xv.y - sn * yv.y, c * xv.z - sn * yv.z,
                       c * xv.w - sn * yv.w);
    y[q] = make_float4(sn * xv.x + c * yv.x, sn * xv.y + c * yv.y, sn * xv.z + c * yv.z,
                       sn * xv.w + c * yv.w);
  }
  for (int q = mq + lane; q < lq; q += g) {
    const float4 xv = x[q], yv = y[q];
    x[q] = make_float4(c * xv.x - sn * yv.x, c * xv.y - sn * yv.y, c * xv.z - sn * yv.z,
                       c * xv.w - sn * yv.w);
    y[q] = make_float4(sn * xv.x + c * yv.x, sn * xv.y + c * yv.y, sn * xv.z + c * yv.z,
                       sn * xv.w + c * yv.w);
  }
  return true;
}

// One call site for both forms: the float4 form when the layout allows it.
template <typename T, int VEC>
struct Rotator {
  static __device__ __forceinline__ bool run(T* S, int ldS, int a, int b, bool act, int mm,
                                             int len, int lane, int g, T tol, T fl) {
    return rotate_pair(S, ldS, a, b, act, mm, len, lane, g, tol, fl);
  }
};
template <>
struct Rotator<float, 4> {
  static __device__ __forceinline__ bool run(float* S, int ldS, int a, int b, bool act, int mm,
                                             int len, int lane, int g, float tol, float fl) {
    return rotate_pair4<4>(S, ldS, a, b, act, mm, len, lane, g, tol, fl);
  }
};

// ---- register-tiled sweeps (fp32, float4 rows) -----------------------------
// The pair-per-group rotations above move both stacked columns through shared
// memory for every rotation, which makes the sweep bound by shared-memory
// bandwidth.  In the tiled form a warp holds 8 columns in registers (c = 0..3
// tile A, 4..7 tile B; lane l keeps the float4 rows q = l + 32 i of the
// dot-product part, rows < mm) and rotates a group of pairs among them before
// writing them back: INNER = the pairs inside each tile (3 sub-rounds),
// CROSS = all A x B pairs (4 sub-rounds).  A sub-round's 4 pairs are disjoint;
// their 12 dot products are reduced across the warp together (a butterfly
// reduce-scatter), lanes 0..3 each compute one angle, and the rotations are
// applied to the registers and recorded.  The recorded rotations are then
// applied in the same order to the V rows of the 8 columns in one streamed
// pass: the rows of a stacked column are rotated independently and the angles
// depend on the W rows only, so the result is the same sequence of rotations
// as in the untiled form.

// Pair q (0..3) of sub-round r of a group, as register columns (a, b).
template <bool INNER>
__device__ __forceinline__ void tile_pair(int r, int q, int& a, int& b) {
  if (INNER) {
    const int o = (q >> 1) * 4, i = q & 1;
    if (r == 0) {
      a = o + 2 * i;
      b = o + 2 * i + 1;
    } else if (r == 1) {
      a = o + i;
      b = o + i + 2;
    } else {
      a = o + i;
      b = o + 3 - i;
    }
  } else {
    a = q;
    b = 4 + ((q + r) & 3);
  }
}

// Warp sum of 16 values at once: after the four halving exchanges and a final
// one, lane l holds the full sum of value (l >> 1) & 15.
__device__ __forceinline__ float reduce16(const float (&v)[16], int lane) {
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
  float u8[8], u4[4], u2[2];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float send = h4 ? v[i] : v[i + 8];
    const float keep = h4 ? v[i + 8] : v[i];
    u8[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = h3 ? u8[i] : u8[i + 4];
    const float keep = h3 ? u8[i + 4] : u8[i];
    u4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h2 ? u4[i] : u4[i + 2];
    const float keep = h2 ? u4[i + 2] : u4[i];
    u2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const float send = h1 ? u2[0] : u2[1];
  const float keep = h1 ? u2[1] : u2[0];
  float u1 = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  u1 += __shfl_xor_sync(0xffffffffu, u1, 1);
  return u1;
}

__device__ __forceinline__ float dot4(const float4& a, const float4& b, float acc) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
}

// Warp sum of 4 values at once: lane l ends with the full sum of value
// 2 ((l >> 4) & 1) + ((l >> 3) & 1), so value q sits in lane 8 q.
__device__ __forceinline__ float reduce4(const float (&v)[4], int lane) {
  const bool h4 = lane & 16, h3 = lane & 8;
  float u2[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h4 ? v[i] : v[i + 2];
    const float keep = h4 ? v[i + 2] : v[i];
    u2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  const float send = h3 ? u2[0] : u2[1];
  const float keep = h3 ? u2[1] : u2[0];
  float u = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  u += __shfl_xor_sync(0xffffffffu, u, 4);
  u += __shfl_xor_sync(0xffffffffu, u, 2);
  u += __shfl_xor_sync(0xffffffffu, u, 1);
  return u;
}

// One group of rotations on tiles A (slots sa.., na columns) and B (slots
// sb.., nb columns) by one warp; columns past na / nb are absent (zero, never
// rotated).  INNER pairs of A (B) only when doA (doB).  mq = mm / 4 float4
// rows of dot-product part, rq = rc / 4 float4 rows of V part.  csw: the
// warp's shared-memory record of the group (per sub-round four (t1, t2)
// pairs, then the eight column scales).  Returns true if any pair was
// rotated.
//
// The squared column norms are reduced once per group and then updated with
// each rotation (alpha' = alpha - t gamma, beta' = beta + t gamma), so a
// sub-round reduces only its four inner products.  The rotations use the
// scaled form: a column is d times its register copy, and the rotation
// (c, t) of the true columns becomes x_a <- x_a - (t d_b / d_a) x_b,
// x_b <- x_b + (t d_a / d_b) x_a on the copies with d_a, d_b <- c d_a, c d_b
// (two FMAs per row instead of four); the scales are folded back when the
// group ends.  Within a group a column takes at most four rotations with
// |t| <= 1, so d stays in [1/4, 1].
template <int NQW, bool INNER>
__device__ __forceinline__ bool tile_group(float* S, int ldS, int sa, int na, int sb, int nb,
                                           bool doA, bool doB, int mq, int rq, int lane,
                                           float tol, float floor_, float4* csw,
                                           float4* glog = nullptr) {
  constexpr int NR = INNER ? 3 : 4;
  float4 x[8][NQW];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const bool valid = c < 4 ? c < na : (c - 4) < nb;
    const int slot = c < 4 ? sa + c : sb + c - 4;
    const float4* col = reinterpret_cast<const float4*>(S + (int64_t)(valid ? slot : 0) * ldS);
#pragma unroll
    for (int i = 0; i < NQW; ++i) {
      const int qq = lane + 32 * i;
      x[c][i] = (valid && qq < mq) ? col[qq] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  // squared norms of the 8 columns, in every lane
  float nrm8[8];
  {
    float v[16];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float a = 0.f;
#pragma unroll
      for (int i = 0; i < NQW; ++i) a = dot4(x[c][i], x[c][i], a);
      v[c] = a;
      v[8 + c] = 0.f;
    }
    const float red = reduce16(v, lane);
#pragma unroll
    for (int c = 0; c < 8; ++c) nrm8[c] = __shfl_sync(0xffffffffu, red, 2 * c);
  }
  float d[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) d[c] = 1.f;
  unsigned mk[NR];
  unsigned any = 0;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    float g4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int a, b;
      tile_pair<INNER>(r, q, a, b);
      float g = 0.f;
#pragma unroll
      for (int i = 0; i < NQW; ++i) g = dot4(x[a][i], x[b][i], g);
      g4[q] = g;
    }
    const float gr = reduce4(g4, lane);
    // lanes 0..3: the angle of pair q = lane (lanes 4..31 repeat them)
    const int q = lane & 3;
    const float gq = __shfl_sync(0xffffffffu, gr, 8 * q);
    float al = 0.f, be = 0.f, dd = 1.f;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      int a, b;
      tile_pair<INNER>(r, qq, a, b);
      if (q == qq) {
        al = nrm8[a];
        be = nrm8[b];
        dd = d[a] * d[b];
      }
    }
    const float ga = gq * dd;
    const bool allowed = INNER ? (q < 2 ? doA : doB) : true;
    float c = 1.f, t = 0.f;
    const bool ok = allowed && Angle<float>::get_ct(al, be, ga, tol, floor_, c, t);
    if (!ok) {   // an exact identity: t = 0, c = 1
      c = 1.f;
      t = 0.f;
    }
    const unsigned m = __ballot_sync(0xffffffffu, ok) & 0xfu;
    mk[r] = m;
    any |= m;
    if (m == 0u) {
      if (glog && lane == 0) {   // a sub-round of identities
        glog[2 * r] = make_float4(0.f, 0.f, 0.f, 0.f);
        glog[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      continue;
    }
    // all four pairs unconditionally (the ones not rotated are identities),
    // so their independent chains interleave
    float cq[4], tq[4], gt[4], t1[4], t2[4];
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      cq[qq] = __shfl_sync(0xffffffffu, c, qq);
      tq[qq] = __shfl_sync(0xffffffffu, t, qq);
      gt[qq] = __shfl_sync(0xffffffffu, ga, qq);
    }
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      int a, b;
      tile_pair<INNER>(r, qq, a, b);
      t1[qq] = __fdividef(tq[qq] * d[b], d[a]);
      t2[qq] = __fdividef(tq[qq] * d[a], d[b]);
#pragma unroll
      for (int i = 0; i < NQW; ++i) {
        const float4 xa = x[a][i], xb = x[b][i];
        x[a][i] = make_float4(fmaf(-t1[qq], xb.x, xa.x), fmaf(-t1[qq], xb.y, xa.y),
                              fmaf(-t1[qq], xb.z, xa.z), fmaf(-t1[qq], xb.w, xa.w));
        x[b][i] = make_float4(fmaf(t2[qq], xa.x, xb.x), fmaf(t2[qq], xa.y, xb.y),
                              fmaf(t2[qq], xa.z, xb.z), fmaf(t2[qq], xa.w, xb.w));
      }
      d[a] *= cq[qq];
      d[b] *= cq[qq];
      nrm8[a] = fmaf(-tq[qq], gt[qq], nrm8[a]);
      nrm8[b] = fmaf(tq[qq], gt[qq], nrm8[b]);
    }
    if (lane == 0) {
      csw[2 * r] = make_float4(t1[0], t2[0], t1[1], t2[1]);
      csw[2 * r + 1] = make_float4(t1[2], t2[2], t1[3], t2[3]);
      if (glog) {
        glog[2 * r] = csw[2 * r];
        glog[2 * r + 1] = csw[2 * r + 1];
      }
    }
  }
  if (glog && lane == 0) {
    // the record: per sub-round the (t1, t2) of its four pairs (identities
    // past NR), then the eight column scales
#pragma unroll
    for (int r = NR; r < 4; ++r) {
      glog[2 * r] = make_float4(0.f, 0.f, 0.f, 0.f);
      glog[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!any) {
      glog[8] = make_float4(1.f, 1.f, 1.f, 1.f);
      glog[9] = make_float4(1.f, 1.f, 1.f, 1.f);
    } else {
      glog[8] = make_float4(d[0], d[1], d[2], d[3]);
      glog[9] = make_float4(d[4], d[5], d[6], d[7]);
    }
  }
  if (!any) return false;
  // fold the scales back and store
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const bool valid = c < 4 ? c < na : (c - 4) < nb;
    if (!valid) continue;
    float4* col = reinterpret_cast<float4*>(S + (int64_t)(c < 4 ? sa + c : sb + c - 4) * ldS);
    const float dc = d[c];
#pragma unroll
    for (int i = 0; i < NQW; ++i) {
      const int qq = lane + 32 * i;
      const float4 v = x[c][i];
      if (qq < mq) col[qq] = make_float4(dc * v.x, dc * v.y, dc * v.z, dc * v.w);
    }
  }
  if (lane == 0) {
    csw[2 * NR] = make_float4(d[0], d[1], d[2], d[3]);
    csw[2 * NR + 1] = make_float4(d[4], d[5], d[6], d[7]);
  }
  __syncwarp();
  // V rows: the same scaled rotations, then the scales
  const float4 d03 = csw[2 * NR], d47 = csw[2 * NR + 1];
  for (int qq = lane; qq < rq; qq += 32) {
    float4 y[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const bool valid = c < 4 ? c < na : (c - 4) < nb;
      const float4* col =
          reinterpret_cast<const float4*>(S + (int64_t)(c < 4 ? sa + c : sb + c - 4) * ldS);
      y[c] = valid ? col[mq + qq] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (mk[r] == 0u) continue;
      const float4 r01 = csw[2 * r], r23 = csw[2 * r + 1];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int a, b;
        tile_pair<INNER>(r, q, a, b);
        const float ta = q == 0 ? r01.x : q == 1 ? r01.z : q == 2 ? r23.x : r23.z;
        const float tb = q == 0 ? r01.y : q == 1 ? r01.w : q == 2 ? r23.y : r23.w;
        const float4 ya = y[a], yb = y[b];
        y[a] = make_float4(fmaf(-ta, yb.x, ya.x), fmaf(-ta, yb.y, ya.y), fmaf(-ta, yb.z, ya.z),
                           fmaf(-ta, yb.w, ya.w));
        y[b] = make_float4(fmaf(tb, ya.x, yb.x), fmaf(tb, ya.y, yb.y), fmaf(tb, ya.z, yb.z),
                           fmaf(tb, ya.w, yb.w));
      }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const bool valid = c < 4 ? c < na : (c - 4) < nb;
      if (!valid) continue;
      float4* col = reinterpret_cast<float4*>(S + (int64_t)(c < 4 ? sa + c : sb + c - 4) * ldS);
      const float dc = c == 0 ? d03.x : c == 1 ? d03.y : c == 2 ? d03.z : c == 3 ? d03.w
                     : c == 4 ? d47.x : c == 5 ? d47.y : c == 6 ? d47.z : d47.w;
      const float4 v = y[c];
      col[mq + qq] = make_float4(dc * v.x, dc * v.y, dc * v.z, dc * v.w);
    }
  }
  __syncwarp();   // the record is rewritten by the warp's next group
  return true;
}

// ---- register-tiled sweeps on part of a warp (short columns) ---------------
// When the dot-product part has at most 4 GW rows (GW = 16, 8 or 4), a task
// needs only GW lanes: lane gl of a group keeps float4 row gl of each of the
// task's 8 columns, and the warp runs 32 / GW tasks side by side, one per
// group of GW lanes.  The tasks of one warp are independent (disjoint tiles
// of the same round), so they share every instruction: reductions are
// shuffles within the group, every branch is taken on the warp-wide OR of
// the groups' conditions, and a group with nothing to do in a sub-round (or
// no task at all, live == false) applies exact identities (t = 0, c = 1).
// The rotations, their order and their arithmetic are those of tile_group.

// Sum of 4 values over a group of GW lanes (GW >= 4): lane gl ends with the
// group sum of value 2 [gl & GW/2] + [gl & GW/4].
template <int GW>
__device__ __forceinline__ float reduce4_group(const float (&v)[4], int gl) {
  const bool h4 = gl & (GW / 2), h3 = gl & (GW / 4);
  float u2[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h4 ? v[i] : v[i + 2];
    const float keep = h4 ? v[i + 2] : v[i];
    u2[i] = keep + __shfl_xor_sync(0xffffffffu, send, GW / 2);
  }
  const float send = h3 ? u2[0] : u2[1];
  const float keep = h3 ? u2[1] : u2[0];
  float u = keep + __shfl_xor_sync(0xffffffffu, send, GW / 4);
#pragma unroll
  for (int o = GW / 8; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
  return u;
}

template <int GW, int NQW, bool INNER>
__device__ __forceinline__ bool tile_group_part(float* S, int ldS, int sa, int na, int sb, int nb,
                                                bool doA, bool doB, int mq, int rq, int gl,
                                                int grp, bool live, float tol, float floor_,
                                                float4* csw) {
  constexpr int NR = INNER ? 3 : 4;
  if (!live) na = nb = 0;
  float4 x[8][NQW];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const bool valid = c < 4 ? c < na : (c - 4) < nb;
    const int slot = c < 4 ? sa + c : sb + c - 4;
    const float4* col = reinterpret_cast<const float4*>(S + (int64_t)(valid ? slot : 0) * ldS);
#pragma unroll
    for (int i = 0; i < NQW; ++i) {
      const int qq = gl + GW * i;
      x[c][i] = (valid && qq < mq) ? col[qq] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  // squared norms of the 8 columns, in every lane of the group
  float nrm8[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float a = 0.f;
#pragma unroll
    for (int i = 0; i < NQW; ++i) a = dot4(x[c][i], x[c][i], a);
#pragma unroll
    for (int o = GW / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    nrm8[c] = a;
  }
  float d[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) d[c] = 1.f;
  unsigned mk[NR];
  unsigned anyg = 0, anyw = 0;
  const int gbase = grp * GW;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    float g4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int a, b;
      tile_pair<INNER>(r, q, a, b);
      float g = 0.f;
#pragma unroll
      for (int i = 0; i < NQW; ++i) g = dot4(x[a][i], x[b][i], g);
      g4[q] = g;
    }
    const float gr = reduce4_group<GW>(g4, gl);
    // lanes 0..3 of the group: the angle of pair q = gl (the others repeat them)
    const int q = gl & 3;
    const float gq = __shfl_sync(0xffffffffu, gr, (q >> 1) * (GW / 2) + (q & 1) * (GW / 4), GW);
    float al = 0.f, be = 0.f, dd = 1.f;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      int a, b;
      tile_pair<INNER>(r, qq, a, b);
      if (q == qq) {
        al = nrm8[a];
        be = nrm8[b];
        dd = d[a] * d[b];
      }
    }
    const float ga = gq * dd;
    const bool allowed = live && (INNER ? (q < 2 ? doA : doB) : true);
    float c = 1.f, t = 0.f;
    const bool ok = allowed && Angle<float>::get_ct(al, be, ga, tol, floor_, c, t);
    if (!ok) {
      c = 1.f;
      t = 0.f;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ok && gl < 4);
    const unsigned m = (bal >> gbase) & 0xfu;
    mk[r] = m;
    anyg |= m;
    anyw |= bal;
    if (bal == 0u) continue;   // warp-uniform
    float cq[4], tq[4], gt[4], t1[4], t2[4];
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      cq[qq] = __shfl_sync(0xffffffffu, c, qq, GW);
      tq[qq] = __shfl_sync(0xffffffffu, t, qq, GW);
      gt[qq] = __shfl_sync(0xffffffffu, ga, qq, GW);
    }
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      int a, b;
      tile_pair<INNER>(r, qq, a, b);
      t1[qq] = __fdividef(tq[qq] * d[b], d[a]);
      t2[qq] = __fdividef(tq[qq] * d[a], d[b]);
#pragma unroll
      for (int i = 0; i < NQW; ++i) {
        const float4 xa = x[a][i], xb = x[b][i];
        x[a][i] = make_float4(fmaf(-t1[qq], xb.x, xa.x), fmaf(-t1[qq], xb.y, xa.y),
                              fmaf(-t1[qq], xb.z, xa.z), fmaf(-t1[qq], xb.w, xa.w));
        x[b][i] = make_float4(fmaf(t2[qq], xa.x, xb.x), fmaf(t2[qq], xa.y, xb.y),
                              fmaf(t2[qq], xa.z, xb.z), fmaf(t2[qq], xa.w, xb.w));
      }
      d[a] *= cq[qq];
      d[b] *= cq[qq];
      nrm8[a] = fmaf(-tq[qq], gt[qq], nrm8[a]);
      nrm8[b] = fmaf(tq[qq], gt[qq], nrm8[b]);
    }
    if (gl == 0) {
      csw[2 * r] = make_float4(t1[0], t2[0], t1[1], t2[1]);
      csw[2 * r + 1] = make_float4(t1[2], t2[2], t1[3], t2[3]);
    }
  }
  if (anyw == 0u) return false;   // warp-uniform
  if (anyg) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const bool valid = c < 4 ? c < na : (c - 4) < nb;
      if (!valid) continue;
      float4* col = reinterpret_cast<float4*>(S + (int64_t)(c < 4 ? sa + c : sb + c - 4) * ldS);
      const float dc = d[c];
#pragma unroll
      for (int i = 0; i < NQW; ++i) {
        const int qq = gl + GW * i;
        const float4 v = x[c][i];
        if (qq < mq) col[qq] = make_float4(dc * v.x, dc * v.y, dc * v.z, dc * v.w);
      }
    }
    if (gl == 0) {
      csw[2 * NR] = make_float4(d[0], d[1], d[2], d[3]);
      csw[2 * NR + 1] = make_float4(d[4], d[5], d[6], d[7]);
    }
  }
  __syncwarp();
  if (anyg) {
    const float4 d03 = csw[2 * NR], d47 = csw[2 * NR + 1];
    for (int qq = gl; qq < rq; qq += GW) {
      float4 y[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const bool valid = c < 4 ? c < na : (c - 4) < nb;
        const float4* col =
            reinterpret_cast<const float4*>(S + (int64_t)(c < 4 ? sa + c : sb + c - 4) * ldS);
        y[c] = valid ? col[mq + qq] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (mk[r] == 0u) continue;
        const float4 r01 = csw[2 * r], r23 = csw[2 * r + 1];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int a, b;
          tile_pair<INNER>(r, q, a, b);
          const float ta = q == 0 ? r01.x : q == 1 ? r01.z : q == 2 ? r23.x : r23.z;
          const float tb = q == 0 ? r01.y : q == 1 ? r01.w : q == 2 ? r23.y : r23.w;
          const float4 ya = y[a], yb = y[b];
          y[a] = make_float4(fmaf(-ta, yb.x, ya.x), fmaf(-ta, yb.y, ya.y), fmaf(-ta, yb.z, ya.z),
                             fmaf(-ta, yb.w, ya.w));
          y[b] = make_float4(fmaf(tb, ya.x, yb.x), fmaf(tb, ya.y, yb.y), fmaf(tb, ya.z, yb.z),
                             fmaf(tb, ya.w, yb.w));
        }
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const bool valid = c < 4 ? c < na : (c - 4) < nb;
        if (!valid) continue;
        float4* col = reinterpret_cast<float4*>(S + (int64_t)(c < 4 ? sa + c : sb + c - 4) * ldS);
        const float dc = c == 0 ? d03.x : c == 1 ? d03.y : c == 2 ? d03.z : c == 3 ? d03.w
                       : c == 4 ? d47.x : c == 5 ? d47.y : c == 6 ? d47.z : d47.w;
        const float4 v = y[c];
        col[mq + qq] = make_float4(dc * v.x, dc * v.y, dc * v.z, dc * v.w);
      }
    }
  }
  __syncwarp();   // the record is rewritten by the group's next task
  return anyg != 0u;
}

// columns of tile t of a block of ncols columns (0 when t is past the end)
__device__ __forceinline__ int tile_cols(int t, int ncols) {
  const int r = ncols - 4 * t;
  return r <= 0 ? 0 : (r < 4 ? r : 4);
}

template <typename T>
__device__ __forceinline__ T load_work(const T* src, int m, int trans, int mm, int r, int c) {
  // stacked column c: rows [0, mm) the working matrix (the slice, m x n with
  // ld m, or its transpose), rows [mm, mm + rc) the identity (V_0 = I)
  if (r >= mm) return (r - mm == c) ? T(1) : T(0);
  return trans ? src[c + (int64_t)r * m] : src[r + (int64_t)c * m];
}

// Pair k of round t of one phase (the work between two stagings).
//   kind 0: round robin over the bI columns in shared memory (cI = bI even-up);
//   kind 1: first nri rounds: round robin inside block I (slots [0, bI), cI
//           players, 0 = skip) and independently inside block J (slots
//           [bc, bc + bJ), cJ players, 0 = skip); then bc rounds of cross
//           pairs I x J: slot k with slot bc + (k + t') % bc.
struct Phase {
  int kind, bI, bJ, bc, cI, cJ, nri, npairs, nrounds;
};

__device__ __forceinline__ bool phase_pair(const Phase& ph, int t, int k, int& a, int& b) {
  if (ph.kind == 0) {
    if (k >= ph.cI / 2) return false;
    const Pair pr = rr_pair(k, t, ph.cI);
    a = pr.a;
    b = pr.b;
    return pr.a < ph.bI && pr.b < ph.bI;
  }
  if (t < ph.nri) {
    const int pI = ph.cI / 2;
    if (k < pI) {
      if (t >= ph.cI - 1) return false;
      const Pair pr = rr_pair(k, t, ph.cI);
      a = pr.a;
      b = pr.b;
      return pr.a < ph.bI && pr.b < ph.bI;
    }
    if (k >= pI + ph.cJ / 2 || t >= ph.cJ - 1) return false;
    const Pair pr = rr_pair(k - pI, t, ph.cJ);
    a = ph.bc + pr.a;
    b = ph.bc + pr.b;
    return pr.a < ph.bJ && pr.b < ph.bJ;
  }
  if (k >= ph.bc) return false;
  const int j = (k + t - ph.nri) % ph.bc;
  a = k;
  b = ph.bc + j;
  return k < ph.bI && j < ph.bJ;
}

// Copy ncols columns of `rows` elements between shared memory (stride ldS)
// and the global workspace (stride ldg); float4 when VEC == 4.  Element e
// always goes to the same thread, so a copy out of a slot region followed by
// a copy into it needs no barrier in between.
template <typename T, int VEC>
__device__ __forceinline__ void copy_cols(T* S, int ldS, T* G, int ldg, int rows, int ncols,
                                          int tid, int nth, bool to_smem) {
  if (VEC == 4) {
    const int rq = rows >> 2;
    for (int e = tid; e < rq * ncols; e += nth) {
      const int r = e % rq, c = e / rq;
      float4* s4 = reinterpret_cast<float4*>(S + (int64_t)c * ldS) + r;
      float4* g4 = reinterpret_cast<float4*>(G + (int64_t)c * ldg) + r;
      if (to_smem) *s4 = *g4;
      else *g4 = *s4;
    }
  } else {
    for (int e = tid; e < rows * ncols; e += nth) {
      const int r = e % rows, c = e / rows;
      if (to_smem) S[(int64_t)c * ldS + r] = G[(int64_t)c * ldg + r];
      else G[(int64_t)c * ldg + r] = S[(int64_t)c * ldS + r];
    }
  }
}

// Rounds of the tiled sweep.  kind 0 (all rc columns in shared memory): a
// round robin over the ntp tile players, ntp - 1 rounds of ntp / 2 tasks, the
// pairs inside each tile in round 0.  kind 1 (blocks I, J staged in slots
// [0, bc) and [bc, 2 bc)): on a block's first visit of the sweep nri rounds of
// round robin inside the block(s) (cI / 2 + cJ / 2 tasks), then btc rounds of
// the cross pairs, tile k of I with tile (k + t) mod btc of J (btI tasks).
struct TPhase {
  int kind, ntp, bI, bJ, bc, btI, btJ, cI, cJ, nri, btc;
};
struct TTask {
  int sa, na, sb, nb;
  bool inner;
};
__device__ __forceinline__ TPhase tphase_smem(int rc) {
  TPhase p{};
  const int nt = (rc + 3) >> 2;
  p.kind = 0;
  p.ntp = nt + (nt & 1);
  p.bI = rc;
  return p;
}
__device__ __forceinline__ TPhase tphase_blocks(int bI, int bJ, int bc, bool doI, bool doJ) {
  TPhase p{};
  p.kind = 1;
  p.bI = bI;
  p.bJ = bJ;
  p.bc = bc;
  p.btI = (bI + 3) >> 2;
  p.btJ = (bJ + 3) >> 2;
  p.cI = doI ? p.btI + (p.btI & 1) : 0;
  p.cJ = doJ ? p.btJ + (p.btJ & 1) : 0;
  p.nri = (doI || doJ) ? max(p.cI, p.cJ) - 1 : 0;
  p.btc = max(p.btI, p.btJ);
  return p;
}
__device__ __forceinline__ int tphase_rounds(const TPhase& p) {
  return p.kind == 0 ? p.ntp - 1 : p.nri + p.btc;
}
__device__ __forceinline__ int tphase_tasks(const TPhase& p, int t) {
  if (p.kind == 0) return p.ntp / 2;
  return t < p.nri ? p.cI / 2 + p.cJ / 2 : p.btI;
}
__device__ __forceinline__ bool tphase_task(const TPhase& p, int t, int k, TTask& d) {
  if (p.kind == 0) {
    const Pair pr = rr_pair(k, t, p.ntp);
    d.sa = 4 * pr.a;
    d.sb = 4 * pr.b;
    d.na = tile_cols(pr.a, p.bI);
    d.nb = tile_cols(pr.b, p.bI);
    d.inner = (t == 0);
    return true;
  }
  if (t < p.nri) {
    int base, nc, cc, kk;
    if (k < p.cI / 2) {
      base = 0; nc = p.bI; cc = p.cI; kk = k;
    } else {
      base = p.bc; nc = p.bJ; cc = p.cJ; kk = k - p.cI / 2;
    }
    if (t >= cc - 1) return false;
    const Pair pr = rr_pair(kk, t, cc);
    d.sa = base + 4 * pr.a;
    d.sb = base + 4 * pr.b;
    d.na = tile_cols(pr.a, nc);
    d.nb = tile_cols(pr.b, nc);
    d.inner = (t == 0);
    return true;
  }
  const int jt = (k + t - p.nri) % p.btc;
  if (jt >= p.btJ) return false;
  d.sa = 4 * k;
  d.na = tile_cols(k, p.bI);
  d.sb = p.bc + 4 * jt;
  d.nb = tile_cols(jt, p.bJ);
  d.inner = false;
  return true;
}

// Block pair of phase ps of a tiled sweep over nb blocks.  The sweep opens
// with the matching (0,1), (2,3), ... in which both blocks also rotate their
// inner pairs (all tasks of those rounds busy), then visits the remaining
// pairs in lexicographic order with cross pairs only; for odd nb the last
// block's inner pairs go with its first visit, (0, nb - 1).
__device__ __forceinline__ void tile_phase_ij(int ps, int nb, int& I, int& J, bool& doI,
                                              bool& doJ) {
  const int nm = nb / 2;
  if (ps < nm) {
    I = 2 * ps;
    J = I + 1;
    doI = doJ = true;
    return;
  }
  int idx = ps - nm;
  for (int a = 0; a < nb; ++a)
    for (int b = a + 1; b < nb; ++b) {
      if ((a & 1) == 0 && b == a + 1) continue;   // a matching pair
      if (idx-- == 0) {
        I = a;
        J = b;
        doI = false;
        doJ = (nb & 1) && a == 0 && b == nb - 1;
        return;
      }
    }
  I = 0;
  J = 1;
  doI = doJ = false;
}

// Block staging of a phase (I, J): block I stays in slots [0, bc) while
// consecutive phases share it (resI), block J goes to slots [bc, 2 bc).
template <typename T, int VEC>
__device__ __forceinline__ void stage_in(T* S, int ldS, T* W, int len, int bc, int rc, int I,
                                         int J, int& resI, int tid, int nth) {
  if (I != resI) {
    if (resI >= 0)
      copy_cols<T, VEC>(S, ldS, W + (int64_t)(resI * bc) * len, len, len, min(bc, rc - resI * bc),
                        tid, nth, false);
    copy_cols<T, VEC>(S, ldS, W + (int64_t)(I * bc) * len, len, len, min(bc, rc - I * bc), tid,
                      nth, true);
    resI = I;
  }
  copy_cols<T, VEC>(S + (int64_t)bc * ldS, ldS, W + (int64_t)(J * bc) * len, len, len,
                    min(bc, rc - J * bc), tid, nth, true);
  __syncthreads();
}

// TILE = 0: pair-per-group rotations; TILE = NQW > 0 (fp32, VEC = 4, mm <= 128
// NQW): the register-tiled form with at most 11 warps.
constexpr int kMaxTileWarps = 12;

// ---- rotation log ----------------------------------------------------------
// One record (kVlogRec float4s) per tile task and kind (inner pairs, cross
// pairs): per sub-round the (t1, t2) of its four pairs, then the eight column
// scales; the columns of V transform as the V pass of tile_group transforms
// the rows of V.  Each round of each sweep and pair set owns a fixed block of
// 2 kVlogRec kmax float4s, so that the replay finds it from the same
// schedule (the bounds of the rounds and tasks of a phase give the
// geometry); inside the block, the record of kind w (0 inner, 1 cross) of
// task k is the kVlogRec float4s from (2 k + w) kVlogRec (one task's record
// in consecutive addresses for the kernel's stores).
constexpr int kVlogRec = 10;
__host__ __device__ inline void vlog_dims(int rc, int bc, bool in_smem, int& nps, int& rmax,
                                          int& kmax) {
  if (in_smem) {   // kind 0: ntp - 1 rounds of ntp / 2 tasks
    const int nt = (rc + 3) / 4, ntp = nt + (nt & 1);
    nps = 1;
    rmax = ntp;
    kmax = ntp / 2 + 1;
  } else {         // kind 1: at most 2 bt rounds of at most bt + 1 tasks
    const int nb = (rc + bc - 1) / bc, bt = (bc + 3) / 4;
    nps = nb * (nb - 1) / 2;
    rmax = 2 * bt + 2;
    kmax = bt + 2;
  }
}
// the first float4 of the block of round t of pair set ps of sweep sw
__host__ __device__ inline int64_t vlog_round(int sw, int ps, int t, int nps, int rmax,
                                              int kmax) {
  return (((int64_t)sw * nps + ps) * rmax + t) * (2 * kVlogRec * kmax);
}

// GW < 32 (whole slice in shared memory, mm <= 4 GW TILE, at most 4 warps):
// the tiled form on groups of GW lanes, 32 / GW tasks per warp.
// REC: the rotation-log form (TILE > 0, GW == 32).
template <typename T, int VEC, int TILE, int GW = 32, bool REC = false>
__global__ void __launch_bounds__(GW < 32 ? 128 : (TILE ? 32 * kMaxTileWarps : 512))
jacobi_kernel(const JacobiParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = blockIdx.x;
  const int tid = threadIdx.x, NTh = blockDim.x;
  const int mm = P.mm, rc = P.rc, ldS = P.ldS, g = P.g;
  // rotation log (register tiles on whole warps only): columns w alone, the
  // rotations recorded instead of applied to V rows
  constexpr bool rec = REC && TILE > 0 && GW == 32;
  const int len = rec ? mm : mm + rc;  // stacked column [w; v] (or w)
  const int lane = tid % g, gid = tid / g, ngroups = NTh / g;
  // Pair slot of this group.  Consecutive pair slots hold consecutive
  // columns, so the groups sharing a warp take slots g apart: their g-row
  // windows then fall on disjoint shared-memory banks (column stride is 1
  // word mod 32).
  int kslot = gid;
  {
    const int nw = NTh / 32, w = tid / 32, j = (tid % 32) / g;
    if (g < 32 && nw % g == 0) kslot = (w % g) + g * j + 32 * (w / g);
  }
  // output pointers are looked up after the sweeps (not kept live in them)
  const T* src = P.desc ? P.desc[s].src : P.src + (int64_t)s * P.src_bs;
  const bool in_smem = rc <= 2 * P.bcols;
  const int ncols_smem = in_smem ? rc : 2 * P.bcols;
  T* S = reinterpret_cast<T*>(smem_raw);
  const int p2 = P.sort_n;  // power of two >= rc
  const size_t sig_off = ((size_t)ncols_smem * ldS * sizeof(T) + 15) & ~(size_t)15;
  double* sig = reinterpret_cast<double*>(smem_raw + sig_off);
  int* idx = reinterpret_cast<int*>(sig + p2);
  T* W = P.W ? P.W + (int64_t)s * P.W_bs : nullptr;
  const int bc = P.bcols;
  const int nb = in_smem ? 1 : (rc + bc - 1) / bc;

  // load the stacked columns [slice; I] into shared memory or the workspace
  __shared__ double red[32];
  double floor_ = 0.0;
  {
    const int tot = len * rc;
    double nrm2 = 0.0;
    for (int e = tid; e < tot; e += NTh) {
      int r, c;
      if (P.trans) { c = e % rc; r = e / rc; } else { r = e % len; c = e / len; }
      const T v = load_work(src, P.m, P.trans, mm, r, c);
      if (r < mm) nrm2 = fma((double)v, (double)v, nrm2);
      if (in_smem) S[(int64_t)c * ldS + r] = v;
      else W[r + (int64_t)c * len] = v;
    }
    nrm2 = block_sum(nrm2, red);
    floor_ = Eps<T>::v * Eps<T>::v * nrm2;
  }
  // convergence thresholds in the working precision (no fp64 in the round)
  const T tol_t = (T)P.tol;
  const T floor_t = (T)floor_;
  int sweeps_used = 0;
  bool converged = (rc <= 1);
  const int npair_sets = in_smem ? 1 : nb * (nb - 1) / 2;
  // (the rotation log holds vlog_sweeps sweeps: the sweep limit in that form)
  const int max_sw = rec ? min(P.max_sweeps, P.vlog_sweeps) : P.max_sweeps;
  for (int sw = 0; sw < max_sw && !converged; ++sw) {
    bool rot = false;
    int I = 0, J = 1;
    int resI = -1;   // block held in slots [0, bc) (block mode)
    if constexpr (TILE > 0) {
      const int wp = tid >> 5, ln = tid & 31, nwp = NTh >> 5;
      const int mq = mm >> 2, rq = rc >> 2;
      if constexpr (GW < 32) {
        // the whole slice in shared memory: round robin over the tiles, the
        // tasks of a round 32 / GW to a warp
        constexpr int TPW = 32 / GW;
        __shared__ float4 cs_part[4 * TPW][10];   // rotation record of each group
        const int grp = ln / GW, gl = ln % GW;
        float4* csg = cs_part[wp * TPW + grp];
        const TPhase ph = tphase_smem(rc);
        const int nrounds = tphase_rounds(ph);
        for (int t = 0; t < nrounds; ++t) {
          const int ntasks = tphase_tasks(ph, t);
          for (int k0 = wp * TPW; k0 < ntasks; k0 += nwp * TPW) {
            const int k = k0 + grp;
            TTask d{0, 0, 0, 0, false};
            const bool live = k < ntasks && tphase_task(ph, t, k, d);
            if (t == 0)
              rot |= tile_group_part<GW, TILE, true>(S, ldS, d.sa, d.na, d.sb, d.nb, d.na > 0,
                                                     d.nb > 0, mq, rq, gl, grp, live, tol_t,
                                                     floor_t, csg);
            const bool cross = live && d.na > 0 && d.nb > 0;
            if (__any_sync(0xffffffffu, cross))
              rot |= tile_group_part<GW, TILE, false>(S, ldS, d.sa, d.na, d.sb, d.nb, false, false,
                                                      mq, rq, gl, grp, cross, tol_t, floor_t, csg);
          }
          __syncthreads();
        }
      } else {
      __shared__ float4 cs_rec[kMaxTileWarps][10];   // rotation record of each warp
      float4* csw = cs_rec[wp];
      int vl_nps = 0, vl_rmax = 0, vl_kmax = 0;
      float4* vlog = nullptr;
      if (rec) {
        vlog_dims(rc, bc, in_smem, vl_nps, vl_rmax, vl_kmax);
        vlog = P.vlog + (int64_t)s * P.vlog_bs;
      }
      const int rqv = rec ? 0 : rq;   // V rows of the stacked columns
      for (int ps = 0; ps < npair_sets; ++ps) {
        TPhase ph;
        if (in_smem) {
          ph = tphase_smem(rc);
        } else {
          bool doI, doJ;
          tile_phase_ij(ps, nb, I, J, doI, doJ);
          stage_in<T, VEC>(S, ldS, W, len, bc, rc, I, J, resI, tid, NTh);
          ph = tphase_blocks(min(bc, rc - I * bc), min(bc, rc - J * bc), bc, doI, doJ);
        }
        const int nrounds = tphase_rounds(ph);
        for (int t = 0; t < nrounds; ++t) {
          const int ntasks = tphase_tasks(ph, t);
          for (int k = wp; k < ntasks; k += nwp) {
            TTask d;
            if (!tphase_task(ph, t, k, d)) continue;
            float4* lg = nullptr;
            if (rec) lg = vlog + vlog_round(sw, ps, t, vl_nps, vl_rmax, vl_kmax) + 2 * kVlogRec * k;
            if (d.inner)
              rot |= tile_group<TILE, true>(S, ldS, d.sa, d.na, d.sb, d.nb, d.na > 0, d.nb > 0, mq,
                                            rqv, ln, tol_t, floor_t, csw, lg);
            if (d.na > 0 && d.nb > 0)
              rot |= tile_group<TILE, false>(S, ldS, d.sa, d.na, d.sb, d.nb, false, false, mq, rqv,
                                             ln, tol_t, floor_t, csw, rec ? lg + kVlogRec : nullptr);
          }
          __syncthreads();
        }
        if (!in_smem)
          copy_cols<T, VEC>(S + (int64_t)bc * ldS, ldS, W + (int64_t)(J * bc) * len, len, len,
                            ph.bJ, tid, NTh, false);
      }
      }
    } else
    for (int ps = 0; ps < npair_sets; ++ps) {
      Phase ph;
      if (in_smem) {
        ph.kind = 0;
        ph.bI = rc;
        ph.cI = rc + (rc & 1);
        ph.bJ = ph.bc = ph.cJ = ph.nri = 0;
        ph.nrounds = ph.cI - 1;
        ph.npairs = ph.cI / 2;
      } else {
        const int bI = min(bc, rc - I * bc), bJ = min(bc, rc - J * bc);
        stage_in<T, VEC>(S, ldS, W, len, bc, rc, I, J, resI, tid, NTh);
        // pairs inside a block on the block's first visit of this sweep
        const bool doI = (I == 0 && J == 1), doJ = (I == 0);
        ph.kind = 1;
        ph.bI = bI;
        ph.bJ = bJ;
        ph.bc = bc;
        ph.cI = doI ? bI + (bI & 1) : 0;
        ph.cJ = doJ ? bJ + (bJ & 1) : 0;
        ph.nri = (doI || doJ) ? max(ph.cI, ph.cJ) - 1 : 0;
        ph.nrounds = ph.nri + bc;
        ph.npairs = max(bc, ph.cI / 2 + ph.cJ / 2);
      }
      for (int t = 0; t < ph.nrounds; ++t) {
        for (int base = 0; base < ph.npairs; base += ngroups) {
          int a = 0, b = 0;
          const bool act = phase_pair(ph, t, base + kslot, a, b);
          rot |= Rotator<T, VEC>::run(S, ldS, a, b, act, mm, len, lane, g, tol_t, floor_t);
        }
        __syncthreads();
      }
      if (!in_smem) {
        copy_cols<T, VEC>(S + (int64_t)bc * ldS, ldS, W + (int64_t)(J * bc) * len, len, len,
                          ph.bJ, tid, NTh, false);
        if (++J == nb) {
          ++I;
          J = I + 1;
        }
      }
    }
    if (resI >= 0)
      copy_cols<T, VEC>(S, ldS, W + (int64_t)(resI * bc) * len, len, len, min(bc, rc - resI * bc),
                        tid, NTh, false);
    sweeps_used = sw + 1;
    if (!__syncthreads_or(rot)) converged = true;
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
  T* Wout;
  T* Vout;
  double* sig_out;
  int* sweeps_out;
  int* status_out;
  if (P.desc) {
    const SliceDesc<T> d = P.desc[s];
    Wout = d.U;
    Vout = d.V;
    sig_out = d.sigma;
    sweeps_out = d.sweeps;
    status_out = d.status;
  } else {
    Wout = P.U + (int64_t)s * P.U_bs;
    Vout = P.V + (int64_t)s * P.V_bs;
    sig_out = P.sigma + (int64_t)s * rc;
    sweeps_out = P.sweeps ? P.sweeps + s : nullptr;
    status_out = P.status;
  }
  double* so = sig_out;
  for (int j = tid; j < rc; j += NTh) {
    so[j] = sig[j];
    if (!isfinite(sig[j])) atomicOr(status_out, SMA_STATUS_BIT(SMA_ERR_NONFINITE));
  }
  T* Wo = Wout;
  T* Vo = Vout;
  for (int e = tid; e < len * rc; e += NTh) {
    const int r = e % len, j = e / len;
    const int c = idx[j];
    const T v = in_smem ? S[(int64_t)c * ldS + r] : W[r + (int64_t)c * len];
    if (r < mm) Wo[r + (int64_t)j * mm] = v;
    else Vo[(r - mm) + (int64_t)j * rc] = v;
  }
  if (rec) {
    for (int j = tid; j < rc; j += NTh) P.order[(int64_t)s * rc + j] = idx[j];
    if (tid == 0) P.vlsweeps[s] = max(converged ? sweeps_used - 1 : sweeps_used, 0);
  }
  if (tid == 0) {
    if (sweeps_out) *sweeps_out = sweeps_used;
    if (!converged) atomicOr(status_out, SMA_STATUS_BIT(SMA_ERR_NOCONVERGE));
  }
}

// ---- one large matrix over many CTAs (cooperative launch) ------------------
// The block mode above walks the block pairs of a sweep one after another in
// one CTA, which leaves one SM to do all of the work for a single matrix (the
// fp64 unfolding Gram of a Tucker variant).  The pairs of one round of a
// block tournament are disjoint, so here CTA c takes pair c of every round:
// nb = 2 gridDim.x blocks of bc columns, round t pairs the blocks by the
// circle method, a block's inner pairs are rotated in round 0 (the first
// round every block plays), and the cross pairs of the two blocks in bc
// sub-rounds as in Phase kind 1.  The stacked columns live in the global
// workspace between rounds (read and written at L2, .cg); rounds are
// separated by a grid barrier on a counter in global memory whose wait is
// bounded: a CTA that gives up sets the abort flag and SMA_ERR_TIMEOUT, and
// every other waiting CTA returns when it sees the flag.

constexpr unsigned long long kCoopWaitNs = 4000000000ull;   // 4 s per barrier

// rotate_pair for fp64 with the angle above; NR rows per lane stay in
// registers between the dot products and the rotation.
template <int NR>
__device__ __forceinline__ bool rotate_pair_f64(double* S, int ldS, int a, int b, bool active,
                                                int mm, int len, int lane, int g, double tol,
                                                double floor_) {
  double xr[NR], yr[NR];
  double al = 0.0, be = 0.0, ga = 0.0;
  double* x = S + (int64_t)(active ? a : 0) * ldS;
  double* y = S + (int64_t)(active ? b : 0) * ldS;
  if (active) {
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int r = lane + i * g;
      xr[i] = 0.0;
      yr[i] = 0.0;
      if (r < mm) {
        xr[i] = x[r];
        yr[i] = y[r];
        al = fma(xr[i], xr[i], al);
        be = fma(yr[i], yr[i], be);
        ga = fma(xr[i], yr[i], ga);
      }
    }
    for (int r = lane + NR * g; r < mm; r += g) {
      const double xv = x[r], yv = y[r];
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
  double c, s;
  if (!angle_fp64_fast(al, be, ga, tol, floor_, c, s)) return false;
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    const int r = lane + i * g;
    if (r < mm) {
      x[r] = c * xr[i] - s * yr[i];
      y[r] = s * xr[i] + c * yr[i];
    }
  }
  for (int r = lane + NR * g; r < mm; r += g) {
    const double xv = x[r], yv = y[r];
    x[r] = c * xv - s * yv;
    y[r] = s * xv + c * yv;
  }
  for (int r = mm + lane; r < len; r += g) {
    const double xv = x[r], yv = y[r];
    x[r] = c * xv - s * yv;
    y[r] = s * xv + c * yv;
  }
  return true;
}

template <typename T>
struct CoopRotator {
  static __device__ __forceinline__ bool run(T* S, int ldS, int a, int b, bool act, int mm,
                                             int len, int lane, int g, T tol, T fl) {
    return Rotator<T, 1>::run(S, ldS, a, b, act, mm, len, lane, g, tol, fl);
  }
};
template <>
struct CoopRotator<double> {
  static __device__ __forceinline__ bool run(double* S, int ldS, int a, int b, bool act, int mm,
                                             int len, int lane, int g, double tol, double fl) {
    return rotate_pair_f64<8>(S, ldS, a, b, act, mm, len, lane, g, tol, fl);
  }
};

__device__ __forceinline__ unsigned long long coop_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier number k (1-based) of the launch: every CTA adds 1 to the counter
// and waits until it reaches k * gridDim.x.  False when the launch aborted.
__device__ bool coop_barrier(const CoopSync& cs, unsigned k, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(cs.bar, 1u);
    const unsigned target = k * gridDim.x;
    const unsigned long long t0 = coop_timer();
    int ok = 1;
    while (*(volatile unsigned*)cs.bar < target) {
      if (*(volatile int*)cs.abort_flag) {
        ok = 0;
        break;
      }
      if (coop_timer() - t0 > kCoopWaitNs) {
        atomicExch(cs.abort_flag, 1);
        atomicOr(status, SMA_STATUS_BIT(SMA_ERR_TIMEOUT));
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ncols stacked columns between shared memory (stride ldS) and the workspace
// (stride len), bypassing L1 so that columns written by other CTAs are seen.
template <typename T>
__device__ __forceinline__ void coop_cols(T* S, int ldS, T* G, int len, int ncols, bool to_smem) {
  for (int e = threadIdx.x; e < len * ncols; e += blockDim.x) {
    const int r = e % len, c = e / len;
    if (to_smem) S[(int64_t)c * ldS + r] = __ldcg(G + (int64_t)c * len + r);
    else __stcg(G + (int64_t)c * len + r, S[(int64_t)c * ldS + r]);
  }
}

template <typename T>
__global__ void __launch_bounds__(512) jacobi_coop_kernel(const JacobiParams<T> P,
                                                          const CoopSync cs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, NTh = blockDim.x;
  const int cta = blockIdx.x, ncta = gridDim.x;
  const int mm = P.mm, rc = P.rc, ldS = P.ldS, g = P.g, bc = P.bcols;
  const int len = mm + rc;
  const int lane = tid % g, kslot = tid / g, ngroups = NTh / g;
  const int nb = 2 * ncta;
  T* S = reinterpret_cast<T*>(smem_raw);
  T* W = P.W;
  unsigned nbar = 0;
  // stacked columns [A; I] into the workspace (the CTAs share the copy) and
  // ||A||_F^2 (every CTA sums it whole, so no reduction across CTAs is needed)
  __shared__ double red[32];
  double nrm2 = 0.0;
  {
    const int64_t tot = (int64_t)len * rc;
    for (int64_t e = (int64_t)cta * NTh + tid; e < tot; e += (int64_t)ncta * NTh) {
      const int r = (int)(e % len), c = (int)(e / len);
      __stcg(W + e, load_work(P.src, P.m, P.trans, mm, r, c));
    }
    for (int64_t e = tid; e < (int64_t)mm * rc; e += NTh) {
      const int r = (int)(e % mm), c = (int)(e / mm);
      const double v = (double)load_work(P.src, P.m, P.trans, mm, r, c);
      nrm2 = fma(v, v, nrm2);
    }
    nrm2 = block_sum(nrm2, red);
  }
  const T tol_t = (T)P.tol;
  const T floor_t = (T)(Eps<T>::v * Eps<T>::v * nrm2);
  if (!coop_barrier(cs, ++nbar, P.status)) return;
  int sweeps_used = 0;
  bool converged = (rc <= 1);
  for (int sw = 0; sw < P.max_sweeps && !converged; ++sw) {
    bool rot = false;
    for (int t = 0; t < nb - 1; ++t) {
      const Pair pr = rr_pair(cta, t, nb);
      const int bI = max(0, min(bc, rc - pr.a * bc)), bJ = max(0, min(bc, rc - pr.b * bc));
      T* WI = W + (int64_t)pr.a * bc * len;
      T* WJ = W + (int64_t)pr.b * bc * len;
      coop_cols<T>(S, ldS, WI, len, bI, true);
      coop_cols<T>(S + (int64_t)bc * ldS, ldS, WJ, len, bJ, true);
      __syncthreads();
      Phase ph;
      ph.kind = 1;
      ph.bI = bI;
      ph.bJ = bJ;
      ph.bc = bc;
      ph.cI = (t == 0 && bI > 1) ? bI + (bI & 1) : 0;
      ph.cJ = (t == 0 && bJ > 1) ? bJ + (bJ & 1) : 0;
      ph.nri = (ph.cI || ph.cJ) ? max(ph.cI, ph.cJ) - 1 : 0;
      ph.nrounds = ph.nri + ((bI > 0 && bJ > 0) ? bc : 0);
      ph.npairs = max(bc, ph.cI / 2 + ph.cJ / 2);
      for (int r = 0; r < ph.nrounds; ++r) {
        for (int base = 0; base < ph.npairs; base += ngroups) {
          int a = 0, b = 0;
          const bool act = phase_pair(ph, r, base + kslot, a, b);
          rot |= CoopRotator<T>::run(S, ldS, a, b, act, mm, len, lane, g, tol_t, floor_t);
        }
        __syncthreads();
      }
      coop_cols<T>(S, ldS, WI, len, bI, false);
      coop_cols<T>(S + (int64_t)bc * ldS, ldS, WJ, len, bJ, false);
      if (!coop_barrier(cs, ++nbar, P.status)) return;
    }
    // sweep result: CTAs that rotated anything count themselves, then every
    // CTA reads the count after one more barrier
    if (__syncthreads_or(rot) && tid == 0) atomicAdd(cs.rot + sw, 1);
    if (!coop_barrier(cs, ++nbar, P.status)) return;
    sweeps_used = sw + 1;
    converged = *(volatile int*)(cs.rot + sw) == 0;
  }
  if (cta != 0) return;
  // CTA 0: column norms, descending sort, outputs (as in jacobi_kernel)
  const int p2 = P.sort_n;
  const size_t sig_off = ((size_t)2 * bc * ldS * sizeof(T) + 15) & ~(size_t)15;
  double* sig = reinterpret_cast<double*>(smem_raw + sig_off);
  int* idx = reinterpret_cast<int*>(sig + p2);
  const int warp = tid >> 5, wl = tid & 31, nwarps = NTh >> 5;
  for (int c = warp; c < p2; c += nwarps) {
    double acc = 0.0;
    if (c < rc)
      for (int r = wl; r < mm; r += 32) {
        const double v = (double)__ldcg(W + r + (int64_t)c * len);
        acc = fma(v, v, acc);
      }
    acc = warp_sum(acc);
    if (wl == 0) {
      sig[c] = (c < rc) ? sqrt(acc) : -1.0;
      idx[c] = c;
    }
  }
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < p2; i += NTh) {
        const int l = i ^ j;
        if (l > i) {
          const double si = sig[i], sl = sig[l];
          const int ii = idx[i], il = idx[l];
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
  for (int j = tid; j < rc; j += NTh) {
    P.sigma[j] = sig[j];
    if (!isfinite(sig[j])) atomicOr(P.status, SMA_STATUS_BIT(SMA_ERR_NONFINITE));
  }
  for (int64_t e = tid; e < (int64_t)len * rc; e += NTh) {
    const int r = (int)(e % len), j = (int)(e / len);
    const T v = __ldcg(W + r + (int64_t)idx[j] * len);
    if (r < mm) P.U[r + (int64_t)j * mm] = v;
    else P.V[(r - mm) + (int64_t)j * rc] = v;
  }
  if (tid == 0) {
    if (P.sweeps) *P.sweeps = sweeps_used;
    if (!converged) atomicOr(P.status, SMA_STATUS_BIT(SMA_ERR_NOCONVERGE));
  }
}

// ---- one fp32 matrix over a cluster of CTAs --------------------------------
// The single-CTA block mode walks the block pairs of a sweep one after
// another on one SM.  Here a cluster of CL CTAs shares one matrix (the fp32
// pass of a Gram eigen-solve): the columns are split into 2 CL blocks of
// bcols (a multiple of 4), round t of a sweep pairs the blocks by the circle
// method and CTA c takes pair c, staging both blocks from the L2-resident
// workspace into its shared memory and running the register-tiled phase of
// the block mode on them (the blocks' inner pairs in round 0, where every
// block plays, then the cross pairs); the blocks go back to the workspace
// and the rounds are separated by the hardware cluster barrier (release /
// acquire at cluster scope; the workspace is read with ld.global.cg so no
// CTA sees a stale L1 line).  Every column pair is rotated exactly once per
// sweep; a sweep that rotates nothing ends the solve (a per-sweep counter in
// global memory, cleared by the launcher).  CTA 0 then sorts and writes the
// outputs as jacobi_kernel does.
constexpr int kClusterCtas = 8;
constexpr int kClusterWarps = 4;

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

// ncols stacked columns of `rows` floats between shared memory (stride ldS)
// and the workspace (stride ldg), float4, L1 bypassed on the loads
__device__ __forceinline__ void cluster_cols(float* S, int ldS, float* G, int ldg, int rows,
                                             int ncols, int tid, int nth, bool to_smem) {
  const int rq = rows >> 2;
  for (int e = tid; e < rq * ncols; e += nth) {
    const int r = e % rq, c = e / rq;
    float4* s4 = reinterpret_cast<float4*>(S + (int64_t)c * ldS) + r;
    float4* g4 = reinterpret_cast<float4*>(G + (int64_t)c * ldg) + r;
    if (to_smem) *s4 = __ldcg(g4);
    else __stcg(g4, *s4);
  }
}

template <int TILE>
__global__ void __launch_bounds__(32 * kClusterWarps)
    jacobi_cluster_kernel(const JacobiParams<float> P, int* __restrict__ rot_count) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, NTh = blockDim.x;
  const int cta = blockIdx.x, ncta = gridDim.x;
  const int mm = P.mm, rc = P.rc, ldS = P.ldS, bc = P.bcols;
  const int len = mm + rc;
  const int nb = 2 * ncta;
  float* S = reinterpret_cast<float*>(smem_raw);
  float* W = P.W;
  const int wp = tid >> 5, ln = tid & 31, nwp = NTh >> 5;
  const int mq = mm >> 2, rq = rc >> 2;
  __shared__ float4 cs_rec[kClusterWarps][10];
  float4* csw = cs_rec[wp];
  // stacked columns [A; I] into the workspace (shared by the cluster's
  // threads) and ||A||_F^2 (every CTA sums it whole: no cross-CTA reduction)
  __shared__ double red[32];
  double nrm2 = 0.0;
  {
    const int64_t tot = (int64_t)len * rc;
    for (int64_t e = (int64_t)cta * NTh + tid; e < tot; e += (int64_t)ncta * NTh) {
      const int r = (int)(e % len), c = (int)(e / len);
      __stcg(W + e, load_work(P.src, P.m, P.trans, mm, r, c));
    }
    for (int64_t e = tid; e < (int64_t)mm * rc; e += NTh) {
      const int r = (int)(e % mm), c = (int)(e / mm);
      const double v = (double)load_work(P.src, P.m, P.trans, mm, r, c);
      nrm2 = fma(v, v, nrm2);
    }
    nrm2 = block_sum(nrm2, red);
  }
  const float tol_t = (float)P.tol;
  const float floor_t = (float)(Eps<float>::v * Eps<float>::v * nrm2);
  cluster_barrier();
  int sweeps_used = 0;
  bool converged = (rc <= 1);
  for (int sw = 0; sw < P.max_sweeps && !converged; ++sw) {
    bool rot = false;
    for (int t = 0; t < nb - 1; ++t) {
      const Pair pr = rr_pair(cta, t, nb);
      const int bI = max(0, min(bc, rc - pr.a * bc)), bJ = max(0, min(bc, rc - pr.b * bc));
      float* WI = W + (int64_t)pr.a * bc * len;
      float* WJ = W + (int64_t)pr.b * bc * len;
      cluster_cols(S, ldS, WI, len, len, bI, tid, NTh, true);
      cluster_cols(S + (int64_t)bc * ldS, ldS, WJ, len, len, bJ, tid, NTh, true);
      __syncthreads();
      const TPhase ph = tphase_blocks(bI, bJ, bc, t == 0 && bI > 1, t == 0 && bJ > 1);
      const int nrounds = (bI > 0 || bJ > 0) ? tphase_rounds(ph) : 0;
      for (int r = 0; r < nrounds; ++r) {
        const int ntasks = tphase_tasks(ph, r);
        for (int k = wp; k < ntasks; k += nwp) {
          TTask d;
          if (!tphase_task(ph, r, k, d)) continue;
          if (d.inner)
            rot |= tile_group<TILE, true>(S, ldS, d.sa, d.na, d.sb, d.nb, d.na > 0, d.nb > 0, mq,
                                          rq, ln, tol_t, floor_t, csw);
          if (d.na > 0 && d.nb > 0)
            rot |= tile_group<TILE, false>(S, ldS, d.sa, d.na, d.sb, d.nb, false, false, mq, rq,
                                           ln, tol_t, floor_t, csw);
        }
        __syncthreads();
      }
      cluster_cols(S, ldS, WI, len, len, bI, tid, NTh, false);
      cluster_cols(S + (int64_t)bc * ldS, ldS, WJ, len, len, bJ, tid, NTh, false);
      cluster_barrier();
    }
    // sweep result: CTAs that rotated anything count themselves, then every
    // CTA reads the count after one more cluster barrier
    if (__syncthreads_or(rot) && tid == 0) atomicAdd(rot_count + sw, 1);
    cluster_barrier();
    sweeps_used = sw + 1;
    converged = __ldcg(rot_count + sw) == 0;
  }
  if (cta != 0) return;
  // CTA 0: column norms, descending sort, outputs (as in jacobi_kernel)
  const int p2 = P.sort_n;
  const size_t sig_off = ((size_t)2 * bc * ldS * sizeof(float) + 15) & ~(size_t)15;
  double* sig = reinterpret_cast<double*>(smem_raw + sig_off);
  int* idx = reinterpret_cast<int*>(sig + p2);
  const int nwarps = NTh >> 5;
  for (int c = wp; c < p2; c += nwarps) {
    double acc = 0.0;
    if (c < rc)
      for (int r = ln; r < mm; r += 32) {
        const double v = (double)__ldcg(W + r + (int64_t)c * len);
        acc = fma(v, v, acc);
      }
    acc = warp_sum(acc);
    if (ln == 0) {
      sig[c] = (c < rc) ? sqrt(acc) : -1.0;
      idx[c] = c;
    }
  }
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < p2; i += NTh) {
        const int l = i ^ j;
        if (l > i) {
          const double si = sig[i], sl = sig[l];
          const int ii = idx[i], il = idx[l];
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
  for (int j = tid; j < rc; j += NTh) {
    P.sigma[j] = sig[j];
    if (!isfinite(sig[j])) atomicOr(P.status, SMA_STATUS_BIT(SMA_ERR_NONFINITE));
  }
  for (int64_t e = tid; e < (int64_t)len * rc; e += NTh) {
    const int r = (int)(e % len), j = (int)(e / len);
    const float v = __ldcg(W + r + (int64_t)idx[j] * len);
    if (r < mm) P.U[r + (int64_t)j * mm] = v;
    else P.V[(r - mm) + (int64_t)j * rc] = v;
  }
  if (tid == 0) {
    if (P.sweeps) *P.sweeps = sweeps_used;
    if (!converged) atomicOr(P.status, SMA_STATUS_BIT(SMA_ERR_NOCONVERGE));
  }
}

// ---- V from the rotation log -----------------------------------------------
// CTA (s, g) forms the needed columns j = d0 + g + VR_SPLIT i of slice s
// (d0 = ranks[s]) in shared memory, x[i] starting as the unit vector of the
// pre-sort column order[j]; the columns of one slice spread over VR_SPLIT
// CTAs, so a slice with few needed columns runs them in parallel.  V is the
// product of the tasks' maps in execution order (each acting on the right,
// on the task's eight columns), so its columns come from applying the maps
// in reverse: sweeps, pair sets and rounds last to first; the tasks of a
// round act on disjoint columns and run in parallel; a task's cross record
// goes before its inner record.  A record maps x as the transpose of the row
// map of tile_group's V pass: x_c *= d_c, then for the sub-rounds last to
// first and each pair (a, b) with (t1, t2): x_a <- x_a + t2 x_b,
// x_b <- x_b - t1 x_a.  The schedule is the same in every sweep, so each
// task's eight columns and kinds are tabled once; the coming rounds' records
// are copied from the log into a ring in shared memory with cp.async
// (field-major there, so that the lanes, one task each, read a field at
// consecutive addresses) while the current round is applied.  A round's work
// is a short dependent chain, so a CTA with one column is replayed by one
// warp without block barriers.
constexpr int VR_THREADS = 256;
constexpr int VR_SPLIT = 32;   // CTAs per slice (grid y)
constexpr int VR_COLS = 8;     // columns per CTA (rc <= VR_SPLIT VR_COLS)
constexpr int VR_AHEAD = 8;    // rounds prefetched ahead
constexpr int VR_RING = VR_AHEAD + 1;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// the schedule position of one round: sweep, pair set, round
struct VrPos {
  int sw, ps, t;
};
// one round back in execution order; false past the first round
__device__ __forceinline__ bool vr_back(VrPos& q, int nps, const unsigned char* nr) {
  if (--q.t >= 0) return true;
  if (--q.ps < 0) {
    q.ps = nps - 1;
    if (--q.sw < 0) return false;
  }
  q.t = nr[q.ps] - 1;
  return true;
}

// the phase of pair set ps (the kernel's, see jacobi_kernel)
__device__ __forceinline__ TPhase vr_phase(int ps, int rc, int bc, bool in_smem, int nb, int& I,
                                           int& J) {
  if (in_smem) {
    I = 0;
    J = 0;
    return tphase_smem(rc);
  }
  bool doI, doJ;
  tile_phase_ij(ps, nb, I, J, doI, doJ);
  return tphase_blocks(min(bc, rc - I * bc), min(bc, rc - J * bc), bc, doI, doJ);
}

// (field f of the record at rec[f fs])
template <bool INNER>
__device__ __forceinline__ void vr_apply(const float4* rec, int fs, float (&x)[8]) {
  constexpr int NR = INNER ? 3 : 4;
  const float4 d03 = rec[8 * fs], d47 = rec[9 * fs];
  x[0] *= d03.x; x[1] *= d03.y; x[2] *= d03.z; x[3] *= d03.w;
  x[4] *= d47.x; x[5] *= d47.y; x[6] *= d47.z; x[7] *= d47.w;
#pragma unroll
  for (int r = NR - 1; r >= 0; --r) {
    const float4 r01 = rec[(2 * r) * fs], r23 = rec[(2 * r + 1) * fs];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int a, b;
      tile_pair<INNER>(r, q, a, b);
      const float t1 = q == 0 ? r01.x : q == 1 ? r01.z : q == 2 ? r23.x : r23.z;
      const float t2 = q == 0 ? r01.y : q == 1 ? r01.w : q == 2 ? r23.y : r23.w;
      const float xa = x[a], xb = x[b];
      x[a] = fmaf(t2, xb, xa);
      x[b] = fmaf(-t1, xa, xb);
    }
  }
}

// task table entry flags
constexpr unsigned char VR_CROSS = 1, VR_INNER = 2;
constexpr unsigned short VR_NOCOL = 0xffff;

// shared-memory bytes of the replay for rc columns, block columns bc
__host__ __device__ inline size_t vr_smem_bytes(int rc, int bc) {
  const bool in_smem = rc <= 2 * bc;
  int nps, rmax, kmax;
  vlog_dims(rc, bc, in_smem, nps, rmax, kmax);
  const size_t ntab = (size_t)nps * rmax * kmax;
  return (size_t)VR_RING * 2 * kVlogRec * kmax * sizeof(float4)   // ring
         + ntab * 8 * sizeof(unsigned short)                       // task columns
         + (size_t)VR_COLS * rc * sizeof(float)                    // x
         + ntab + (size_t)nps * rmax + nps;                        // flags, tasks, rounds
}

__global__ void __launch_bounds__(VR_THREADS)
    jacobi_v_replay_kernel(const JacobiParams<float> P, int bc, const int* __restrict__ ranks) {
  extern __shared__ __align__(16) unsigned char vr_smem[];
  const int s = blockIdx.x, g = blockIdx.y, rc = P.rc, tid = threadIdx.x;
  const int d0 = ranks ? min(max(ranks[s], 0), rc) : 0;
  const int nd = rc - d0;
  // this CTA's columns j = d0 + g + VR_SPLIT i, i < nv
  const int nv = nd > g ? min((nd - g + VR_SPLIT - 1) / VR_SPLIT, VR_COLS) : 0;
  if (nv == 0) return;   // (uniform over the CTA)
  const bool in_smem = rc <= 2 * bc;
  const int nb = in_smem ? 1 : (rc + bc - 1) / bc;
  int nps, rmax, kmax;
  vlog_dims(rc, bc, in_smem, nps, rmax, kmax);
  const int ntab = nps * rmax * kmax;
  const int rec4 = 2 * kVlogRec * kmax;   // float4s of one round's records
  float4* ring = reinterpret_cast<float4*>(vr_smem);                        // [VR_RING][rec4]
  uint4* tcol = reinterpret_cast<uint4*>(ring + (size_t)VR_RING * rec4);     // [ntab] 8 x u16
  float* x = reinterpret_cast<float*>(tcol + ntab);                         // [VR_COLS][rc]
  unsigned char* tflag = reinterpret_cast<unsigned char*>(x + (size_t)VR_COLS * rc);  // [ntab]
  unsigned char* ntk = tflag + ntab;                                        // [nps][rmax]
  unsigned char* nr = ntk + nps * rmax;                                     // [nps]
  // the task table (the same in every sweep), by the whole CTA
  for (int e = tid; e < nps * rmax; e += VR_THREADS) {
    const int ps = e / rmax, t = e % rmax;
    int I, J;
    const TPhase ph = vr_phase(ps, rc, bc, in_smem, nb, I, J);
    const int nrounds = tphase_rounds(ph);
    if (t == 0) nr[ps] = (unsigned char)nrounds;
    const int ntasks = t < nrounds ? tphase_tasks(ph, t) : 0;
    ntk[e] = (unsigned char)ntasks;
    for (int k = 0; k < kmax; ++k) {
      TTask d;
      unsigned char fl = 0;
      unsigned short cl[8];
      if (k < ntasks && tphase_task(ph, t, k, d)) {
        fl = (d.na > 0 && d.nb > 0 ? VR_CROSS : 0) | (d.inner ? VR_INNER : 0);
        for (int c = 0; c < 8; ++c) {
          const int slot = c < 4 ? d.sa + c : d.sb + c - 4;
          const bool valid = c < 4 ? c < d.na : (c - 4) < d.nb;
          const int cg = in_smem ? slot : (slot < bc ? I * bc + slot : J * bc + slot - bc);
          cl[c] = valid ? (unsigned short)cg : VR_NOCOL;
        }
      } else {
        for (int c = 0; c < 8; ++c) cl[c] = VR_NOCOL;
      }
      tflag[e * kmax + k] = fl;
      tcol[e * kmax + k] = make_uint4(cl[0] | ((unsigned)cl[1] << 16), cl[2] | ((unsigned)cl[3] << 16),
                                      cl[4] | ((unsigned)cl[5] << 16), cl[6] | ((unsigned)cl[7] << 16));
    }
  }
  __syncthreads();
  // a round's units (task, column of V) fit one warp when few columns are
  // needed: then warp 0 alone replays and synchronises by __syncwarp
  const bool one = nv * kmax <= 32;
  if (one && tid >= 32) return;   // (uniform over each warp; no block barrier follows)
  const int nth = one ? 32 : VR_THREADS;
  auto sync = [&]() {
    if (one) __syncwarp();
    else __syncthreads();
  };
  const float4* vlog = P.vlog + (int64_t)s * P.vlog_bs;
  const int nsw = P.vlsweeps[s];
  const int* order = P.order + (int64_t)s * rc;
  float* Vs = P.V + (int64_t)s * P.V_bs;
  {
    for (int e = tid; e < rc * nv; e += nth) x[e] = 0.f;
    sync();
    for (int v = tid; v < nv; v += nth) {
      const int c = order[d0 + g + VR_SPLIT * v];
      if ((unsigned)c < (unsigned)rc) x[v * rc + c] = 1.f;
    }
    // rounds in reverse execution order, from the last round of the last
    // rotating sweep; the ring slot of the i-th round is i mod VR_RING
    VrPos cur{nsw - 1, nps - 1, nr[nps - 1] - 1};
    bool cur_ok = nsw > 0;
    VrPos pre = cur;
    bool pre_ok = cur_ok;
    int issued = 0, done = 0;
    auto issue = [&]() {
      if (pre_ok) {
        // the round's cross records (and, in a round with inner pairs, the
        // inner ones), field-major into the ring slot
        const float4* src = vlog + vlog_round(pre.sw, pre.ps, pre.t, nps, rmax, kmax);
        float4* dst = ring + (size_t)(issued % VR_RING) * rec4;
        const int nt = ntk[pre.ps * rmax + pre.t];
        const int kinds = pre.t == 0 ? 2 : 1;
        for (int e = tid; e < nt * kinds; e += nth) {
          const int k = e % nt, w = kinds == 2 ? e / nt : 1;
          const float4* rs = src + (2 * k + w) * kVlogRec;
#pragma unroll
          for (int f = 0; f < kVlogRec; ++f) cp_async16(dst + (w * kVlogRec + f) * kmax + k, rs + f);
        }
        pre_ok = vr_back(pre, nps, nr);
      }
      cp_async_commit();
      ++issued;
    };
    for (int j = 0; j < VR_AHEAD; ++j) issue();
    while (cur_ok) {
      cp_async_wait<VR_AHEAD - 1>();
      sync();   // the round's records (and the previous round's x) visible
      const float4* rr = ring + (size_t)(done % VR_RING) * rec4;
      const int tb = (cur.ps * rmax + cur.t) * kmax;
      const int ntasks = ntk[cur.ps * rmax + cur.t];
      for (int u = tid; u < ntasks * nv; u += nth) {
        const int k = u % ntasks, v = u / ntasks;   // (lanes on tasks: distinct columns)
        const unsigned char fl = tflag[tb + k];
        if (!fl) continue;
        const uint4 cw = tcol[tb + k];
        const unsigned short col[8] = {
            (unsigned short)(cw.x & 0xffff), (unsigned short)(cw.x >> 16),
            (unsigned short)(cw.y & 0xffff), (unsigned short)(cw.y >> 16),
            (unsigned short)(cw.z & 0xffff), (unsigned short)(cw.z >> 16),
            (unsigned short)(cw.w & 0xffff), (unsigned short)(cw.w >> 16)};
        float* xv0 = x + (size_t)v * rc;
        float xv[8];
        bool nz = false;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          xv[c] = col[c] != VR_NOCOL ? xv0[col[c]] : 0.f;
          nz |= xv[c] != 0.f;
        }
        if (!nz) continue;   // the maps keep zero entries zero
        if (fl & VR_CROSS) vr_apply<false>(rr + kVlogRec * kmax + k, kmax, xv);
        if (fl & VR_INNER) vr_apply<true>(rr + k, kmax, xv);
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (col[c] != VR_NOCOL) xv0[col[c]] = xv[c];
      }
      ++done;
      cur_ok = vr_back(cur, nps, nr);
      sync();   // the round is applied: its ring slot may be refilled
      issue();
    }
    cp_async_wait<0>();
    sync();
    for (int e = tid; e < rc * nv; e += nth) {
      const int r = e % rc, v = e / rc;
      Vs[r + (int64_t)(d0 + g + VR_SPLIT * v) * rc] = x[e];
    }
  }
}

}  // namespace

template <typename T>
JacobiPlan jacobi_plan_impl(int m, int n, int max_smem, bool allow_tile, bool rec = false) {
  JacobiPlan pl;
  const int max_smem_in = max_smem;
  // leave room for the kernel's static shared memory
  max_smem = max_smem > 3072 ? max_smem - 3072 : 0;
  pl.trans = (m < n) ? 1 : 0;
  pl.mm = pl.trans ? n : m;
  pl.rc = pl.trans ? m : n;
  pl.vec = (sizeof(T) == 4 && pl.mm % 4 == 0 && pl.rc % 4 == 0) ? 4 : 1;
  // the rotation-log form: register tiles on whole warps (fp32, float4 rows,
  // 64 < mm <= 256), the stacked columns without their V rows
  pl.rec = (rec && allow_tile && sizeof(T) == 4 && pl.vec == 4 && pl.mm > 64 && pl.mm <= 256 &&
            pl.rc >= 32) ? 1 : 0;
  pl.ldS = pl.mm + (pl.rec ? 0 : pl.rc) + (pl.vec == 4 ? 4 : 1);
  int p2 = 1;
  while (p2 < pl.rc) p2 <<= 1;
  pl.sort_n = p2;
  const size_t sort_bytes = (size_t)p2 * (sizeof(double) + sizeof(int)) + 16;
  const size_t col_bytes = (size_t)pl.ldS * sizeof(T);
  const size_t full = (size_t)pl.rc * col_bytes + sort_bytes;
  // block mode needs two stacked columns and the sort buffer in shared
  // memory at the least; a slice whose columns are longer than that has no
  // plan (smem = 0: callers reject the shape before any launch)
  if (2 * col_bytes + sort_bytes > (size_t)max_smem) {
    pl.bcols = 0;
    pl.threads = 0;
    pl.g = 0;
    pl.block_mode = 0;
    pl.tile = 0;
    pl.smem = 0;
    return pl;
  }
  if (full <= (size_t)max_smem) {
    pl.bcols = (pl.rc + 1) / 2 > 0 ? (pl.rc + 1) / 2 : 1;
    pl.smem = full;
  } else {
    const int bmax = (int)(((size_t)max_smem - sort_bytes) / (2 * col_bytes));
    const int nb = (pl.rc + bmax - 1) / bmax < 3 ? 3 : (pl.rc + bmax - 1) / bmax;
    pl.bcols = (pl.rc + nb - 1) / nb;
    pl.smem = 2 * (size_t)pl.bcols * col_bytes + sort_bytes;
  }
  // register-tiled sweeps: fp32 float4 rows, dot-product part <= 256 rows,
  // enough tiles of 4 columns to keep 12 warps busy
  pl.tile = (allow_tile && sizeof(T) == 4 && pl.vec == 4 && pl.mm <= 256 && pl.rc >= 32)
                ? (pl.mm <= 128 ? 1 : 2)
                : 0;
  if (pl.tile) {
    // one warp per tile-pair task of a round, at most kTileWarps
    constexpr int kTileWarps = kMaxTileWarps;
    pl.g = 32;
    if (full > (size_t)max_smem) {
      // blocks of a multiple of 4 columns, at most 4 per warp (one tile pair
      // per warp and cross round)
      int bmax = (int)(((size_t)max_smem - sort_bytes) / (2 * col_bytes)) & ~3;
      // (without V rows twice the columns fit: two tile pairs per warp and round)
      const int bcap = (pl.rec ? 8 : 4) * kTileWarps;
      if (bmax > bcap) bmax = bcap;
      if (bmax >= 4) {
        int nb = (pl.rc + bmax - 1) / bmax;
        if (nb < 3) nb = 3;
        pl.bcols = (((pl.rc + nb - 1) / nb) + 3) & ~3;
        pl.smem = 2 * (size_t)pl.bcols * col_bytes + sort_bytes;
        pl.block_mode = pl.rc <= 2 * pl.bcols ? 0 : 1;
        pl.threads = 32 * kTileWarps;   // the spare warps shorten the first-visit rounds
        if (pl.block_mode) return pl;
      }
      pl.tile = 0;   // fall back to the pair-per-group plan below
      const int bm2 = (int)(((size_t)max_smem - sort_bytes) / (2 * col_bytes));
      const int nb2 = (pl.rc + bm2 - 1) / bm2 < 3 ? 3 : (pl.rc + bm2 - 1) / bm2;
      pl.bcols = (pl.rc + nb2 - 1) / nb2;
      pl.smem = 2 * (size_t)pl.bcols * col_bytes + sort_bytes;
    } else {
      const int nt = (pl.rc + 3) / 4, tasks = (nt + (nt & 1)) / 2;
      if (pl.mm <= 64) {
        // short columns (at most 16 float4 rows): groups of g = 16 or 8 lanes
        // per task, so no lane idles; the round's tasks on at most 4 warps
        const int gw = pl.mm <= 32 ? 8 : 16, tpw = 32 / gw;
        pl.g = gw;
        pl.tile = 1;
        pl.threads = 32 * std::min(4, (tasks + tpw - 1) / tpw);
      } else {
        pl.threads = 32 * (tasks < 4 ? 4 : (tasks > kTileWarps ? kTileWarps : tasks));
      }
      pl.block_mode = 0;
      return pl;
    }
  }
  if (pl.rec) return jacobi_plan_impl<T>(m, n, max_smem_in, allow_tile, false);
  const bool in_smem = pl.rc <= 2 * pl.bcols;
  const int maxpairs = in_smem ? (pl.rc + 1) / 2 : pl.bcols;
  // threads: one group of g lanes per pair of a round, about 16 rows per lane
  int gd = 1;
  while (gd < 32 && gd * 16 < pl.mm + pl.rc) gd <<= 1;
  int nt = 32;
  while (nt < 512 && nt < maxpairs * gd) nt <<= 1;
  int gp = 1;
  while (gp * 2 <= 32 && gp * 2 * (maxpairs > 0 ? maxpairs : 1) <= nt) gp <<= 1;
  pl.threads = nt;
  pl.g = gp;
  pl.block_mode = in_smem ? 0 : 1;
  return pl;
}

template <typename T>
JacobiPlan jacobi_plan(int m, int n, int max_smem, bool rec) {
  return jacobi_plan_impl<T>(m, n, max_smem, true, rec);
}

size_t jacobi_log_size(const JacobiPlan& pl, int sweeps) {
  if (!pl.rec) return 0;
  int nps = 0, rmax = 0, kmax = 0;
  vlog_dims(pl.rc, pl.bcols, pl.rc <= 2 * pl.bcols, nps, rmax, kmax);
  return (size_t)(sweeps > 0 ? sweeps : 1) * nps * rmax * kmax * 2 * kVlogRec;
}

// Alternatives to the default plan for the autotuner, all with the default's
// storage mode (whole slice in shared memory or block mode), so one
// workspace serves them: the untiled form where the default is tiled, and
// for tiled block mode 4 columns more or fewer per block and 11 or 12 warps.
template <typename T>
std::vector<JacobiPlan> jacobi_plan_candidates(int m, int n, int max_smem, bool rec) {
  std::vector<JacobiPlan> out;
  const JacobiPlan base = jacobi_plan<T>(m, n, max_smem, rec);
  out.push_back(base);
  if (base.smem == 0) return out;   // no plan for this shape
  if (base.tile && !base.rec) {
    const JacobiPlan u = jacobi_plan_impl<T>(m, n, max_smem, false);
    if (u.block_mode == base.block_mode) out.push_back(u);
  }
  if (base.tile && base.block_mode) {
    const int cap = (max_smem > 3072 ? max_smem - 3072 : 0);
    const size_t sort_bytes = (size_t)base.sort_n * (sizeof(double) + sizeof(int)) + 16;
    const size_t col_bytes = (size_t)base.ldS * sizeof(T);
    for (int d : {-4, 4}) {
      JacobiPlan v = base;
      v.bcols = base.bcols + d;
      v.smem = 2 * (size_t)v.bcols * col_bytes + sort_bytes;
      // (the rotation-log form keeps the base's block count: the log is
      // sized for the largest candidate)
      const bool same_nb = !base.rec || (base.rc + v.bcols - 1) / v.bcols ==
                                            (base.rc + base.bcols - 1) / base.bcols;
      if (same_nb && v.bcols >= 8 && v.bcols <= (base.rec ? 96 : 48) && v.smem <= (size_t)cap &&
          base.rc > 2 * v.bcols &&
          (base.rc + v.bcols - 1) / v.bcols >= 3)
        out.push_back(v);
    }
    JacobiPlan w = base;
    w.threads = base.threads == 384 ? 352 : 384;
    out.push_back(w);
  }
  // whole slice in shared memory: smaller CTAs put more slices on an SM (the
  // round robin then takes several passes of the warps per round)
  if (!base.block_mode && base.rec) {
    for (int t : {64, 128})
      if (t < base.threads) {
        JacobiPlan v = base;
        v.threads = t;
        out.push_back(v);
      }
    return out;
  }
  if (!base.block_mode) {
    if (base.tile) {
      for (int t : {64, 128})
        if (t < base.threads) {
          JacobiPlan v = base;
          v.threads = t;
          out.push_back(v);
        }
      if (base.g < 32) {
        // partial-warp groups: half as many lanes with two float4 rows each
        // (twice the tasks per warp), and the full-warp tiled form
        const int nt = (base.rc + 3) / 4, tasks = (nt + (nt & 1)) / 2;
        JacobiPlan h2 = base;
        h2.g = base.g / 2;
        h2.tile = 2;
        const int tpw = 32 / h2.g;
        h2.threads = 32 * std::min(4, (tasks + tpw - 1) / tpw);
        out.push_back(h2);
        JacobiPlan f = base;
        f.g = 32;
        f.tile = 1;
        f.threads = 32 * std::max(4, std::min(kMaxTileWarps, tasks));
        out.push_back(f);
      }
      JacobiPlan u = jacobi_plan_impl<T>(m, n, max_smem, false);
      if (!u.block_mode && u.threads >= 64) {
        const int nt = u.threads / 2;
        int gp = 1;
        const int mp = (u.rc + 1) / 2;
        while (gp * 2 <= 32 && gp * 2 * (mp > 0 ? mp : 1) <= nt) gp <<= 1;
        u.threads = nt;
        u.g = gp;
        out.push_back(u);
      }
    } else if (base.threads >= 64) {
      JacobiPlan u = base;
      const int nt = u.threads / 2;
      int gp = 1;
      const int mp = (u.rc + 1) / 2;
      while (gp * 2 <= 32 && gp * 2 * (mp > 0 ? mp : 1) <= nt) gp <<= 1;
      u.threads = nt;
      u.g = gp;
      out.push_back(u);
    }
  }
  return out;
}

template <typename T>
cudaError_t jacobi_svd(const JacobiParams<T>& P, int nslices, int threads, size_t smem,
                       cudaStream_t st) {
  if (nslices <= 0) return cudaSuccess;
  if (smem == 0 || threads <= 0) return cudaErrorInvalidValue;   // shape without a plan
  void (*kern)(const JacobiParams<T>) = jacobi_kernel<T, 1, 0>;
  if constexpr (sizeof(T) == 4) {
    if (P.ldS % 4 == 0 && P.mm % 4 == 0 && P.rc % 4 == 0) {
      kern = jacobi_kernel<T, 4, 0>;
      if (P.tile == 1 && P.mm <= 128)
        kern = P.vlog ? jacobi_kernel<T, 4, 1, 32, true> : jacobi_kernel<T, 4, 1>;
      if (P.tile == 2 && P.mm <= 256)
        kern = P.vlog ? jacobi_kernel<T, 4, 2, 32, true> : jacobi_kernel<T, 4, 2>;
      if (P.tile > 0 && P.g < 32) {
        // partial-warp groups of g lanes, tile float4 rows per lane: whole
        // slice in shared memory, mm <= 4 g tile rows, at most 4 warps (the
        // size of the kernel's rotation record)
        if (P.mm > 4 * P.g * P.tile || P.rc > 2 * P.bcols || threads > 128 || threads % 32)
          return cudaErrorInvalidValue;
        if (P.g == 16 && P.tile == 1) kern = jacobi_kernel<T, 4, 1, 16>;
        else if (P.g == 8 && P.tile == 1) kern = jacobi_kernel<T, 4, 1, 8>;
        else if (P.g == 8 && P.tile == 2) kern = jacobi_kernel<T, 4, 2, 8>;
        else if (P.g == 4 && P.tile == 2) kern = jacobi_kernel<T, 4, 2, 4>;
        else return cudaErrorInvalidValue;
      }
    }
  }
  if (P.vlog) {
    // the log needs the whole-warp register-tiled form
    bool rec_kern = false;
    if constexpr (sizeof(T) == 4)
      rec_kern = kern == jacobi_kernel<T, 4, 1, 32, true> || kern == jacobi_kernel<T, 4, 2, 32, true>;
    if (!rec_kern || P.desc || !P.order || !P.vlsweeps) return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nslices, threads, smem, st>>>(P);
  return cudaGetLastError();
}

template <typename T>
JacobiPlan jacobi_coop_plan(int rows, int max_smem) {
  JacobiPlan pl{};
  pl.trans = 0;
  pl.mm = pl.rc = rows;
  pl.vec = 1;
  pl.bcols = 4;
  const int len = 2 * rows;
  pl.ldS = len + 1;
  int p2 = 1;
  while (p2 < rows) p2 <<= 1;
  pl.sort_n = p2;
  pl.g = rows >= 64 ? 32 : 16;
  pl.threads = pl.bcols * pl.g;
  const int nblk = (rows + pl.bcols - 1) / pl.bcols;
  pl.block_mode = (nblk + 1) / 2;   // CTAs of the launch
  pl.tile = 0;
  pl.smem = (((size_t)2 * pl.bcols * pl.ldS * sizeof(T) + 15) & ~(size_t)15) +
            (size_t)p2 * (sizeof(double) + sizeof(int));
  if (pl.smem > (size_t)max_smem) pl.smem = 0;
  // every CTA of the launch must be resident at once (the rounds wait on one
  // another): otherwise the plan is unusable and the caller takes the
  // single-CTA kernel
  if (pl.smem > 0) {
    void (*kern)(const JacobiParams<T>, const CoopSync) = jacobi_coop_kernel<T>;
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) !=
            cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, pl.threads, pl.smem) !=
            cudaSuccess ||
        (int64_t)per_sm * nsm < pl.block_mode) {
      cudaGetLastError();
      pl.smem = 0;
    }
  }
  return pl;
}

template <typename T>
cudaError_t jacobi_svd_coop(const JacobiParams<T>& P, const JacobiPlan& pl, const CoopSync& cs,
                            cudaStream_t st) {
  if (pl.smem == 0 || pl.block_mode < 1) return cudaErrorInvalidValue;
  if (P.mm != P.rc || P.bcols != pl.bcols || P.g != pl.g || P.trans != 0)
    return cudaErrorInvalidValue;
  void (*kern)(const JacobiParams<T>, const CoopSync) = jacobi_coop_kernel<T>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, pl.threads, pl.smem)) !=
      cudaSuccess)
    return e;
  if ((int64_t)per_sm * nsm < pl.block_mode) return cudaErrorCooperativeLaunchTooLarge;
  JacobiParams<T> p = P;
  CoopSync c = cs;
  void* args[] = {&p, &c};
  if ((e = cudaMemsetAsync(cs.bar, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(cs.abort_flag, 0, sizeof(int), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(cs.rot, 0, sizeof(int) * (size_t)P.max_sweeps, st)) != cudaSuccess)
    return e;
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(pl.block_mode), dim3(pl.threads), args,
                                  pl.smem, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

JacobiPlan jacobi_cluster_plan(int rows, int max_smem) {
  JacobiPlan pl{};
  pl.trans = 0;
  pl.mm = pl.rc = rows;
  pl.vec = 4;
  pl.ldS = 2 * rows + 4;
  const int nblk = 2 * kClusterCtas;
  pl.bcols = (((rows + nblk - 1) / nblk) + 3) & ~3;
  int p2 = 1;
  while (p2 < rows) p2 <<= 1;
  pl.sort_n = p2;
  pl.g = 32;
  pl.threads = 32 * kClusterWarps;
  pl.tile = rows <= 128 ? 1 : 2;
  pl.block_mode = kClusterCtas;   // CTAs of the cluster
  pl.smem = (((size_t)2 * pl.bcols * pl.ldS * sizeof(float) + 15) & ~(size_t)15) +
            (size_t)p2 * (sizeof(double) + sizeof(int)) + 16;
  // fp32 float4 columns, a tile per 4 columns, at least one full tile per block
  if (rows % 4 || rows > 256 || rows < 8 * kClusterCtas || pl.smem + 3072 > (size_t)max_smem)
    pl.smem = 0;
  return pl;
}

cudaError_t jacobi_svd_cluster(const JacobiParams<float>& P, const JacobiPlan& pl, int* rot_count,
                               cudaStream_t st) {
  if (pl.smem == 0 || P.mm != P.rc || P.trans != 0 || P.bcols != pl.bcols || P.ldS != pl.ldS ||
      !P.W || !rot_count)
    return cudaErrorInvalidValue;
  void (*kern)(const JacobiParams<float>, int*) =
      pl.tile == 2 ? jacobi_cluster_kernel<2> : jacobi_cluster_kernel<1>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(rot_count, 0, sizeof(int) * (size_t)P.max_sweeps, st)) != cudaSuccess)
    return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(pl.threads);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  JacobiParams<float> p = P;
  if ((e = cudaLaunchKernelEx(&cfg, kern, p, rot_count)) != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t jacobi_v_replay(const JacobiParams<float>& P, const JacobiPlan& pl, const int* ranks,
                            int nslices, cudaStream_t st) {
  if (nslices <= 0) return cudaSuccess;
  if (!pl.rec || !P.vlog || !P.order || !P.vlsweeps || !P.V || P.rc != pl.rc)
    return cudaErrorInvalidValue;
  int nps = 0, rmax = 0, kmax = 0;
  vlog_dims(pl.rc, pl.bcols, pl.rc <= 2 * pl.bcols, nps, rmax, kmax);
  // (rounds, tasks and columns held in bytes and 16-bit words)
  if (nps < 1 || rmax > 255 || kmax > 255 || pl.rc >= 0xffff) return cudaErrorInvalidValue;
  const size_t smem = vr_smem_bytes(pl.rc, pl.bcols);
  cudaError_t e = cudaFuncSetAttribute(jacobi_v_replay_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (pl.rc > VR_SPLIT * VR_COLS) return cudaErrorInvalidValue;
  jacobi_v_replay_kernel<<<dim3(nslices, VR_SPLIT), VR_THREADS, smem, st>>>(P, pl.bcols, ranks);
  return cudaGetLastError();
}

template JacobiPlan jacobi_plan<float>(int, int, int, bool);
template JacobiPlan jacobi_plan<double>(int, int, int, bool);
template std::vector<JacobiPlan> jacobi_plan_candidates<float>(int, int, int, bool);
template std::vector<JacobiPlan> jacobi_plan_candidates<double>(int, int, int, bool);
template cudaError_t jacobi_svd<float>(const JacobiParams<float>&, int, int, size_t, cudaStream_t);
template cudaError_t jacobi_svd<double>(const JacobiParams<double>&, int, int, size_t, cudaStream_t);

template JacobiPlan jacobi_coop_plan<double>(int, int);
template JacobiPlan jacobi_coop_plan<float>(int, int);
template cudaError_t jacobi_svd_coop<double>(const JacobiParams<double>&, const JacobiPlan&,
                                             const CoopSync&, cudaStream_t);
template cudaError_t jacobi_svd_coop<float>(const JacobiParams<float>&, const JacobiPlan&,
                                            const CoopSync&, cudaStream_t);

}  // namespace sma
