// tcgen05 GEMM with 3-piece bf16 split operands (mixed path).
//
//   C[i * ldc + j] = sum_k A(i, k) B(j, k),   i < M, j < N,
//
// where A and B are fp32 matrices given as three bf16 planes each
// (x = hi + mid + lo, hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid)),
// stored K-major ([row][Kp], Kp a multiple of 64, zero padded).  The six
// products with i + j <= 2 (hi hi, hi mid, mid hi, hi lo, lo hi, mid mid)
// are accumulated in fp32 in tensor memory, which carries the operands'
// fp32 accuracy.
//
// One CTA per 128 x 256 tile of C: an elected thread of warp 0
// streams (A plane, B plane) tile pairs with TMA (3-D tensor maps, 128B
// swizzle) through a 4-stage mbarrier ring; an elected thread of warp 1
// issues tcgen05.mma (M128 x N256 x K16) into tensor memory.
//
// Accumulation is chunked: the tensor core adds each step into the fp32
// accumulator with about half an ulp of error, which over the long K of the
// Kronecker-sum matvec (tens of thousands of steps) would cost most of the
// fp32 accuracy.  So every CHUNK k-blocks start a fresh accumulator (two TMEM
// buffers, ping-pong), and eight epilogue warps (warps 2-9) drain finished
// chunks with tcgen05.ld into fp32 register sums (IEEE round-to-nearest),
// 128 columns per thread, while the other buffer fills.  Every wait is
// bounded: on timeout the kernel sets an error bit, drains what it issued,
// frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "tc_gemm.cuh"

namespace sma {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4, CHUNK = 2;
constexpr int A_BYTES = BM * BK * 2;        // 16 KB
constexpr int B_BYTES = BN * BK * 2;        // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int TMEM_COLS = 512;  // two 256-column accumulators
constexpr uint64_t WAIT_NS = 4000000000ull;  // 4 s per wait
constexpr uint32_t WAIT_ITERS = 1u << 30;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
static_assert(THREADS == 320, "two control warps and eight epilogue warps");

__constant__ int kProdA[6] = {0, 0, 1, 0, 2, 1};
__constant__ int kProdB[6] = {0, 1, 0, 2, 0, 1};
// fp16 two-piece split (x = hi + lo): hi hi, hi lo, lo hi
__constant__ int kProdA3[3] = {0, 0, 1};
__constant__ int kProdB3[3] = {0, 1, 0};
template <int NP> __device__ __forceinline__ int prod_a(int pr) {
  return NP == 6 ? kProdA[pr] : kProdA3[pr];
}
template <int NP> __device__ __forceinline__ int prod_b(int pr) {
  return NP == 6 ? kProdB[pr] : kProdB3[pr];
}

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = gtimer();
  for (uint32_t i = 0; i < WAIT_ITERS; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (gtimer() - t0 > WAIT_NS) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(saddr(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// K-major operand tile with 128-byte swizzle: rows of 128 B, 8-row atoms of
// 1024 B (stride byte offset), descriptor version 1, layout type 2.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused here), 16 B
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}
// kind::f16 instruction descriptor: fp32 accumulator, bf16 (or, with f16,
// fp16) A and B, both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc16(int M, int N, bool f16) {
  return (1u << 4) | (f16 ? 0u : ((1u << 7) | (1u << 10))) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t dtm, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          saddr(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
  int M, N, Kp;
  float* C;
  int64_t ldc;
  int col_major;  // 0: C[i * ldc + j]; 1: C[i + j * ldc]
  int* err;
  const float* scale;   // C is multiplied by *scale when set
};

// NP = 6: three bf16 planes per operand, six products; NP = 3: two fp16
// planes per operand (scaled into fp16's range by the caller), three products.
template <int NP>
__global__ void __launch_bounds__(THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               const TcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* tiles = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(tiles + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;   // chunk in buffer b complete (MMA commit)
  uint64_t* acce = accf + 2;         // buffer b drained (one arrive per epilogue warp)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int nkb = args.Kp / BK;
  const int total = nkb * NP;
  const int nch = (nkb + CHUNK - 1) / CHUNK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: (A plane, B plane) tiles for iteration it = 6 kb + product
    int issued = 0;
    for (int it = 0; it < total; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const int kb = it / NP, pr = it % NP;
      uint8_t* st = tiles + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_3d(st, &mapA, &full[s], kb * BK, m0, prod_a<NP>(pr));
      tma_load_3d(st + A_BYTES, &mapB, &full[s], kb * BK, n0, prod_b<NP>(pr));
      issued = it + 1;
    }
    // drain: the copies of the last stages must land before the CTA exits
    for (int it = (issued > STAGES ? issued - STAGES : 0); it < issued; ++it)
      if (!mbar_wait(&full[it % STAGES], (uint32_t)(it / STAGES) & 1u)) *abort_flag = 1;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: chunk c (CHUNK k-blocks) accumulates into buffer c & 1
    const uint32_t id = idesc16(BM, BN, NP == 3);
    int it = 0;
    for (int c = 0; c < nch && !*abort_flag; ++c) {
      const int b = c & 1;
      if (c >= 2 && !mbar_wait(&acce[b], (uint32_t)((c >> 1) - 1) & 1u)) {
        *abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t dt = tmem + (uint32_t)(b * BN);
      const int it_end = min(total, (c + 1) * CHUNK * NP);
      bool first = true;
      for (; it < it_end; ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        if (!mbar_wait(&full[s], ph)) {
          *abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t a0 = saddr(tiles + s * STAGE_BYTES);
        const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          mma(dt, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), id, first ? 0u : 1u);
          first = false;
        }
        mma_commit(&empty[s]);
      }
      mma_commit(&accf[b]);  // arrives when this chunk's MMAs have completed
    }
  } else if (warp >= 2) {
    // epilogue: warp e drains rows of quadrant (warp & 3), columns half h
    const int e = warp - 2;
    const int q = warp & 3, hc = e >> 2;
    const int row = q * 32 + lane;
    const int grow = m0 + row;
    float acc[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) acc[j] = 0.f;
    for (int c = 0; c < nch; ++c) {
      const int b = c & 1;
      const bool ok = mbar_wait(&accf[b], (uint32_t)(c >> 1) & 1u);
      fence_after();
      if (!ok) *abort_flag = 1;
      __syncwarp();
      if (*abort_flag) break;
#pragma unroll
      for (int part = 0; part < 4; ++part) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + hc * 128 + part * 32), r);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[part * 32 + j] += __uint_as_float(r[j]);
      }
      fence_before();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&acce[b])) : "memory");
    }
    const float sc = args.scale ? *args.scale : 1.f;   // (a power of two: exact)
    if (!*abort_flag && grow < args.M && args.col_major) {
      // lanes hold consecutive rows: each store instruction is coalesced
      const int c0 = n0 + hc * 128;
      const int nv = args.N - c0;
      float* dst = args.C + grow + (int64_t)c0 * args.ldc;
#pragma unroll
      for (int j = 0; j < 128; ++j)
        if (j < nv) dst[(int64_t)j * args.ldc] = acc[j] * sc;
    } else if (!*abort_flag && grow < args.M) {
      const int c0 = n0 + hc * 128;
      float* dst = args.C + (int64_t)grow * args.ldc + c0;
      const int nv = args.N - c0;
      if (nv >= 128 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
        for (int j = 0; j < 128; j += 4)
          *reinterpret_cast<float4*>(dst + j) =
              make_float4(acc[j] * sc, acc[j + 1] * sc, acc[j + 2] * sc, acc[j + 3] * sc);
      } else {
#pragma unroll
        for (int j = 0; j < 128; ++j)
          if (j < nv) dst[j] = acc[j] * sc;
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(args.err, SMA_STATUS_BIT(SMA_ERR_TIMEOUT));
}

// ---- mid-index contraction of the Kronecker-sum matvec ----------------------
// Z(i, j) = sum_k A(i, k) B(j, k) over the six split products for a short K
// (Kq = a few k-blocks), written as three bf16 planes straight into the
// operand layout of the long-K product: row i = c + n s, column j = a + ell t
// go to Z[p * plane + (a + ell s) * Kp + c + n t].  One CTA per 128 x 256
// tile, two stages (two CTAs per SM, so one CTA's epilogue overlaps the other
// CTA's loads and MMAs), 256 TMEM columns.  The kernel is bound by writing the
// planes: sixteen epilogue warps (four per TMEM lane quadrant, a quarter of
// the columns each) keep enough stores in flight, and the stores are
// streaming (.cs), since the planes are read back only by the next kernel.
constexpr int MID_STAGES = 2;
constexpr int MID_EPI_WARPS = 16;
constexpr int MID_THREADS = 64 + 32 * MID_EPI_WARPS;
constexpr int MID_TMEM = 256;
constexpr int MID_SMEM = MID_STAGES * STAGE_BYTES + 1024 + 256;

struct MidArgs {
  int M, N, Kq, n, ell;
  int pairs;   // n even and Z, Kp, plane allow 32-bit stores of two rows
  int64_t Kp, plane;
  uint16_t* Z;          // bf16 (three planes) or fp16 (two planes) elements
  int* err;
  const float* mult;    // fp16 form: Z is scaled by *mult before the split
};

// x = hi + lo in fp16 (x already scaled into fp16's range)
__device__ __forceinline__ void split2h(float x, uint16_t& hi, uint16_t& lo) {
  const __half h = __float2half_rn(x);
  hi = __half_as_ushort(h);
  lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& hi, __nv_bfloat16& mid,
                                       __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(hi);
  mid = __float2bfloat16_rn(r1);
  lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

template <int NP>
__global__ void __launch_bounds__(MID_THREADS)
tc_mid_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const MidArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* tiles = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(tiles + MID_STAGES * STAGE_BYTES);
  uint64_t* empty = full + MID_STAGES;
  uint64_t* accf = empty + MID_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int total = (args.Kq / BK) * NP;

  if (threadIdx.x == 0) {
    for (int s = 0; s < MID_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tmem_slot)),
                 "r"(MID_TMEM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int it = 0; it < total; ++it) {
      const int s = it % MID_STAGES;
      const uint32_t ph = (uint32_t)(it / MID_STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const int kb = it / NP, pr = it % NP;
      uint8_t* st = tiles + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_3d(st, &mapA, &full[s], kb * BK, m0, prod_a<NP>(pr));
      tma_load_3d(st + A_BYTES, &mapB, &full[s], kb * BK, n0, prod_b<NP>(pr));
      issued = it + 1;
    }
    for (int it = (issued > MID_STAGES ? issued - MID_STAGES : 0); it < issued; ++it)
      if (!mbar_wait(&full[it % MID_STAGES], (uint32_t)(it / MID_STAGES) & 1u)) *abort_flag = 1;
  } else if (warp == 1 && lane == 0) {
    const uint32_t id = idesc16(BM, BN, NP == 3);
    for (int it = 0; it < total; ++it) {
      const int s = it % MID_STAGES;
      const uint32_t ph = (uint32_t)(it / MID_STAGES) & 1u;
      if (*abort_flag || !mbar_wait(&full[s], ph)) {
        *abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t a0 = saddr(tiles + s * STAGE_BYTES);
      const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        mma(tmem, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), id, (it > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(accf);  // arrives when every MMA issued above has completed
  } else if (warp >= 2) {
    const int q = warp & 3;
    const int hp = (warp - 2) >> 2;   // which quarter of the columns
    const int grow = m0 + q * 32 + lane;
    const float mult = (NP == 3 && args.mult) ? *args.mult : 1.f;
    const bool ok = mbar_wait(accf, 0u);
    fence_after();
    if (!ok) *abort_flag = 1;
    __syncwarp();
    if (!*abort_flag && args.pairs) {
      // rows c and c + 1 (an even and an odd lane) are adjacent in Z: the lane
      // pair swaps one value per column pair so that each lane holds both rows
      // of one column, splits them together and stores 32-bit words
      const bool odd = lane & 1;
      const int row0 = grow - (odd ? 1 : 0);                // the pair's first row
      const int c0 = row0 % args.n, s0 = row0 / args.n;
      const bool rows_ok = row0 + 1 < args.M;
      const int64_t rbase = (int64_t)args.ell * s0 * args.Kp + c0;
#pragma unroll 1
      for (int part = hp * (BN / 128); part < (hp + 1) * (BN / 128); ++part) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(part * 32), r);
        const int g0 = n0 + part * 32;
        // (a, t) of the even column of each pair, advanced by two per pair
        int t = g0 / args.ell, a = g0 - t * args.ell;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          const float xe = __uint_as_float(r[2 * kk]), xo = __uint_as_float(r[2 * kk + 1]);
          const float got = __shfl_xor_sync(0xffffffffu, odd ? xe : xo, 1);
          const float v0 = odd ? got : xe;                  // row0 at this lane's column
          const float v1 = odd ? xo : got;                  // row0 + 1
          int aj = a + (odd ? 1 : 0), tj = t;
          if (aj >= args.ell) {
            aj -= args.ell;
            ++tj;
          }
          const int gj = g0 + 2 * kk + (odd ? 1 : 0);
          if (rows_ok && gj < args.N) {
            uint16_t* d = args.Z + rbase + (int64_t)aj * args.Kp + (int64_t)args.n * tj;
            if (NP == 3) {
              uint16_t h0, l0, h1, l1;
              split2h(v0 * mult, h0, l0);
              split2h(v1 * mult, h1, l1);
              const uint32_t wh = (uint32_t)h0 | ((uint32_t)h1 << 16);
              const uint32_t wl = (uint32_t)l0 | ((uint32_t)l1 << 16);
              asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(d), "r"(wh) : "memory");
              asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(d + args.plane), "r"(wl) : "memory");
            } else {
              __nv_bfloat16 h0, m0_, l0, h1, m1, l1;
              split3(v0, h0, m0_, l0);
              split3(v1, h1, m1, l1);
              const uint32_t wh = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
              const uint32_t wm = (uint32_t)__bfloat16_as_ushort(m0_) | ((uint32_t)__bfloat16_as_ushort(m1) << 16);
              const uint32_t wl = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
              asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(d), "r"(wh) : "memory");
              asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(d + args.plane), "r"(wm) : "memory");
              asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(d + 2 * args.plane), "r"(wl) : "memory");
            }
          }
          a += 2;
          while (a >= args.ell) {
            a -= args.ell;
            ++t;
          }
        }
      }
    }
    if (!*abort_flag && !args.pairs) {
      const int c = grow % args.n, s = grow / args.n;
      const int64_t rbase = (int64_t)args.ell * s * args.Kp + c;
#pragma unroll 1
      for (int part = hp * (BN / 128); part < (hp + 1) * (BN / 128); ++part) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(part * 32), r);
        const int g0 = n0 + part * 32;
        int t = g0 / args.ell, a = g0 - t * args.ell;
        if (grow < args.M) {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            if (g0 + jj < args.N) {
              uint16_t* d = args.Z + rbase + (int64_t)a * args.Kp + (int64_t)args.n * t;
              if (NP == 3) {
                uint16_t hi, lo;
                split2h(__uint_as_float(r[jj]) * mult, hi, lo);
                asm volatile("st.global.cs.u16 [%0], %1;" ::"l"(d), "h"(hi) : "memory");
                asm volatile("st.global.cs.u16 [%0], %1;" ::"l"(d + args.plane), "h"(lo) : "memory");
              } else {
                __nv_bfloat16 hi, mi, lo;
                split3(__uint_as_float(r[jj]), hi, mi, lo);
                asm volatile("st.global.cs.u16 [%0], %1;" ::"l"(d), "h"(__bfloat16_as_ushort(hi)) : "memory");
                asm volatile("st.global.cs.u16 [%0], %1;" ::"l"(d + args.plane), "h"(__bfloat16_as_ushort(mi)) : "memory");
                asm volatile("st.global.cs.u16 [%0], %1;" ::"l"(d + 2 * args.plane), "h"(__bfloat16_as_ushort(lo)) : "memory");
              }
            }
            if (++a == args.ell) {
              a = 0;
              ++t;
            }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(MID_TMEM));
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(args.err, SMA_STATUS_BIT(SMA_ERR_TIMEOUT));
}

// fp32 -> three bf16 planes, with transposition: plane[p][j * Kp + k] from
// src[j * s_rs + k * s_cs] for j < R, k < K (32 x 32 tiles through shared
// memory so both sides are coalesced when s_rs == 1).
__global__ void split_transpose_kernel(const float* __restrict__ src, int64_t s_rs, int64_t s_cs,
                                       int R, int K, int64_t Kp, __nv_bfloat16* __restrict__ dst,
                                       int64_t plane, int64_t src_bs, int64_t dst_bs) {
  __shared__ float tile[32][33];
  const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  src += (int64_t)blockIdx.z * src_bs;
  dst += (int64_t)blockIdx.z * dst_bs;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int k = k0 + i, j = j0 + threadIdx.x;
    tile[i][threadIdx.x] = (j < R && k < K) ? src[(int64_t)j * s_rs + (int64_t)k * s_cs] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int j = j0 + i, k = k0 + threadIdx.x;
    if (j < R && k < K) {
      const float x = tile[threadIdx.x][i];
      const __nv_bfloat16 hi = __float2bfloat16_rn(x);
      const float r1 = x - __bfloat162float(hi);
      const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
      const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
      const int64_t o = (int64_t)j * Kp + k;
      dst[o] = hi;
      dst[o + plane] = mid;
      dst[o + 2 * plane] = lo;
    }
  }
}

// fp32 -> two fp16 planes of x * (*scale), with transposition (as above)
__global__ void split2_transpose_kernel(const float* __restrict__ src, int64_t s_rs, int64_t s_cs,
                                        int R, int K, int64_t Kp, uint16_t* __restrict__ dst,
                                        int64_t plane, int64_t src_bs, int64_t dst_bs,
                                        const float* __restrict__ scale) {
  __shared__ float tile[32][33];
  const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const float sc = *scale;
  src += (int64_t)blockIdx.z * src_bs;
  dst += (int64_t)blockIdx.z * dst_bs;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int k = k0 + i, j = j0 + threadIdx.x;
    tile[i][threadIdx.x] = (j < R && k < K) ? src[(int64_t)j * s_rs + (int64_t)k * s_cs] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int j = j0 + i, k = k0 + threadIdx.x;
    if (j < R && k < K) {
      uint16_t hi, lo;
      split2h(tile[threadIdx.x][i] * sc, hi, lo);
      const int64_t o = (int64_t)j * Kp + k;
      dst[o] = hi;
      dst[o + plane] = lo;
    }
  }
}

// The same planes from a source whose k is contiguous (s_cs = 1): rows j,
// k along the threads, coalesced on both sides without a transposition.
__global__ void split2_rows_kernel(const float* __restrict__ src, int64_t s_rs, int R, int K,
                                   int64_t Kp, uint16_t* __restrict__ dst, int64_t plane,
                                   const float* __restrict__ scale) {
  const float sc = *scale;
  const int64_t tot = (int64_t)R * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / K, k = e - j * K;
    uint16_t hi, lo;
    split2h(src[j * s_rs + k] * sc, hi, lo);
    dst[j * Kp + k] = hi;
    dst[j * Kp + k + plane] = lo;
  }
}

// *out = max(*out, max |a[r rs + c cs]|) over r < rows, c < cols, on the
// bit patterns of non-negative floats (NaN ignored)
__global__ void absmax_kernel(const float* __restrict__ a, int64_t rows, int64_t cols, int64_t rs,
                              int64_t cs, unsigned* __restrict__ out) {
  float m = 0.f;
  const int64_t tot = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, r = e - c * rows;
    m = fmaxf(m, fabsf(a[r * rs + c * cs]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

// *out = max over (a, j) of sum_b |C_j[a, b]|, C_j[a, b] = C[a + ell b + ell q j]
__global__ void rowl1max_kernel(const float* __restrict__ C, int ell, int q, int nt,
                                unsigned* __restrict__ out) {
  float m = 0.f;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ell * nt;
       idx += gridDim.x * blockDim.x) {
    const int a = idx % ell, j = idx / ell;
    const float* c = C + a + (int64_t)ell * q * j;
    float sum = 0.f;
    for (int b = 0; b < q; ++b) sum += fabsf(c[(int64_t)ell * b]);
    m = fmaxf(m, sum);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

// 2^(14 - e) for a maximum m = 1.x 2^e (1 for m = 0 or not finite): m s < 2^15
__device__ __forceinline__ float pow2_scale(float m) {
  if (!(m > 0.f) || !isfinite(m)) return 1.f;
  const int e = max(-100, min(100, ilogbf(m)));
  return ldexpf(1.f, 14 - e);
}
// mx: max |X|, max |C|, max row L1 of C, max |D|; sc: s_X, s_C, s_D, s_Z,
// s_Z / (s_X s_C) (the mid product's factor), 1 / (s_Z s_D) (the output's);
// |Z| <= max |X| max row L1 (C), so Z s_Z < 2^15 as well.  All powers of two.
__global__ void f16_scales_kernel(const unsigned* __restrict__ mx, float* __restrict__ sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const float mX = __uint_as_float(mx[0]), mC = __uint_as_float(mx[1]);
  const float mL = __uint_as_float(mx[2]), mD = __uint_as_float(mx[3]);
  const float sX = pow2_scale(mX), sC = pow2_scale(mC), sD = pow2_scale(mD);
  const float sZ = pow2_scale(mX * mL);
  sc[0] = sX;
  sc[1] = sC;
  sc[2] = sD;
  sc[3] = sZ;
  sc[4] = sZ / (sX * sC);
  sc[5] = 1.f / (sZ * sD);
}

// s = the scale of one operand; out = {s_B, 1 / (s_A s_B)} of a product
__global__ void f16_scale1_kernel(const unsigned* __restrict__ mx, float* __restrict__ s) {
  if (threadIdx.x == 0 && blockIdx.x == 0) s[0] = pow2_scale(__uint_as_float(mx[0]));
}
__global__ void f16_scale_out_kernel(const unsigned* __restrict__ mxA,
                                     const unsigned* __restrict__ mxB, float* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const float sA = pow2_scale(__uint_as_float(mxA[0])), sB = pow2_scale(__uint_as_float(mxB[0]));
  out[0] = sB;
  out[1] = 1.f / (sA * sB);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

bool make_map(CUtensorMap* map, const void* planes, int rows, int64_t Kp, int box_rows,
              int nplanes = 3, bool f16 = false) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)nplanes};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * rows};
  const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
            const_cast<void*>(planes), dims,
            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tc_gemm_available(int major, int minor) {
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

int64_t tc_pad_k(int64_t K) { return (K + BK - 1) / BK * BK; }

cudaError_t tc_split_transpose(const float* src, int64_t s_rs, int64_t s_cs, int R, int K,
                               int64_t Kp, __nv_bfloat16* dst, cudaStream_t st) {
  if (R <= 0 || K <= 0) return cudaSuccess;
  dim3 grid((R + 31) / 32, (K + 31) / 32);
  split_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(src, s_rs, s_cs, R, K, Kp, dst,
                                                      (int64_t)R * Kp, 0, 0);
  return cudaGetLastError();
}

cudaError_t tc_split_transpose_batched(const float* src, int64_t s_rs, int64_t s_cs, int R, int K,
                                       int64_t Kp, int nbatch, int64_t src_bs, int64_t dst_bs,
                                       int64_t plane, __nv_bfloat16* dst, cudaStream_t st) {
  if (R <= 0 || K <= 0 || nbatch <= 0) return cudaSuccess;
  if (nbatch > 65535) return cudaErrorInvalidValue;
  dim3 grid((R + 31) / 32, (K + 31) / 32, nbatch);
  split_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(src, s_rs, s_cs, R, K, Kp, dst, plane,
                                                      src_bs, dst_bs);
  return cudaGetLastError();
}

cudaError_t tc_gemm_planes(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N,
                           int64_t Kp, float* C, int64_t ldc, int* err, cudaStream_t st,
                           bool col_major) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (Kp % BK != 0 || Kp <= 0 || (N + BN - 1) / BN > 65535) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, Kp, BM) || !make_map(&mb, B, N, Kp, BN)) return cudaErrorInvalidValue;
  const cudaError_t attr = cudaFuncSetAttribute(
      tc_gemm_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  TcArgs a{M, N, (int)Kp, C, ldc, col_major ? 1 : 0, err, nullptr};
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
  tc_gemm_kernel<6><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, a);
  return cudaGetLastError();
}

cudaError_t tc_gemm_planes_f16(const uint16_t* A, const uint16_t* B, int M, int N, int64_t Kp,
                               float* C, int64_t ldc, const float* scale, int* err,
                               cudaStream_t st, bool col_major) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (Kp % BK != 0 || Kp <= 0 || (N + BN - 1) / BN > 65535) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, Kp, BM, 2, true) || !make_map(&mb, B, N, Kp, BN, 2, true))
    return cudaErrorInvalidValue;
  const cudaError_t attr = cudaFuncSetAttribute(
      tc_gemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  TcArgs a{M, N, (int)Kp, C, ldc, col_major ? 1 : 0, err, scale};
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
  tc_gemm_kernel<3><<<grid, THREADS, SMEM_BYTES, st>>>(ma, mb, a);
  return cudaGetLastError();
}

cudaError_t tc_mid_planes(const __nv_bfloat16* A, int M, const __nv_bfloat16* B, int N, int64_t Kq,
                          __nv_bfloat16* Z, int64_t Kp, int64_t zplane, int n, int ell, int* err,
                          cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (Kq % BK != 0 || Kq <= 0 || n <= 0 || ell <= 0) return cudaErrorInvalidValue;
  if ((M + BM - 1) / BM > 0x7fffffff || (N + BN - 1) / BN > 65535) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, Kq, BM) || !make_map(&mb, B, N, Kq, BN)) return cudaErrorInvalidValue;
  const cudaError_t attr = cudaFuncSetAttribute(
      tc_mid_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, MID_SMEM);
  if (attr != cudaSuccess) return attr;
  const int pairs = (n % 2 == 0 && M % 2 == 0 && Kp % 2 == 0 && zplane % 2 == 0 &&
                     (reinterpret_cast<uintptr_t>(Z) & 3) == 0)
                        ? 1
                        : 0;
  MidArgs a{M, N, (int)Kq, n, ell, pairs, Kp, zplane, reinterpret_cast<uint16_t*>(Z), err,
            nullptr};
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
  tc_mid_kernel<6><<<grid, MID_THREADS, MID_SMEM, st>>>(ma, mb, a);
  return cudaGetLastError();
}

cudaError_t tc_mid_planes_f16(const uint16_t* A, int M, const uint16_t* B, int N, int64_t Kq,
                              uint16_t* Z, int64_t Kp, int64_t zplane, int n, int ell,
                              const float* mult, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (Kq % BK != 0 || Kq <= 0 || n <= 0 || ell <= 0 || !mult) return cudaErrorInvalidValue;
  if ((M + BM - 1) / BM > 0x7fffffff || (N + BN - 1) / BN > 65535) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, Kq, BM, 2, true) || !make_map(&mb, B, N, Kq, BN, 2, true))
    return cudaErrorInvalidValue;
  const cudaError_t attr = cudaFuncSetAttribute(
      tc_mid_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, MID_SMEM);
  if (attr != cudaSuccess) return attr;
  const int pairs = (n % 2 == 0 && M % 2 == 0 && Kp % 2 == 0 && zplane % 2 == 0 &&
                     (reinterpret_cast<uintptr_t>(Z) & 3) == 0)
                        ? 1
                        : 0;
  MidArgs a{M, N, (int)Kq, n, ell, pairs, Kp, zplane, Z, err, mult};
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
  tc_mid_kernel<3><<<grid, MID_THREADS, MID_SMEM, st>>>(ma, mb, a);
  return cudaGetLastError();
}

cudaError_t tc_split2_transpose_batched(const float* src, int64_t s_rs, int64_t s_cs, int R, int K,
                                        int64_t Kp, int nbatch, int64_t src_bs, int64_t dst_bs,
                                        int64_t plane, const float* scale, uint16_t* dst,
                                        cudaStream_t st) {
  if (R <= 0 || K <= 0 || nbatch <= 0) return cudaSuccess;
  if (nbatch > 65535 || !scale) return cudaErrorInvalidValue;
  if (s_cs == 1 && s_rs != 1 && nbatch == 1) {
    const int64_t tot = (int64_t)R * K;
    const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 8192);
    split2_rows_kernel<<<blocks, 256, 0, st>>>(src, s_rs, R, K, Kp, dst, plane, scale);
    return cudaGetLastError();
  }
  dim3 grid((R + 31) / 32, (K + 31) / 32, nbatch);
  split2_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(src, s_rs, s_cs, R, K, Kp, dst, plane,
                                                       src_bs, dst_bs, scale);
  return cudaGetLastError();
}

cudaError_t tc_absmax(const float* a, int64_t rows, int64_t cols, int64_t ld, unsigned* out,
                      cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned), st);
  if (e != cudaSuccess || rows <= 0 || cols <= 0) return e;
  const int64_t tot = rows * cols;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 2048);
  absmax_kernel<<<blocks, 256, 0, st>>>(a, rows, cols, 1, ld, out);
  return cudaGetLastError();
}

cudaError_t tc_absmax_strided(const float* a, int64_t rows, int64_t cols, int64_t rs, int64_t cs,
                              unsigned* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned), st);
  if (e != cudaSuccess || rows <= 0 || cols <= 0) return e;
  if (cs == 1 && rs != 1) {   // the unit stride along the threads
    std::swap(rows, cols);
    std::swap(rs, cs);
  }
  const int64_t tot = rows * cols;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 2048);
  absmax_kernel<<<blocks, 256, 0, st>>>(a, rows, cols, rs, cs, out);
  return cudaGetLastError();
}

cudaError_t tc_f16_scale1(const unsigned* mx, float* s, cudaStream_t st) {
  f16_scale1_kernel<<<1, 32, 0, st>>>(mx, s);
  return cudaGetLastError();
}

cudaError_t tc_f16_scale_out(const unsigned* mxA, const unsigned* mxB, float* out,
                             cudaStream_t st) {
  f16_scale_out_kernel<<<1, 32, 0, st>>>(mxA, mxB, out);
  return cudaGetLastError();
}

cudaError_t tc_rowl1max(const float* C, int ell, int q, int nt, unsigned* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned), st);
  if (e != cudaSuccess || ell <= 0 || q <= 0 || nt <= 0) return e;
  const int64_t tot = (int64_t)ell * nt;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 1024);
  rowl1max_kernel<<<blocks, 256, 0, st>>>(C, ell, q, nt, out);
  return cudaGetLastError();
}

cudaError_t tc_f16_scales(const unsigned* mx, float* sc, cudaStream_t st) {
  f16_scales_kernel<<<1, 32, 0, st>>>(mx, sc);
  return cudaGetLastError();
}

bool tc_gemm_eligible(const GemmParams<float>&) { return false; }
cudaError_t tc_gemm_bf16x3(const GemmParams<float>& g, cudaStream_t st) { return gemm<float>(g, st); }

}  // namespace sma
