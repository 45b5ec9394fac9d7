// Device helpers shared by the split-precision translation units
// (hfx_mixed.cu, hfx_t1umma.cu): index lookups, bf16 splitting, warp sums and
// the tcgen05 / mbarrier / bulk-copy wrappers (inline PTX).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "hfx_internal.h"

namespace hfx {
namespace dev {

__device__ __forceinline__ int rup16(int x) { return (x + 15) & ~15; }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// x = p0 + p1 (+ p2) + r with p_i bf16, each the round-to-nearest of what the
// earlier pieces leave.
template <int NP>
__device__ __forceinline__ void split_f(float x, uint16_t (&p)[NP]) {
  float r = x;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const __nv_bfloat16 h = __float2bfloat16_rn(r);
    p[i] = __bfloat16_as_ushort(h);
    r -= __bfloat162float(h);
  }
}

// The same split for four consecutive values, packed as 4 bf16 per piece
// (element 0 in the low half of .x).
template <int NP>
__device__ __forceinline__ void split4(const float (&x)[4], uint2 (&p)[NP]) {
  float r0 = x[0], r1 = x[1], r2 = x[2], r3 = x[3];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(r0, r1);
    const __nv_bfloat162 h23 = __floats2bfloat162_rn(r2, r3);
    p[i].x = *reinterpret_cast<const uint32_t*>(&h01);
    p[i].y = *reinterpret_cast<const uint32_t*>(&h23);
    r0 -= __low2float(h01);
    r1 -= __high2float(h01);
    r2 -= __low2float(h23);
    r3 -= __high2float(h23);
  }
}

__device__ __forceinline__ int ylut_get(const DevPlan& P, int i, int j, int r0, int r1, int r2) {
  if (r0 < -P.HY0 || r0 > P.HY0 || r1 < -P.HY1 || r1 > P.HY1 || r2 < -P.HY2 || r2 > P.HY2) return -1;
  const long long n0 = 2 * P.HY0 + 1, n1 = 2 * P.HY1 + 1, n2 = 2 * P.HY2 + 1;
  const long long idx = (((((long long)i * P.N + j) * n0 + (r0 + P.HY0)) * n1 + (r1 + P.HY1)) * n2) + (r2 + P.HY2);
  return P.ylut[idx];
}

__device__ __forceinline__ int dlut_get(const DevPlan& P, int i, int j, int r0, int r1, int r2) {
  if (r0 < -P.HD0 || r0 > P.HD0 || r1 < -P.HD1 || r1 > P.HD1 || r2 < -P.HD2 || r2 > P.HD2) return -1;
  const long long n0 = 2 * P.HD0 + 1, n1 = 2 * P.HD1 + 1, n2 = 2 * P.HD2 + 1;
  const long long idx = (((((long long)i * P.N + j) * n0 + (r0 + P.HD0)) * n1 + (r1 + P.HD1)) * n2) + (r2 + P.HD2);
  return P.dlut[idx];
}

// ------------------------------------------------------------- warp-level MMA
// bf16 m16n8k16 MMAs with FP32 accumulation, the split products over NP
// pieces and the ldmatrix loads of their fragments.
__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// All piece products (i, j) with i + j < NP, smallest first.
template <int NP>
__device__ __forceinline__ void mma_split(float (&c)[4], const uint32_t (&a)[NP][4], const uint32_t (&b)[NP][2]) {
  if (NP == 3) {
    mma16816(c, a[1], b[1]);
    mma16816(c, a[0], b[2]);
    mma16816(c, a[2], b[0]);
  }
  if (NP >= 2) {
    mma16816(c, a[0], b[1]);
    mma16816(c, a[1], b[0]);
  }
  mma16816(c, a[0], b[0]);
}

// Two independent accumulators with their product chains interleaved, so the
// dependent MMAs of one tile overlap the other's.
template <int NP>
__device__ __forceinline__ void mma_split2(float (&c0)[4], const uint32_t (&a0)[NP][4], const uint32_t (&b0)[NP][2],
                                           float (&c1)[4], const uint32_t (&a1)[NP][4], const uint32_t (&b1)[NP][2]) {
  if (NP == 3) {
    mma16816(c0, a0[1], b0[1]);
    mma16816(c1, a1[1], b1[1]);
    mma16816(c0, a0[0], b0[2]);
    mma16816(c1, a1[0], b1[2]);
    mma16816(c0, a0[2], b0[0]);
    mma16816(c1, a1[2], b1[0]);
  }
  if (NP >= 2) {
    mma16816(c0, a0[0], b0[1]);
    mma16816(c1, a1[0], b1[1]);
    mma16816(c0, a0[1], b0[0]);
    mma16816(c1, a1[1], b1[0]);
  }
  mma16816(c0, a0[0], b0[0]);
  mma16816(c1, a1[0], b1[0]);
}

__device__ __forceinline__ void ldm_x4(uint32_t (&r)[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldm_x2(uint32_t (&r)[2], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

__device__ __forceinline__ void ldm_x2_trans(uint32_t (&r)[2], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

// ------------------------------------------------------------- tcgen05 / TMA
constexpr unsigned long long kWaitNs = 1000000000ull;   // limit of one mbarrier wait (1 s of wall time)

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor, no swizzle: start address, the byte
// distance between core matrices adjacent in K (lbo) and between core
// matrices adjacent in M/N (sbo), descriptor version 1 of the sm_100 family.
// The same two fields serve K-major and MN-major operands: lbo always steps
// along K, sbo along M/N.
__device__ __forceinline__ uint64_t sdesc2(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16 with bf16 A and B, FP32 accumulator;
// b_mn = 1 reads B as MN-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// One potentially blocking test: the thread may sleep in hardware up to
// kTryNs for the phase instead of polling the barrier through the shared-
// memory pipe (which the tensor cores' operand reads also use).
constexpr uint32_t kTryNs = 20000;

template <uint32_t HintNs = kTryNs>
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  if (HintNs) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(mbar), "r"(parity), "r"(HintNs)
                 : "memory");
  } else {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(mbar), "r"(parity)
                 : "memory");
  }
  return done != 0;
}

// Wait for the phase of the given parity to complete; false once kWaitNs has
// passed without it (the caller then records an error and stops).  HintNs is
// the suspend-time hint of each test (0: the hardware's own default).
template <uint32_t HintNs = kTryNs>
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  if (mbar_try<HintNs>(mbar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try<HintNs>(mbar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// Bulk asynchronous copy global -> shared (both 16-byte aligned, size a
// multiple of 16), completion counted in bytes on mbar.
__device__ __forceinline__ void bulk_g2s(uint32_t sdst, const void* gsrc, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(sdst),
               "l"(gsrc), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
               "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// 32 lanes x 32 consecutive 32-bit columns of tensor memory (lane = thread of
// the warp's quarter), waited on.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

}  // namespace dev
}  // namespace hfx
