// Shared device/host definitions of the sm_103a engine: model constants, pool layouts,
// and thin inline-PTX wrappers for mbarriers, bulk copies and the tcgen05 tensor cores.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstdio>

namespace sedacs {

// ------------------------------------------------------------------------------------
// Model constants (copied from the caller's sedacs_model at context creation).
// ------------------------------------------------------------------------------------
struct ModelDev {
  int n_orb[3];
  double eps_s[3], eps_p[3], hubbard_u[3], z_val[3], mass[3];
  double v0[3][3][4];     // [s-atom or i][p-atom or j][ss, sp, pps, ppp]
  double decay, overlap_scale, r_on, r_off;
  double rep_a[3][3];
  double rep_decay;
};

// Unit conversions (CODATA 2018).
constexpr double kBohrA = 0.529177210903;
constexpr double kAccHaAAmu = 0.2625499639;   // (Ha/A)/amu expressed in A/fs^2

// Bounded spin limit for every device-side wait (cycles; ~0.2 s at 2 GHz).  Legitimate
// waits of the pipelines here last microseconds.
constexpr long long kWaitLimitCycles = 400000000LL;

// Error flags raised by kernels (OR-ed into a device word, read by the host).
enum DevErr : int {
  kErrTimeout = 1,
  kErrBounds = 2,
  kErrNumeric = 4,
  kErrCapacity = 8,
};

// ------------------------------------------------------------------------------------
// Blocked split-plane operand layout ("UMMA-blocked").
//
// A matrix of n_rows x n_cols (both multiples of 128 / 64) is stored as blocks of
// 128 rows x 64 columns, block (rb, kb) at byte offset (rb * (n_cols / 64) + kb) * 16384.
// Inside a block, row r occupies bytes [r*128, r*128+128); its 16-byte chunk j
// (columns 8j .. 8j+7) sits at chunk position j ^ (r & 7).  This is the shared-memory
// image the tensor core reads with the 128-byte swizzle, so one bulk copy moves a
// block from global memory to a 1024-byte aligned shared tile unchanged.
// A value x is kept as up to three bf16 planes hi + mid + lo (x - hi - mid rounded), or
// (format kPlanesF16x2) as two fp16 planes hi + lo: the dual half-precision representation
// of Finkelstein et al. (2021), x = hi + 2^-11 lo with hi = fp16(x) and lo = fp16(2^11 (x - hi)).
// |x - hi| <= 2^-11 |x|, so the scaled lo has the magnitude of x and stays out of the fp16
// subnormal range wherever hi does; hi + 2^-11 lo carries 22 significant bits.
// ------------------------------------------------------------------------------------
constexpr int kBlkRows = 128;
constexpr int kBlkCols = 64;
constexpr int kBlkBytes = kBlkRows * kBlkCols * 2;   // 16384

// Plane formats: 1, 2, 3 = that many bf16 planes; kPlanesF16x2 = two fp16 planes (hi, scaled lo).
constexpr int kPlanesF16x2 = 4;
constexpr float kF16LoScale = 2048.f;
constexpr float kF16LoInv = 1.f / 2048.f;
__host__ __device__ constexpr int planes_of(int fmt) { return fmt == kPlanesF16x2 ? 2 : fmt; }

__host__ __device__ inline long long blocked_offset(int row, int col, int n_cols) {
  const int rb = row >> 7, r = row & 127;
  const int kb = col >> 6, c = col & 63;
  const int j = c >> 3, e = c & 7;
  return ((long long)rb * (n_cols >> 6) + kb) * kBlkBytes + r * 128 + ((j ^ (r & 7)) << 4) + e * 2;
}

#if defined(__CUDACC__)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier --------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on a phase parity; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitLimitCycles) return false;
  }
  return true;
}

// ---- bulk copy global -> shared (completes on an mbarrier with a byte count) ------------
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---- tcgen05 (5th generation tensor cores, accumulators in tensor memory) ----------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, bf16 inputs, fp32 accumulate, M = 128.
__device__ __forceinline__ void tc_mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on an mbarrier once every previously issued tcgen05.mma of this thread completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// 32 lanes x 32 consecutive 32-bit columns: thread t of the warp gets lane (base_lane + t).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                          // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}
// Shared-memory descriptor of an MN-major operand with the 128-byte swizzle: each K row holds
// 64 consecutive MN elements (128 B), 8-row K groups 1024 B apart, 64-element MN atoms
// atom_stride bytes apart.  A K-major stored block of a symmetric matrix read this way is the
// operand's transpose, i.e. the block on the other side of the diagonal.
__device__ __forceinline__ uint64_t smem_desc_sw128_mn(uint32_t saddr, uint32_t atom_stride) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)((atom_stride >> 4) & 0x3FFF) << 16;   // leading byte offset: next MN atom
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row K group
  d |= (uint64_t)1 << 46;                          // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}
// Instruction descriptor bits marking A / B as MN-major.
constexpr uint32_t kIdescTransA = 1u << 15, kIdescTransB = 1u << 16;

// Instruction descriptor: kind::f16, A = B = bf16, D = f32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// The same with A = B = fp16 (A and B formats 0).
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Split x into bf16 planes hi + mid + lo.
__device__ __forceinline__ void split3(float x, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(hi);
  mid = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(mid);
  lo = __float2bfloat16_rn(r2);
}

// Split x into the fp16 planes hi and lo (x = hi + 2^-11 lo to 22 bits).
__device__ __forceinline__ void split_f16x2(float x, __half& hi, __half& lo) {
  hi = __float2half_rn(x);
  lo = __float2half_rn((x - __half2float(hi)) * kF16LoScale);
}
__device__ __forceinline__ float join_f16x2(__half hi, __half lo) {
  return fmaf(__half2float(lo), kF16LoInv, __half2float(hi));
}

// Write 8 consecutive values (one 16-byte granule per plane) in plane format fmt at byte
// offset off of plane 0.
__device__ __forceinline__ void write_planes8(uint8_t* arena, long long off, long long plane, int fmt,
                                              const float* v) {
  if (fmt == kPlanesF16x2) {
    __align__(16) __half h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) split_f16x2(v[e], h[e], l[e]);
    *reinterpret_cast<uint4*>(arena + off) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(arena + off + plane) = *reinterpret_cast<const uint4*>(l);
    return;
  }
  __align__(16) __nv_bfloat16 h[8], m[8], l[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) split3(v[e], h[e], m[e], l[e]);
  *reinterpret_cast<uint4*>(arena + off) = *reinterpret_cast<const uint4*>(h);
  if (fmt > 1) *reinterpret_cast<uint4*>(arena + off + plane) = *reinterpret_cast<const uint4*>(m);
  if (fmt > 2) *reinterpret_cast<uint4*>(arena + off + 2 * plane) = *reinterpret_cast<const uint4*>(l);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

#endif  // __CUDACC__

}  // namespace sedacs
