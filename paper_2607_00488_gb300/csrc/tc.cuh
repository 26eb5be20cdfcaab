// tcgen05 / TMA helpers for sm_103a (inline PTX): tensor-memory allocation,
// kind::f16 MMAs with FP32 accumulation, commits to mbarriers, TMEM loads,
// 2-D tiled TMA loads and L2 prefetches, shared-memory matrix descriptors for 128-byte-swizzled
// K-major operands, and warp-uniform bounded waits.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "ptx.cuh"

namespace srw {
namespace tc {

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ptx::smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrives once on `bar` when every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   ptx::smem_addr(bar))
               : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          ptx::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(ptx::smem_addr(bar))
      : "memory");
}

// Hint: bring the tile at {x, y} of `map` into L2 (no shared memory, no
// completion); same coordinate rules as tma_load_2d.
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO); LBO unused for this layout.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                  // LBO (unused) = 16 B
  d |= (uint64_t)(1024u >> 4) << 32;        // SBO = 1024 B
  d |= (uint64_t)1u << 46;                  // descriptor version for sm_100 family
  d |= (uint64_t)2u << 61;                  // 128-byte swizzle
  return d;
}

// The same for rows of 64 bytes (32 BF16/FP16 along K): 64-byte swizzle,
// 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                  // LBO (unused) = 16 B
  d |= (uint64_t)(512u >> 4) << 32;         // SBO = 512 B
  d |= (uint64_t)1u << 46;                  // descriptor version for sm_100 family
  d |= (uint64_t)4u << 61;                  // 64-byte swizzle
  return d;
}

// Descriptor of a K-major tile whose rows hold BK 16-bit elements (BK = 64 or 32).
template <int BK>
__device__ __forceinline__ uint64_t smem_desc_k(uint32_t saddr) {
  static_assert(BK == 64 || BK == 32, "rows of 128 or 64 bytes");
  return BK == 64 ? smem_desc_sw128(saddr) : smem_desc_sw64(saddr);
}

// Byte offset of 16-byte chunk `ch` of tile row `row` in the swizzled K-major
// layout that TMA writes and the descriptors above read: rows of 2 BK bytes,
// the chunk index XOR-ed with row bits (128-byte swizzle: row & 7; 64-byte
// swizzle: (row >> 1) & 3).
template <int BK>
__device__ __forceinline__ uint32_t swz_offset(int row, int ch) {
  return BK == 64 ? (uint32_t)(row * 128 + ((ch ^ (row & 7)) << 4))
                  : (uint32_t)(row * 64 + ((ch ^ ((row >> 1) & 3)) << 4));
}

// Instruction descriptor, kind::f16, FP32 accumulator, both operands K-major
// and of one type: BF16 x BF16 (operand format 1) or F16 x F16 (format 0).
__host__ __device__ constexpr uint32_t idesc_f16kind(int m, int n, bool f16) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ bool aborted(const unsigned* f) { return *(const volatile unsigned*)f != 0u; }

// Bounded wait taken by all 32 lanes of a warp; the warp proceeds only if
// every lane saw the phase complete, so no lane can run ahead into a
// .sync.aligned instruction or a __syncwarp that the others skip.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, unsigned* abort_flag) {
  const bool ok = ptx::mbar_wait(bar, parity, abort_flag);
  return __all_sync(0xffffffffu, ok);
}

}  // namespace tc
}  // namespace srw
