// Device helpers shared by the tensor-core product kernels (tcgen05 with TMA
// and mbarriers): bounded mbarrier waits, 3D TMA loads, the shared-memory and
// instruction descriptors of K-major bf16 / tf32 operands in 128-byte
// swizzled slabs.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "tc_gemm.cuh"

namespace rssri {
namespace tcx {

constexpr int TBM = 128, SLAB = 128;  // rows per CTA tile; bytes of K per stage and row
constexpr int A_STAGE = TBM * SLAB;

// Element size and K elements per stage / per instruction of each kind.
template <int KIND> struct KindT;
template <> struct KindT<TC_BF16> {
  static constexpr int ES = 2, TBK = SLAB / 2, KMMA = 16;
};
template <> struct KindT<TC_TF32> {
  static constexpr int ES = 4, TBK = SLAB / 4, KMMA = 8;
};


__device__ __forceinline__ uint32_t s_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(b)), "r"(c));
}
__device__ __forceinline__ void bar_expect(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ uint32_t bar_try(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(s_u32(b)), "r"(parity)
      : "memory");
  return ok;
}
// Bounded wait (each try_wait may suspend for a while): ~2^22 polls, or
// `polls` when positive.
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity, int *err, int code,
                                         int polls = 0) {
  const int lim = polls > 0 ? polls : (1 << 22);
  for (int i = 0; i < lim; ++i)
    if (bar_try(b, parity)) return true;
  if (err) atomicExch(err, code);
  return false;
}
// Test mode: the producer waits (bounded) until a consumer has flagged its
// expired wait, and then issues nothing.  Returns true when it may proceed.
__device__ __forceinline__ bool test_mode_gate(int polls, int *err) {
  if (polls <= 0) return true;
  for (int i = 0; i < (1 << 22); ++i) {
    if (err && *(volatile int *)err) return false;
    __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *m, uint64_t *bar, int x,
                                          int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(s_u32(dst)),
      "l"(m), "r"(s_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// Bulk tensor store of a shared-memory box to global (bulk-group tracked).
__device__ __forceinline__ void tma_store3(const CUtensorMap *m, const void *src, int x, int y,
                                           int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(m),
      "r"(s_u32(src)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until at most one committed group still reads shared memory.
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// Waits until every committed group has completed.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (TMA) reads of them.
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows
// of 128 bytes grouped by 8 (stride 1024 bytes between groups).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor: D fp32, A and B of the same type (bf16 = 1 under
// kind::f16, tf32 = 2 under kind::tf32), both K-major, M = 128, N = n.
template <int KIND>
__device__ __forceinline__ uint32_t instr_desc(int n) {
  constexpr uint32_t ab = KIND == TC_BF16 ? 1u : 2u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(TBM >> 4) << 24);
}

// fp32 rounded to the nearest tf32 (10 stored mantissa bits), kept in fp32.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tcx

// Tensor map of one operand (TcOperand: rows x K per batch entry, K
// contiguous) for 128-byte swizzled slabs of box_rows rows.
cudaError_t tc_make_map(CUtensorMap *m, int kind, const TcOperand &op, int K, int batch,
                        int box_rows);
// Tensor map of an output [batch][rows][ld] (elements of elem_bytes = 4:
// fp32, 2: bf16; cols <= ld valid per row) for stores of 32-row x 16-column
// boxes, no swizzle.  ld * elem_bytes and the base must be 16-byte aligned.
cudaError_t tc_make_out_map(CUtensorMap *m, void *base, int elem_bytes, long long cols,
                            long long rows, long long batch, long long ld);

}  // namespace rssri
