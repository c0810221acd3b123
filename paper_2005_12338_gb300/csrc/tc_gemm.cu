// BF16 x BF16 -> FP32 and TF32 x TF32 -> FP32 products on the 5th-generation
// tensor cores.
//
// One CTA computes a 128 x BN tile (BN <= 256, a multiple of 16) of one
// output group: warp 0 lane 0 streams A and B slabs (128 bytes of K per row:
// 64 bf16 or 32 tf32, 128-byte swizzled) into a ring of shared-memory stages
// with TMA, warp 1 lane 0 issues tcgen05.mma (kind::f16 with K = 16, or
// kind::tf32 with K = 8, per instruction: 32 bytes of K either way; M = 128,
// N = BN) into an fp32 accumulator in tensor memory and releases each stage with
// tcgen05.commit, and all four warps drain the accumulator with tcgen05.ld
// (warp w owns TMEM lanes 32w..32w+31, i.e. output rows).  Several batch
// entries and two K segments can feed one accumulator, which turns sums of
// products (long-K contractions over sample pairs) into a single pass.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records an error
// code in a device flag, skips the remaining work, and still waits (bounded)
// for its own tensor-core work and frees its tensor memory before returning.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "tc_ptx.cuh"

namespace rssri {
namespace {

using namespace tcx;

struct TcParams {
  CUtensorMap ta[2];
  CUtensorMap tb[2];
  int K[2];
  int nseg, M, N, BN, stages, batch, bpc;
  uint32_t tmem_cols;
  float *c32;
  void *cop;
  long long ldcop;
  int *err;
  int wait_polls;  // 0: normal; > 0: test mode (see TcGemm)
};

template <int KIND>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ TcParams p) {
  constexpr int TBK = KindT<KIND>::TBK, KMMA = KindT<KIND>::KMMA;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int BN = p.BN, S = p.stages;
  const int B_STAGE = BN * SLAB;
  uint8_t *sA = smem;
  uint8_t *sB = smem + S * A_STAGE;
  uint64_t *full = (uint64_t *)(sB + S * B_STAGE);
  uint64_t *empty = full + S;
  uint64_t *accum = empty + S;
  uint32_t *tslot = (uint32_t *)(accum + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * BN;
  const int z = blockIdx.z;
  const int b_lo = z * p.bpc, b_hi = min(p.batch, b_lo + p.bpc);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    bar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     s_u32(tslot)),
                 "r"(p.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  if (threadIdx.x == 0) {
    // producer: the same (b, segment, k-block) sequence as the MMA issuer
    int it = 0;
    bool ok = test_mode_gate(p.wait_polls, p.err);
    for (int b = b_lo; b < b_hi && ok; ++b)
      for (int s = 0; s < p.nseg && ok; ++s)
        for (int k0 = 0; k0 < p.K[s]; k0 += TBK, ++it) {
          const int st = it % S;
          if (it >= S && !bar_wait(&empty[st], ((it / S) - 1) & 1, p.err, 1, p.wait_polls)) {
            ok = false;
            break;
          }
          bar_expect(&full[st], A_STAGE + B_STAGE);
          tma_load3(sA + st * A_STAGE, &p.ta[s], &full[st], k0, m0, b);
          tma_load3(sB + st * B_STAGE, &p.tb[s], &full[st], k0, n0, b);
        }
  } else if (threadIdx.x == 32) {
    const uint32_t idesc = instr_desc<KIND>(BN);
    int it = 0;
    bool ok = true, first = true;
    for (int b = b_lo; b < b_hi && ok; ++b)
      for (int s = 0; s < p.nseg && ok; ++s)
        for (int k0 = 0; k0 < p.K[s]; k0 += TBK, ++it) {
          const int st = it % S;
          if (!bar_wait(&full[st], (it / S) & 1, p.err, 2, p.wait_polls)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t da = smem_desc(s_u32(sA + st * A_STAGE));
          const uint64_t db = smem_desc(s_u32(sB + st * B_STAGE));
          // each instruction takes the next 32 bytes of K: +2 in the
          // descriptor's 16-byte start-address units
          const int nk = min(TBK / KMMA, (p.K[s] - k0 + KMMA - 1) / KMMA);
          for (int kk = 0; kk < nk; ++kk) {
            const uint32_t acc = first ? 0u : 1u;
            first = false;
            if (KIND == TC_BF16)
              asm volatile(
                  "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}" ::"r"(tmem),
                  "l"(da + 2 * kk), "l"(db + 2 * kk), "r"(idesc), "r"(acc));
            else
              asm volatile(
                  "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}" ::"r"(tmem),
                  "l"(da + 2 * kk), "l"(db + 2 * kk), "r"(idesc), "r"(acc));
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  s_u32(&empty[st]))
              : "memory");
        }
    // arrives once every MMA issued above has completed (also after a timeout)
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            s_u32(accum))
        : "memory");
  }
  __syncwarp();
  const bool ready = bar_wait(accum, 0, p.err, 3, p.wait_polls);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ready && b_lo < b_hi) {
    const int row = m0 + warp * 32 + lane;
    const long long MN = (long long)p.M * p.N;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < p.M) {
        const int col0 = n0 + c0;
        const bool full16 = col0 + 16 <= p.N;
        // 16 consecutive columns of one row per thread: vector stores fill whole sectors
        if (p.c32) {
          float *dst = p.c32 + z * MN + (long long)row * p.N + col0;
          if (full16 && (p.N % 4) == 0) {
#pragma unroll
            for (int v = 0; v < 4; ++v)
              reinterpret_cast<float4 *>(dst)[v] =
                  make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                              __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col0 + j < p.N) dst[j] = __uint_as_float(r[j]);
          }
        }
        if (p.cop && KIND == TC_BF16) {
          __nv_bfloat16 *dst = static_cast<__nv_bfloat16 *>(p.cop) + z * (long long)p.M * p.ldcop +
                               (long long)row * p.ldcop + col0;
          if (full16 && (p.ldcop % 8) == 0) {
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              uint4 q;
              uint32_t *w = reinterpret_cast<uint32_t *>(&q);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(__uint_as_float(r[8 * v + 2 * u]),
                                                                __uint_as_float(r[8 * v + 2 * u + 1]));
                w[u] = *reinterpret_cast<const uint32_t *>(&h2);
              }
              reinterpret_cast<uint4 *>(dst)[v] = q;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col0 + j < p.N) dst[j] = __float2bfloat16_rn(__uint_as_float(r[j]));
          }
        }
        if (p.cop && KIND == TC_TF32) {
          float *dst = static_cast<float *>(p.cop) + z * (long long)p.M * p.ldcop +
                       (long long)row * p.ldcop + col0;
          if (full16 && (p.ldcop % 4) == 0) {
#pragma unroll
            for (int v = 0; v < 4; ++v)
              reinterpret_cast<float4 *>(dst)[v] = make_float4(
                  round_tf32(__uint_as_float(r[4 * v])), round_tf32(__uint_as_float(r[4 * v + 1])),
                  round_tf32(__uint_as_float(r[4 * v + 2])), round_tf32(__uint_as_float(r[4 * v + 3])));
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col0 + j < p.N) dst[j] = round_tf32(__uint_as_float(r[j]));
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(p.tmem_cols));
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

void load_encode() {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
}

}  // namespace

cudaError_t tc_make_map(CUtensorMap *m, int kind, const TcOperand &op, int K, int batch,
                        int box_rows) {
  if (!g_encode) return cudaErrorNotSupported;
  const int es_bytes = kind == TC_BF16 ? 2 : 4;
  const int per16 = 16 / es_bytes;  // elements per 16 bytes
  if ((op.ld % per16) || (op.sb % per16) || ((uintptr_t)op.ptr % 16)) return cudaErrorInvalidValue;
  const long long sb = op.sb ? op.sb : op.ld * op.rows;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)op.rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)op.ld * es_bytes, (cuuint64_t)sb * es_bytes};
  cuuint32_t box[3] = {(cuuint32_t)(SLAB / es_bytes), (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = g_encode(m, kind == TC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                              3, const_cast<void *>(op.ptr),
                              dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}


cudaError_t tc_make_out_map(CUtensorMap *m, void *base, int elem_bytes, long long cols,
                            long long rows, long long batch, long long ld) {
  if (!g_encode) return cudaErrorNotSupported;
  if ((elem_bytes != 4 && elem_bytes != 2) || (uintptr_t)base % 16 || (ld * elem_bytes) % 16 ||
      cols <= 0 || rows <= 0 || batch <= 0 || cols > ld)
    return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * elem_bytes), (cuuint64_t)(ld * rows * elem_bytes)};
  cuuint32_t box[3] = {16, 32, 1};
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = g_encode(m, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                              3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool tc_available() {
  std::call_once(g_encode_once, load_encode);
  return g_encode != nullptr;
}

cudaError_t tc_prepare() {
  // the largest dynamic shared memory any launch asks for (4 stages, BN = 256),
  // set once per device outside any stream capture
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  RS_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!done[dev]) {
    const int smem = 1024 + 4 * (A_STAGE + 256 * SLAB) + 256;
    RS_TRY(cudaFuncSetAttribute(tc_gemm_kernel<TC_BF16>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RS_TRY(cudaFuncSetAttribute(tc_gemm_kernel<TC_TF32>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    done[dev] = true;
  }
  return cudaSuccess;
}

cudaError_t tc_gemm(const TcGemm &g, cudaStream_t s) {
  if (!tc_available()) return cudaErrorNotSupported;
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0 || g.nseg < 1 || g.nseg > 2 || g.bpc < 1 ||
      (g.kind != TC_BF16 && g.kind != TC_TF32))
    return cudaErrorInvalidValue;
  const int tbk = g.kind == TC_BF16 ? KindT<TC_BF16>::TBK : KindT<TC_TF32>::TBK;
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  // N tile: <= 256, a multiple of 16, with the least padding
  const int ntiles = (g.N + 255) / 256;
  const int BN = std::min(256, ((ceil_div(g.N, ntiles) + 15) / 16) * 16);
  long long iters = 0;
  for (int s2 = 0; s2 < g.nseg; ++s2) {
    if (g.K[s2] <= 0) return cudaErrorInvalidValue;
    RS_TRY(tc_make_map(&p.ta[s2], g.kind, g.A[s2], g.K[s2], g.batch, TBM));
    RS_TRY(tc_make_map(&p.tb[s2], g.kind, g.B[s2], g.K[s2], g.batch, BN));
    p.K[s2] = g.K[s2];
    iters += ceil_div(g.K[s2], tbk);
  }
  iters *= g.bpc;
  p.nseg = g.nseg;
  p.M = g.M;
  p.N = g.N;
  p.BN = BN;
  // short K: two stages so that two CTAs share an SM and overlap their epilogues
  p.stages = iters <= 8 ? 2 : 4;
  p.batch = g.batch;
  p.bpc = g.bpc;
  p.tmem_cols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  p.c32 = g.c32;
  p.cop = g.cop;
  p.ldcop = g.ldcop ? g.ldcop : g.N;
  p.err = g.err;
  p.wait_polls = g.wait_polls;
  size_t smem = 1024 + (size_t)p.stages * (A_STAGE + BN * SLAB) + 256;
  // at most two CTAs per SM, so that their tensor memory (<= 2 x 256 columns) always fits
  smem = std::max<size_t>(smem, 80 * 1024);
  RS_TRY(tc_prepare());
  const int groups = ceil_div(g.batch, g.bpc);
  for (int z0 = 0; z0 < groups; z0 += 65535) {
    // grid.z above 65535 is split into launches over group ranges
    const int nz = std::min(65535, groups - z0);
    if (z0 > 0) return cudaErrorInvalidValue;  // not needed by the path's shapes
    dim3 grid(ceil_div(g.N, BN), ceil_div(g.M, TBM), nz);
    if (g.kind == TC_BF16) tc_gemm_kernel<TC_BF16><<<grid, 128, smem, s>>>(p);
    else tc_gemm_kernel<TC_TF32><<<grid, 128, smem, s>>>(p);
    ++launch_counter();
    RS_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace rssri
