// Persistent grouped tensor-core products (see tc_group.cuh).
//
// The host lays out a work queue of output tiles: the 128 x BN tiles of each
// product (of its own shape and N tile), product after product.  One CTA per
// SM walks the queue with a fixed stride (tile q goes to CTA q mod grid, so
// the assignment and every result are deterministic).  Per CTA:
//   warp 0 lane 0  TMA producer of A and B slabs (128 bytes of K per row,
//                  128-byte swizzle) into a ring of shared-memory stages,
//                  running ahead across tile boundaries;
//   warp 1 lane 0  MMA issuer: tcgen05.mma into one of two fp32 accumulators
//                  in tensor memory (2 x 256 columns), alternating per tile,
//                  so that the products of tile i+1 run while the epilogue
//                  drains tile i;
//   warps 2-5      epilogue: tcgen05.ld of the accumulator (warp w reads lanes
//                  32 (w mod 4) ...), 16 columns at a time, staged through a
//                  double-buffered 32-row x 16-column box in shared memory
//                  and written by TMA bulk tensor stores (fp32 and/or
//                  operand-type outputs; plain stores where an output's rows
//                  are not 16-byte aligned), then release of the accumulator.
// Every mbarrier wait is bounded; on expiry the kernel records an error code
// in a device flag and stops; before tensor memory is freed the epilogue
// waits (bounded) for every product the issuer started.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "tc_group.cuh"
#include "tc_ptx.cuh"

namespace rssri {
namespace {

using namespace tcx;

constexpr int GTHREADS = 192;  // 6 warps
constexpr int ACC_COLS = 256;  // per accumulator (max N tile)
// epilogue staging per warp and buffer: 32 x 16 fp32 (c32) + 32 x 16 fp32
// or bf16 (operand-type output)
constexpr int STG_HALF = 32 * 16 * 4;
constexpr int STG_BUF = 2 * STG_HALF;
constexpr int STG_WARP = 2 * STG_BUF;

struct GProb {
  CUtensorMap ta[2], tb[2];
  int K[2], nseg, M, N, BN, batch, bpc;
  int mtiles, ntiles, tile0;
  int ashared, bshared;  // operand with batch stride 0: every batch entry reads entry 0
  float *c32;
  void *cop;
  long long ldcop;
  CUtensorMap t32, top;  // output maps (valid where tma bit 0 / bit 1 is set)
  int tma;
};

struct GParams {
  GProb p[TC_GROUP_MAX];
  int np, total, stages, wait_polls;
  int *err;
};

struct Tile {
  int pi, m0, n0, z;
};

__device__ __forceinline__ Tile decode(const GParams &p, int q) {
  int pi = 0;
  while (pi + 1 < p.np && q >= p.p[pi + 1].tile0) ++pi;
  const GProb &P = p.p[pi];
  const int local = q - P.tile0;
  Tile t;
  t.pi = pi;
  t.n0 = (local % P.ntiles) * P.BN;
  t.m0 = ((local / P.ntiles) % P.mtiles) * TBM;
  t.z = local / (P.ntiles * P.mtiles);
  return t;
}

// Plain stores of one row's 16 columns (the outputs whose tma bit is clear).
template <int KIND>
__device__ void epilogue_store(const GProb &P, int z, int row, int col0, const uint32_t *r) {
  const long long MN = (long long)P.M * P.N;
  const bool full16 = col0 + 16 <= P.N;
  if (P.c32 && !(P.tma & 1)) {
    float *dst = P.c32 + z * MN + (long long)row * P.N + col0;
    if (full16 && (P.N % 4) == 0) {
#pragma unroll
      for (int v = 0; v < 4; ++v)
        reinterpret_cast<float4 *>(dst)[v] =
            make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                        __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (col0 + j < P.N) dst[j] = __uint_as_float(r[j]);
    }
  }
  if (P.cop && !(P.tma & 2) && KIND == TC_BF16) {
    __nv_bfloat16 *dst = static_cast<__nv_bfloat16 *>(P.cop) + z * (long long)P.M * P.ldcop +
                         (long long)row * P.ldcop + col0;
    if (full16 && (P.ldcop % 8) == 0) {
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
        if (col0 + j < P.N) dst[j] = __float2bfloat16_rn(__uint_as_float(r[j]));
    }
  }
  if (P.cop && !(P.tma & 2) && KIND == TC_TF32) {
    float *dst = static_cast<float *>(P.cop) + z * (long long)P.M * P.ldcop +
                 (long long)row * P.ldcop + col0;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (col0 + j < P.N) dst[j] = round_tf32(__uint_as_float(r[j]));
  }
}

template <int KIND>
__global__ void __launch_bounds__(GTHREADS, 1) tc_group_kernel(const __grid_constant__ GParams p) {
  constexpr int TBK = KindT<KIND>::TBK, KMMA = KindT<KIND>::KMMA;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  constexpr int B_STAGE = ACC_COLS * SLAB;  // room for the widest N tile
  uint8_t *sA = smem;
  uint8_t *sB = smem + S * A_STAGE;
  uint64_t *full = (uint64_t *)(sB + S * B_STAGE);
  uint64_t *empty = full + S;
  uint64_t *accf = empty + S;  // [2] accumulator complete
  uint64_t *acce = accf + 2;   // [2] accumulator drained
  uint64_t *done = acce + 2;   // every product of this CTA completed
  uint32_t *tslot = (uint32_t *)(done + 1);
  uint8_t *stg = sB + S * B_STAGE + 1024;  // epilogue staging, 1024-byte aligned
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(&accf[b], 1);
      bar_init(&acce[b], 4);
    }
    bar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     s_u32(tslot)),
                 "r"(2 * ACC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      bool ok = test_mode_gate(p.wait_polls, p.err);
      int it = 0;
      for (int q = blockIdx.x; q < p.total && ok; q += gridDim.x) {
        const Tile t = decode(p, q);
        const GProb &P = p.p[t.pi];
        const int b_lo = t.z * P.bpc, b_hi = min(P.batch, b_lo + P.bpc);
        const uint32_t bytes = A_STAGE + P.BN * SLAB;
        for (int b = b_lo; b < b_hi && ok; ++b)
          for (int sg = 0; sg < P.nseg && ok; ++sg)
            for (int k0 = 0; k0 < P.K[sg]; k0 += TBK, ++it) {
              const int st = it % S;
              if (it >= S && !bar_wait(&empty[st], ((it / S) - 1) & 1, p.err, 1, p.wait_polls)) {
                ok = false;
                break;
              }
              bar_expect(&full[st], bytes);
              tma_load3(sA + st * A_STAGE, &P.ta[sg], &full[st], k0, t.m0, P.ashared ? 0 : b);
              tma_load3(sB + st * B_STAGE, &P.tb[sg], &full[st], k0, t.n0, P.bshared ? 0 : b);
            }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int it = 0, lt = 0;
      for (int q = blockIdx.x; q < p.total && ok; q += gridDim.x, ++lt) {
        const Tile t = decode(p, q);
        const GProb &P = p.p[t.pi];
        const int buf = lt & 1;
        if (lt >= 2) {
          if (!bar_wait(&acce[buf], ((lt >> 1) - 1) & 1, p.err, 2, p.wait_polls)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
        }
        const uint32_t idesc = instr_desc<KIND>(P.BN);
        const uint32_t acc_addr = tmem + (uint32_t)(buf * ACC_COLS);
        const int b_lo = t.z * P.bpc, b_hi = min(P.batch, b_lo + P.bpc);
        bool first = true;
        for (int b = b_lo; b < b_hi && ok; ++b)
          for (int sg = 0; sg < P.nseg && ok; ++sg)
            for (int k0 = 0; k0 < P.K[sg]; k0 += TBK, ++it) {
              const int st = it % S;
              if (!bar_wait(&full[st], (it / S) & 1, p.err, 3, p.wait_polls)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;");
              const uint64_t da = smem_desc(s_u32(sA + st * A_STAGE));
              const uint64_t db = smem_desc(s_u32(sB + st * B_STAGE));
              const int nk = min(TBK / KMMA, (P.K[sg] - k0 + KMMA - 1) / KMMA);
              for (int kk = 0; kk < nk; ++kk) {
                const uint32_t acc = first ? 0u : 1u;
                first = false;
                if (KIND == TC_BF16)
                  asm volatile(
                      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}" ::"r"(acc_addr),
                      "l"(da + 2 * kk), "l"(db + 2 * kk), "r"(idesc), "r"(acc));
                else
                  asm volatile(
                      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}" ::"r"(acc_addr),
                      "l"(da + 2 * kk), "l"(db + 2 * kk), "r"(idesc), "r"(acc));
              }
              asm volatile(
                  "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                      s_u32(&empty[st]))
                  : "memory");
            }
        if (ok)
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  s_u32(&accf[buf]))
              : "memory");
      }
      // arrives once every product issued above has completed (also after a timeout)
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              s_u32(done))
          : "memory");
    }
  } else {
    // epilogue warps 2-5
    const int lq = warp & 3;
    uint8_t *wst = stg + (warp - 2) * STG_WARP;
    bool ok = true;
    int lt = 0, sc = 0;  // tiles and staged chunks of this warp
    for (int q = blockIdx.x; q < p.total && ok; q += gridDim.x, ++lt) {
      const Tile t = decode(p, q);
      const GProb &P = p.p[t.pi];
      const int buf = lt & 1;
      if (!bar_wait(&accf[buf], (lt >> 1) & 1, p.err, 4, p.wait_polls)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int row0 = t.m0 + lq * 32, row = row0 + lane;
      for (int c0 = 0; c0 < P.BN && t.n0 + c0 < P.N; c0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(buf * ACC_COLS + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (P.tma && row0 < P.M) {
          // this row into the staging box, then one bulk store per output
          uint8_t *sbuf = wst + (sc & 1) * STG_BUF;
          if (sc >= 2) {
            if (lane == 0) bulk_wait_read1();  // the box two chunks back has been read
            __syncwarp();
          }
          if (P.tma & 1) {
            uint4 *d = reinterpret_cast<uint4 *>(sbuf + lane * 64);
#pragma unroll
            for (int v = 0; v < 4; ++v)
              d[v] = make_uint4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
          }
          if (P.tma & 2) {
            if (KIND == TC_BF16) {
              uint4 *d = reinterpret_cast<uint4 *>(sbuf + STG_HALF + lane * 32);
#pragma unroll
              for (int v = 0; v < 2; ++v) {
                uint32_t w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const __nv_bfloat162 h2 = __floats2bfloat162_rn(
                      __uint_as_float(r[8 * v + 2 * u]), __uint_as_float(r[8 * v + 2 * u + 1]));
                  w[u] = *reinterpret_cast<const uint32_t *>(&h2);
                }
                d[v] = make_uint4(w[0], w[1], w[2], w[3]);
              }
            } else {
              float4 *d = reinterpret_cast<float4 *>(sbuf + STG_HALF + lane * 64);
#pragma unroll
              for (int v = 0; v < 4; ++v)
                d[v] = make_float4(round_tf32(__uint_as_float(r[4 * v])),
                                   round_tf32(__uint_as_float(r[4 * v + 1])),
                                   round_tf32(__uint_as_float(r[4 * v + 2])),
                                   round_tf32(__uint_as_float(r[4 * v + 3])));
            }
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            if (P.tma & 1) tma_store3(&P.t32, sbuf, t.n0 + c0, row0, t.z);
            if (P.tma & 2) tma_store3(&P.top, sbuf + STG_HALF, t.n0 + c0, row0, t.z);
            bulk_commit();
          }
          ++sc;
        }
        if (row < P.M && (P.tma & 3) != 3) epilogue_store<KIND>(P, t.z, row, t.n0 + c0, r);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(&acce[buf])) : "memory");
    }
    // the bulk stores are complete (and done reading shared memory)
    if (lane == 0) bulk_wait_all();
    __syncwarp();
    // every product the issuer started is complete before tensor memory is freed
    bar_wait(done, 0, p.err, 5, p.wait_polls);
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * ACC_COLS));
}

size_t group_smem(int stages) {
  // alignment slack, stages, barriers (1024), epilogue staging
  return 1024 + (size_t)stages * (A_STAGE + ACC_COLS * SLAB) + 1024 + 4 * STG_WARP;
}

cudaError_t group_prepare() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  RS_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!done[dev]) {
    const int smem = (int)group_smem(4);
    RS_TRY(cudaFuncSetAttribute(tc_group_kernel<TC_BF16>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RS_TRY(cudaFuncSetAttribute(tc_group_kernel<TC_TF32>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    done[dev] = true;
  }
  return cudaSuccess;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 152;
  }
  return n;
}

// The N tile with the least padding (<= 256, a multiple of 16).
int default_bn(int N) {
  const int ntiles = (N + 255) / 256;
  return std::min(256, ((ceil_div(N, ntiles) + 15) / 16) * 16);
}

using Key = std::tuple<int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<Key, int> g_tuned;

Key key_of(int kind, const TcProb &t) {
  return Key(kind, t.M, t.N, t.K[0] + t.K[1], t.nseg, t.batch, t.bpc);
}

cudaError_t launch_group(int kind, const TcProb *probs, int np, int *err, cudaStream_t s,
                         int wait_polls) {
  GParams gp;
  std::memset(&gp, 0, sizeof(gp));
  int total = 0;
  long long kslabs = 0;
  const int tbk = kind == TC_BF16 ? KindT<TC_BF16>::TBK : KindT<TC_TF32>::TBK;
  for (int i = 0; i < np; ++i) {
    const TcProb &t = probs[i];
    if (t.M <= 0 || t.N <= 0 || t.batch <= 0 || t.bpc < 1 || t.nseg < 1 || t.nseg > 2)
      return cudaErrorInvalidValue;
    GProb &P = gp.p[i];
    int bn = t.bn;
    if (bn <= 0) {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tuned.find(key_of(kind, t));
      bn = it != g_tuned.end() ? it->second : default_bn(t.N);
    }
    if (bn < 16 || bn > ACC_COLS || bn % 16) return cudaErrorInvalidValue;
    P.BN = bn;
    // a zero batch stride shares the operand across the batch (map of one entry)
    P.ashared = t.A[0].sb == 0 && t.batch > 1;
    P.bshared = t.B[0].sb == 0 && t.batch > 1;
    for (int sg = 0; sg < t.nseg; ++sg) {
      if (t.K[sg] <= 0) return cudaErrorInvalidValue;
      if ((t.A[sg].sb == 0) != (t.A[0].sb == 0) || (t.B[sg].sb == 0) != (t.B[0].sb == 0))
        return cudaErrorInvalidValue;
      RS_TRY(tc_make_map(&P.ta[sg], kind, t.A[sg], t.K[sg], P.ashared ? 1 : t.batch, TBM));
      RS_TRY(tc_make_map(&P.tb[sg], kind, t.B[sg], t.K[sg], P.bshared ? 1 : t.batch, bn));
      P.K[sg] = t.K[sg];
      kslabs += (long long)ceil_div(t.K[sg], tbk) * t.batch;
    }
    P.nseg = t.nseg;
    P.M = t.M;
    P.N = t.N;
    P.batch = t.batch;
    P.bpc = t.bpc;
    P.mtiles = ceil_div(t.M, TBM);
    P.ntiles = ceil_div(t.N, bn);
    P.tile0 = total;
    P.c32 = t.c32;
    P.cop = t.cop;
    P.ldcop = t.ldcop ? t.ldcop : t.N;
    // outputs whose rows are 16-byte aligned are written by TMA stores
    P.tma = 0;
    const long long zc = ceil_div(t.batch, t.bpc);
    if (t.c32 && tc_make_out_map(&P.t32, t.c32, 4, t.N, t.M, zc, t.N) == cudaSuccess) P.tma |= 1;
    if (t.cop && tc_make_out_map(&P.top, t.cop, kind == TC_BF16 ? 2 : 4, t.N, t.M, zc,
                                 P.ldcop) == cudaSuccess)
      P.tma |= 2;
    const long long tiles = (long long)P.mtiles * P.ntiles * ceil_div(t.batch, t.bpc);
    if (total + tiles > (1LL << 30)) return cudaErrorInvalidValue;
    total += (int)tiles;
  }
  if (total == 0) return cudaSuccess;
  gp.np = np;
  gp.total = total;
  gp.stages = 4;
  gp.wait_polls = wait_polls;
  gp.err = err;
  RS_TRY(group_prepare());
  const int grid = std::min(total, sm_count());
  const size_t smem = group_smem(gp.stages);
  if (kind == TC_BF16) tc_group_kernel<TC_BF16><<<grid, GTHREADS, smem, s>>>(gp);
  else tc_group_kernel<TC_TF32><<<grid, GTHREADS, smem, s>>>(gp);
  ++launch_counter();
  (void)kslabs;
  return cudaGetLastError();
}

}  // namespace

cudaError_t tc_group(int kind, const TcProb *probs, int np, int *err, cudaStream_t s,
                     int wait_polls) {
  if (!tc_available()) return cudaErrorNotSupported;
  if (kind != TC_BF16 && kind != TC_TF32) return cudaErrorInvalidValue;
  for (int i0 = 0; i0 < np; i0 += TC_GROUP_MAX)
    RS_TRY(launch_group(kind, probs + i0, std::min(TC_GROUP_MAX, np - i0), err, s, wait_polls));
  return cudaSuccess;
}

int tc_group_tune(int kind, TcProb &prob, int *err, cudaStream_t s) {
  const Key k = key_of(kind, prob);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(k);
    if (it != g_tuned.end()) return it->second;
  }
  // candidates: the least-padding width and the multiples of 64 up to 256
  int cands[6], nc = 0;
  cands[nc++] = default_bn(prob.N);
  for (int b = 64; b <= 256; b += 64)
    if (b != cands[0] && b <= ((prob.N + 15) / 16) * 16 + 48) cands[nc++] = b;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cands[0];
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cands[0];
  }
  int best = cands[0];
  float best_ms = 1e30f;
  for (int c = 0; c < nc; ++c) {
    TcProb t = prob;
    t.bn = cands[c];
    if (launch_group(kind, &t, 1, err, s, 0) != cudaSuccess) continue;  // warm-up
    cudaEventRecord(e0, s);
    bool ok = true;
    for (int r = 0; r < 3 && ok; ++r) ok = launch_group(kind, &t, 1, err, s, 0) == cudaSuccess;
    cudaEventRecord(e1, s);
    float ms = 0;
    if (ok && cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = cands[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[k] = best;
  return best;
}

int tc_group_tuned_shapes() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return (int)g_tuned.size();
}

}  // namespace rssri
