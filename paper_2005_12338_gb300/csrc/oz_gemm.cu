// fp64-accurate products on the bf16 tensor cores (tcgen05, TMA, TMEM) by
// error-free digit slicing; see oz_gemm.cuh for the number scheme.
//
// Kernel layout (persistent: one CTA per SM walks the 128 x 128 output tiles
// with a fixed stride; 18 warps):
//   warp 0 lane 0  TMA producer: per K step of 16, the digits of A and of B
//                  into a ring of shared-memory stages, per operand digits
//                  0-3 as one 128 x 128-byte tile (128-byte swizzle) and
//                  digits 4-5 as one 128 x 64-byte tile (64-byte swizzle):
//                  the digit layout interleaves the digits of each block of
//                  16 columns, so every TMA row is 128 or 64 bytes wide;
//   warp 1 lane 0  MMA issuer: per K step, the 21 digit products p + q <= 5
//                  (tcgen05.mma kind::f16, M = N = 128, K = 16) into four fp32
//                  accumulators in tensor memory, one per level p + q = 0, 1,
//                  2 and one for p + q >= 3 (4 x 128 of the 512 columns);
//   warps 2-17     drain: after every 256 terms of K (16 steps) they read the
//                  four accumulators (tcgen05.ld, 16 x 8 fragments) and add them
//                  exactly into double-float running totals held in registers
//                  (each thread: 32 outputs, column pairs of four rows), then
//                  release the accumulators; at the end they assemble fp64 from
//                  the running totals with integer exponent arithmetic and
//                  store column pairs as 16-byte stores.
// Levels 0-2 are exact over 256 terms (< 2^24 grid units), so a chunk's sum
// a0 + a1 + a2 is exact in two TwoSums; level >= 3 (~2^-24 of the result)
// and the running sum round at ~2^-48 relative.
//
// Every mbarrier wait is bounded; on expiry the kernel records an error code
// in a device flag and stops waiting; tensor memory is freed on every path.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "oz_gemm.cuh"

namespace rssri {
namespace {

constexpr int BM = 128, BN = 128, KS = 16;   // tile rows, columns; K per step (32 bytes of bf16)
constexpr int TILE0 = BM * 64 * 2;           // digits 0-3 of one K step: 128 rows x 128 bytes
constexpr int TILE1 = BM * 32 * 2;           // digits 4-5: 128 rows x 64 bytes
constexpr int OPB = TILE0 + TILE1;           // one operand's digits of one K step
constexpr int STAGE = 2 * OPB;               // A and B digits of one K step
constexpr int STAGES = 4;
constexpr int CHUNK = 16;                    // K steps between drains (256 terms)
constexpr int EPI = 16;                      // drain warps (4 per tensor-memory lane quarter)
constexpr int DC = BN / 4;                   // accumulator columns per drain thread
constexpr int THREADS = (2 + EPI) * 32;
constexpr int TMEM_COLS = 512;               // 4 accumulators x 128 columns
// (+8 KB slack beyond the last tile)
constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256 + 8192;

// Bounds checks (RSSRI_CHECKS builds): the first violation is recorded and
// the access skipped; release builds compile them away.
__device__ int g_check[4];
__device__ long long g_check_ctx[12];  // context of the first violation (where recorded)
#ifdef RSSRI_CHECKS
__device__ __noinline__ void check_fail(int code, int line, long long idx) {
  if (atomicCAS(&g_check[0], 0, code) == 0) {
    g_check[1] = line;
    g_check[2] = (int)(idx & 0xFFFFFFFF);
    g_check[3] = (int)(idx >> 32);
  }
}
#define OZ_IN(idx, cap, code) \
  ((cap) <= 0 || ((idx) >= 0 && (idx) < (cap)) ? true : (check_fail((code), __LINE__, (idx)), false))
#else
#define OZ_IN(idx, cap, code) true
#endif

struct OzParams {
  CUtensorMap ta0, ta1, tb0, tb1;  // digits 0-3 and 4-5 of A and B
  int M, N;          // dense: C rows / columns per batch; exchange: n, n_aux
  int kst;           // K steps per CTA
  int ksplit;        // dense: K splits (tile z = batch * ksplit + split)
  int bshared;       // dense: B has one batch entry
  const int *efa, *efb;
  long long efa_bs, efb_bs;
  int neg;    // C = -(the product) instead of +(the product)
  int vec2;   // every output row starts 16-byte aligned: column pairs go out as one store
  int mfast;  // dense: m tile fastest in the tile order (else n tile fastest)
  double *C;
  long long ldc, sC;
  int bk, nl16, jtiles, lb0;  // exchange geometry
  int tiles, ntiles, mtiles;  // the output tiles the persistent CTAs share
  int *err;
  long long ccap, efa_cap, efb_cap;  // bounds of C and the exponent arrays (checks)
  int wait_polls;  // 0: normal; > 0: test mode (see OzGemm)
};

// ------------------------------------------------------------ PTX helpers --
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
__device__ __forceinline__ void bar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(b)) : "memory");
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
// Bounded wait: gives up after ~2^22 polls (`polls` when positive), or at
// once when another thread of the launch has already flagged an error.
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity, int *err, int code,
                                         int polls = 0) {
  const int lim = polls > 0 ? polls : (1 << 22);
  for (int i = 0; i < lim; ++i) {
    if (bar_try(b, parity)) return true;
    if ((i & 1023) == 1023 && err && *(volatile int *)err) return false;
  }
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
__device__ __forceinline__ void tma_load4(void *dst, const CUtensorMap *m, uint64_t *bar, int x,
                                          int y, int z, int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(s_u32(dst)),
      "l"(m), "r"(s_u32(bar)), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}
// Shared-memory matrix descriptor of a K-major operand in rows of 128 bytes
// (128-byte swizzle, layout code 2, 1024 bytes between groups of 8 rows) or
// of 64 bytes (64-byte swizzle, code 4, 512 bytes between groups).
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t saddr, uint32_t sbo, uint32_t layout) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(sbo >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)layout << 61;
  return d;
}
// Digit p of an operand's stage slot at `base`: its 16 columns start 32 p
// bytes into the 128-byte rows (p < 4) or 32 (p - 4) into the 64-byte rows.
__device__ __forceinline__ uint64_t digit_desc(uint32_t base, int p) {
  return p < 4 ? smem_desc_sw(base + 32 * p, 1024, 2)
               : smem_desc_sw(base + TILE0 + 32 * (p - 4), 512, 4);
}
// Instruction descriptor: D fp32, A and B bf16, both K-major, M = N = 128.
__device__ __forceinline__ uint32_t instr_desc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          s_u32(bar))
      : "memory");
}
// 16 lanes x 256 bits (8 columns): thread t holds lane (t >> 2) at columns
// 2 (t & 3) and 2 (t & 3) + 1 in r[0], r[1], and lane (t >> 2) + 8 at the same
// columns in r[2], r[3]; four threads cover a lane's 8 columns.
__device__ __forceinline__ void tmem_ld16x256(uint32_t taddr, uint32_t *r) {
  asm volatile("tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}

// ----------------------------------------------------- exact float sums ----
// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (hi, lo) += a0 + a1 + a2 + a3, where a0, a1, a2 are exact chunk sums and a3
// the small rounded level.
__device__ __forceinline__ void fold(float &hi, float &lo, float a0, float a1, float a2,
                                     float a3) {
  float s, e, s2, e2;
  two_sum(a0, a1, s, e);
  two_sum(s, a2, s2, e2);
  e = (e + e2) + a3;
  float t, f;
  two_sum(hi, s2, t, f);
  f = f + (lo + e);
  two_sum(t, f, hi, lo);
}

// f * 2^E as an fp64 value, built from the float's bits (no fp64 arithmetic).
__device__ __forceinline__ double f32_scaled(float f, int E) {
  const uint32_t u = __float_as_uint(f);
  const int ef = (int)((u >> 23) & 0xFF);
  if (ef == 0) return 0.0;  // zero, or an fp32 subnormal: < 2^-126 of one grid unit
  const int e64 = ef - 127 + 1023 + E;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  unsigned long long mant = (unsigned long long)(u & 0x7FFFFF) << 29;
  if (e64 >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  if (e64 <= 0) {
    // fp64 subnormal: shift the significand (with its leading one) right, truncating
    const int sh = 1 - e64;
    mant = sh < 64 ? ((mant | (1ull << 52)) >> sh) : 0ull;
    return __longlong_as_double((long long)(sign | mant));
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)e64 << 52) | mant));
}

// The rare operands of df_to_f64 (zero, tiny, huge, non-finite): one fp64 add.
// Kept out of line so that the fp64 work is never executed speculatively on
// the common path (the fp64 pipe runs at 1/64 of the fp32 rate).
__device__ __noinline__ double df_to_f64_add(float hi, float lo, int E) {
  return f32_scaled(hi, E) + f32_scaled(lo, E);
}

// (hi + lo) 2^E as fp64 with integer operations only (the fp64 pipe runs at
// 1/64 of the fp32 rate here): hi's 53-bit significand plus lo in units of
// hi's fp64 ulp, renormalised by at most one bit.  (hi, lo) comes from a
// TwoSum, so |lo| <= ulp_f32(hi) / 2 and lo moves the significand by less
// than 2^29 units; lo's bits below one unit are dropped and a renormalising
// right shift truncates, so the result is within 2 ulp of the exact sum,
// far inside the 2^-48 rounding of the running totals.  Tiny, huge,
// non-finite or out-of-pattern operands take one fp64 add instead.
__device__ __forceinline__ double df_to_f64(float hi, float lo, int E) {
  const uint32_t uh = __float_as_uint(hi), ul = __float_as_uint(lo);
  const int eh = (int)((uh >> 23) & 0xFF), el = (int)((ul >> 23) & 0xFF);
  const int e64 = eh - 127 + 1023 + E;
  const int sh = el - eh + 29;  // lo's unit shift relative to hi's fp64 ulp
  const bool lo_zero = (ul << 1) == 0;
  if (eh < 64 || eh == 255 || e64 < 2 || e64 > 2045 || (!lo_zero && (el == 0 || sh > 6)))
    return df_to_f64_add(hi, lo, E);
  long long S = (long long)((1u << 23) | (uh & 0x7FFFFFu)) << 29;
  if (!lo_zero) {
    const long long ml = (long long)((1u << 23) | (ul & 0x7FFFFFu));
    const long long u = sh >= 0 ? ml << sh : (sh > -40 ? ml >> -sh : 0LL);
    S += ((uh ^ ul) >> 31) ? -u : u;
  }
  int e = e64;
  if (S >= (1LL << 53)) {
    S >>= 1;
    ++e;
  } else if (S < (1LL << 52)) {
    S <<= 1;
    --e;
  }
  return __longlong_as_double((long long)(((unsigned long long)(uh >> 31) << 63) |
                                          ((unsigned long long)e << 52) |
                                          ((unsigned long long)S & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ int row_scale(int ef) { return max(ef, 1) - 1022; }

// ------------------------------------------------------------- the GEMM ----
// One output tile of a persistent CTA's queue (tile q = n tile + ntiles * rest):
// dense: rest = m tile + mtiles * (batch * ksplit + split); exchange: rest = row tile.
struct OzTile {
  int n0, m0, zb, split, rt, mt, jt;
};
// With mfast: q = m tile + mtiles * (n tile + ntiles * (batch * ksplit + split)).
template <int MODE>
__device__ __forceinline__ OzTile oz_tile(const OzParams &p, int q) {
  OzTile t;
  if (MODE == 0) {
    int z;
    if (p.mfast) {
      const int rest = q / p.mtiles;
      t.m0 = (q - rest * p.mtiles) * BM;
      z = rest / p.ntiles;
      t.n0 = (rest - z * p.ntiles) * BN;
    } else {
      const int rest = q / p.ntiles;
      t.n0 = (q - rest * p.ntiles) * BN;
      z = rest / p.mtiles;
      t.m0 = (rest - z * p.mtiles) * BM;
    }
    t.zb = z / p.ksplit;
    t.split = z - t.zb * p.ksplit;
    t.rt = t.mt = t.jt = 0;
  } else {
    const int rest = q / p.ntiles;
    t.n0 = (q - rest * p.ntiles) * BN;
    t.rt = rest;
    t.mt = rest / p.jtiles;
    t.jt = rest - t.mt * p.jtiles;
    t.m0 = t.zb = t.split = 0;
  }
  return t;
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) oz_gemm_kernel(const __grid_constant__ OzParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + STAGES * STAGE);
  uint64_t *empty = full + STAGES;
  uint64_t *accf = empty + STAGES;  // a chunk's accumulators are complete
  uint64_t *acce = accf + 1;        // the drain warps have read them
  uint64_t *done = acce + 1;        // every product this CTA issued has completed
  uint32_t *tslot = (uint32_t *)(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kst = p.kst;
  const int nchunks = (kst + CHUNK - 1) / CHUNK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    bar_init(accf, 1);
    bar_init(acce, EPI);
    bar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     s_u32(tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: the K steps of this CTA's tiles, one after another
      bool go = test_mode_gate(p.wait_polls, p.err);
      int it = 0;  // K steps loaded so far (all tiles)
      for (int q = blockIdx.x; q < p.tiles && go; q += gridDim.x) {
        const OzTile t = oz_tile<MODE>(p, q);
        for (int st = 0; st < kst; ++st, ++it) {
          const int s = it % STAGES;
          if (it >= STAGES &&
              !bar_wait(&empty[s], ((it / STAGES) - 1) & 1, p.err, 1, p.wait_polls)) {
            go = false;
            break;
          }
          bar_expect(&full[s], STAGE);
          uint8_t *sa = smem + s * STAGE, *sb = sa + OPB;
          // coordinates (inner, 16-column block, ...): dense (0, kb, row, batch);
          // exchange A (0, st, 0, tile), B (0, l block, k, q)
          int ay, az, aw, by, bz, bw;
          if (MODE == 0) {
            ay = by = t.split * kst + st;
            az = t.m0;
            aw = t.zb;
            bz = t.n0;
            bw = p.bshared ? 0 : t.zb;
          } else {
            const int kidx = st / p.nl16, ls = st % p.nl16;
            ay = st;
            az = 0;
            aw = t.rt;
            by = t.jt + p.lb0 + ls;         // block of l' (may lie outside: zeros)
            bz = t.mt * 8 - p.bk + kidx;    // k (may lie outside: zeros)
            bw = t.n0;                      // q
          }
          tma_load4(sa, &p.ta0, &full[s], 0, ay, az, aw);
          tma_load4(sa + TILE0, &p.ta1, &full[s], 0, ay, az, aw);
          tma_load4(sb, &p.tb0, &full[s], 0, by, bz, bw);
          tma_load4(sb + TILE0, &p.tb1, &full[s], 0, by, bz, bw);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      const uint32_t idesc = instr_desc_bf16();
      bool ok = true;
      int it = 0, gc = 0;  // K steps and chunks issued so far (all tiles)
      for (int q = blockIdx.x; q < p.tiles && ok; q += gridDim.x) {
        for (int st = 0; st < kst; ++st, ++it) {
          const int s = it % STAGES, cs = st % CHUNK;
          if (cs == 0 && gc > 0) {
            // the previous chunk's accumulators have been read
            if (!bar_wait(acce, (gc - 1) & 1, p.err, 2, p.wait_polls)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
          }
          if (!bar_wait(&full[s], (it / STAGES) & 1, p.err, 3, p.wait_polls)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t base_a = s_u32(smem + s * STAGE), base_b = base_a + OPB;
#pragma unroll
          for (int pa = 0; pa < OZ_S; ++pa)
#pragma unroll
            for (int pb = 0; pb < OZ_S - pa; ++pb) {
              const int acc = min(pa + pb, 3);
              // the first product into each accumulator in a chunk overwrites it
              const uint32_t en = (cs > 0 || !(pa == 0 && pb <= 3)) ? 1u : 0u;
              mma_bf16(tmem + (uint32_t)(acc * 128), digit_desc(base_a, pa),
                       digit_desc(base_b, pb), idesc, en);
            }
          mma_commit(&empty[s]);
          if (cs == CHUNK - 1 || st == kst - 1) {
            mma_commit(accf);
            ++gc;
          }
        }
      }
      // a drain that is still waiting sees its phase complete once the MMAs
      // issued so far are done (and then stops on the error flag)
      if (!ok) mma_commit(accf);
      mma_commit(done);
    }
  } else {
    // drain warps: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (the
    // rows of its lane quarter) and columns 32 cq .. + 31 of each accumulator,
    // as eight 16 x 8 fragments (16x256b loads): fragment f = 4 h + g covers
    // rows 16 h .. + 15 of the quarter and columns 8 g .. + 7.  Value c = 4 f + u
    // of a thread is row 16 h + fr + 8 (u >> 1), column 8 g + fc + (u & 1).
    const int lq = warp & 3;
    const int cq = (warp - 2) >> 2;
    const int fr = lane >> 2, fc = 2 * (lane & 3);
    bool ok = true;
    int gc = 0;  // chunks drained so far (all tiles)
    for (int q = blockIdx.x; q < p.tiles && ok; q += gridDim.x) {
      const OzTile t = oz_tile<MODE>(p, q);
      float hi[DC], lo[DC];
#pragma unroll
      for (int c = 0; c < DC; ++c) hi[c] = lo[c] = 0.f;
      for (int c = 0; c < nchunks; ++c, ++gc) {
        if (!bar_wait(accf, gc & 1, p.err, 4, p.wait_polls) ||
            (p.err && *(volatile int *)p.err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int f = 0; f < 8; ++f) {
          const uint32_t tl = tmem + ((uint32_t)(lq * 32 + 16 * (f >> 2)) << 16) +
                              (uint32_t)(cq * DC + 8 * (f & 3));
          uint32_t r0[4], r1[4], r2[4], r3[4];
          tmem_ld16x256(tl, r0);
          tmem_ld16x256(tl + 128, r1);
          tmem_ld16x256(tl + 256, r2);
          tmem_ld16x256(tl + 384, r3);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int u = 0; u < 4; ++u)
            fold(hi[4 * f + u], lo[4 * f + u], __uint_as_float(r0[u]), __uint_as_float(r1[u]),
                 __uint_as_float(r2[u]), __uint_as_float(r3[u]));
        }
        // the accumulators are free for the next chunk (of this tile or the next)
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) bar_arrive(acce);
      }
      if (!ok) break;
      // assemble fp64 (while the issuer runs the next tile): C = +-2^(eA + eB - 14) (hi + lo).
      // A thread's four rows: hr = 2 h + (u >> 1), tile row 32 lq + 16 h + fr + 8 (u >> 1).
      double *dst[4];
      int ea[4];
      bool valid[4];
#pragma unroll
      for (int hr = 0; hr < 4; ++hr) {
        const int row = lq * 32 + 16 * (hr >> 1) + fr + 8 * (hr & 1);
        bool v;
        if (MODE == 0) {
          const int i = t.m0 + row;
          v = i < p.M;
          if (v && !OZ_IN(t.zb * p.efa_bs + i, p.efa_cap, 10)) v = false;
          ea[hr] = v ? row_scale(p.efa[t.zb * p.efa_bs + i]) : 0;
          dst[hr] = p.ksplit > 1 ? p.C + (long long)(t.zb * p.ksplit + t.split) * p.M * p.N +
                                       (long long)i * p.N
                                 : p.C + t.zb * p.sC + (long long)i * p.ldc;
        } else {
          const int m = t.mt * 8 + (row >> 4), j = t.jt * 16 + (row & 15);
          v = m < p.M && j < p.M;
          if (!OZ_IN((long long)t.rt * BM + row, p.efa_cap, 11)) v = false;
          ea[hr] = v ? row_scale(p.efa[(long long)t.rt * BM + row]) : 0;
          dst[hr] = p.C + ((long long)j * p.M + m) * p.N;
        }
        valid[hr] = v;
      }
      const int ncol = p.N;
      // the sign of -1 products flips the sign bit only
      const unsigned long long sgn = p.neg ? (1ull << 63) : 0ull;
      const long long eb_off = MODE == 0 && !p.bshared ? t.zb * p.efb_bs : 0;
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        const int j = t.n0 + cq * DC + 8 * (f & 3) + fc;  // this thread's column pair j, j + 1
        if (j >= ncol) continue;
        const bool two = j + 1 < ncol;
        if (!OZ_IN(eb_off + j + (two ? 1 : 0), p.efb_cap, 12)) continue;
        const int eb0 = row_scale(p.efb[eb_off + j]) - 14;
        const int eb1 = two ? row_scale(p.efb[eb_off + j + 1]) - 14 : 0;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const int hr = 2 * (f >> 2) + rr, c = 4 * f + 2 * rr;
          if (!valid[hr]) continue;
          double *d = dst[hr] + j;
          if (!OZ_IN((long long)(d - p.C) + (two ? 1 : 0), p.ccap, 13)) continue;
          const double v0 = __longlong_as_double(
              (long long)((unsigned long long)__double_as_longlong(
                              df_to_f64(hi[c], lo[c], ea[hr] + eb0)) ^
                          sgn));
          if (two) {
            const double v1 = __longlong_as_double(
                (long long)((unsigned long long)__double_as_longlong(
                                df_to_f64(hi[c + 1], lo[c + 1], ea[hr] + eb1)) ^
                            sgn));
            if (p.vec2) {
              *reinterpret_cast<double2 *>(d) = make_double2(v0, v1);
            } else {
              d[0] = v0;
              d[1] = v1;
            }
          } else {
            d[0] = v0;
          }
        }
      }
    }
    // every product the issuer started is complete before tensor memory is freed
    bar_wait(done, 0, p.err, 5, p.wait_polls);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
}

// C[b][i][j] = sum over splits of work[(b ks + s)][i][j], in split order.
__global__ void oz_reduce_kernel(const double *__restrict__ work, int ks, int M, int N, int batch,
                                 double *__restrict__ C, long long ldc, long long sC,
                                 long long ccap) {
  const long long mn = (long long)M * N, tot = mn * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / mn, r = e % mn;
    const int i = (int)(r / N), j = (int)(r % N);
    double s = 0.0;
    for (int k = 0; k < ks; ++k) s += work[(b * ks + k) * mn + r];
    const long long o = b * sC + (long long)i * ldc + j;
    if (OZ_IN(o, ccap, 20)) C[o] = s;
  }
}

// --------------------------------------------------------------- slicing ----
// Tiles of 32 rows x 64 digit columns; the source is read along its
// contiguous index (rows when rs == 1, else columns) through shared memory.
constexpr int SR = 32, SK = 64;
constexpr int KC = 8;  // columns per thread of the digit passes

// Element (b, r, kk) of the view, kk = k1 k2pad + k2 given as (k1, k2).
__device__ __forceinline__ double view_at(const OzView &v, int b, long long r, long long k1,
                                          long long k2) {
  k2 -= v.k2off;
  if (k2 < 0 || k2 >= v.k2n) return 0.0;
  const long long o = b * v.bs + r * v.rs + k1 * v.cs1 + k2 * v.cs2;
#ifdef RSSRI_CHECKS
  if (v.xlen > 0 && (o < 0 || o >= v.xlen)) {
    if (atomicCAS((int *)&g_check_ctx[11], 0, 1) == 0) {
      g_check_ctx[0] = b; g_check_ctx[1] = r; g_check_ctx[2] = k1; g_check_ctx[3] = k2;
      g_check_ctx[4] = v.bs; g_check_ctx[5] = v.rs; g_check_ctx[6] = v.cs1; g_check_ctx[7] = v.cs2;
      g_check_ctx[8] = v.k2pad; g_check_ctx[9] = v.k2n; g_check_ctx[10] = v.xlen;
    }
  }
#endif
  if (!OZ_IN(o, v.xlen, 30)) return 0.0;
  if (v.x2) {
    const float2 f = v.x2[o];
    return (double)f.x + (double)f.y;
  }
  return v.x[o];
}

// Column k of row r of a 32 x 64 shared tile sits at s[r][tile_col(r, k)]: the
// low four bits of k are XORed with bits 4-5 of k (times 2) and with r, so
// that the tile's writes (16 rows at one column, or 16 columns of one row)
// and the digit pass's reads (2 rows x 8 columns 8 apart) each touch 16
// different 8-byte bank pairs per half warp.
__device__ __forceinline__ int tile_col(int r, int k) {
  return k ^ ((((k >> 4) & 3) << 1) ^ (r & 15));
}

// Load a 32 x 64 tile of the view into s (zeros outside); blockDim.x
// == 256, eight values per thread, all eight loads issued before the stores.
constexpr int SLICE_THREADS = 256, SLICE_PER = SR * SK / SLICE_THREADS;
__device__ __forceinline__ void load_tile(const OzView &v, int b, long long r0, long long k0,
                                          int rows, long long K, double (*s)[SK]) {
  const bool rmaj = v.rs == 1;
  const long long k1_0 = k0 / v.k2pad, k2_0 = k0 - k1_0 * v.k2pad;  // once per tile
  double val[SLICE_PER];
#pragma unroll
  for (int i = 0; i < SLICE_PER; ++i) {
    const int idx = threadIdx.x + i * SLICE_THREADS;
    const int r = rmaj ? idx % SR : idx / SK, k = rmaj ? idx / SR : idx % SK;
    const long long rr = r0 + r;
    val[i] = 0.0;
    if (rr < rows && k0 + k < K) {
      long long k1 = k1_0, k2 = k2_0 + k;
      if (k2 >= v.k2pad) {
        const long long q = k2 / v.k2pad;
        k1 += q;
        k2 -= q * v.k2pad;
      }
      val[i] = view_at(v, b, rr, k1, k2);
    }
  }
#pragma unroll
  for (int i = 0; i < SLICE_PER; ++i) {
    const int idx = threadIdx.x + i * SLICE_THREADS;
    const int r = rmaj ? idx % SR : idx / SK, k = rmaj ? idx / SR : idx % SK;
    s[r][tile_col(r, k)] = val[i];
  }
}

__device__ __forceinline__ int ef_of(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

__global__ void __launch_bounds__(256) oz_rowmax_kernel(OzView v, int rows, long long K,
                                                        int *__restrict__ ef) {
  __shared__ double s[SR][SK];
  const int b = blockIdx.z;
  // one tile per block: blockIdx.x = row tile + (rows / SR) * column tile
  const long long rtiles = (rows + SR - 1) / SR;
  const long long r0 = ((long long)blockIdx.x % rtiles) * SR, k0 = ((long long)blockIdx.x / rtiles) * SK;
  load_tile(v, b, r0, k0, rows, K, s);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < SR; r += blockDim.x / 32) {
    int m = max(ef_of(s[r][tile_col(r, lane)]), ef_of(s[r][tile_col(r, lane + 32)]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && r0 + r < rows && m > 0) atomicMax(&ef[(long long)b * rows + r0 + r], m);
  }
}

// The OZ_S balanced base-256 digits of x relative to the row scale 2^e, as
// integers carrying x's sign: x ~ 2^e sum_p dd[p] 2^(-7 - 8 p).
__device__ __forceinline__ void digit_ints(double x, int e, int *dd) {
  const long long bits = __double_as_longlong(x);
  const int efx = (int)((bits >> 52) & 0x7FF);
  unsigned long long M = (unsigned long long)bits & 0xFFFFFFFFFFFFFull;
  if (efx) M |= 1ull << 52;
  // F = round(|x| 2^(FB - e)) = M 2^(max(efx,1) - 1075 + FB - e), FB = 7 + 8 (S - 1)
  // fraction bits; |x| < 2^e makes the shift >= 53 - FB
  constexpr int FB = 7 + 8 * (OZ_S - 1);
  const int sh = 1075 - FB + e - max(efx, 1);
  long long F = 0;
  if (sh < 64) F = (long long)((M + (1ull << (sh - 1))) >> sh);
#pragma unroll
  for (int p = OZ_S - 1; p > 0; --p) {
    int lo8 = (int)(F & 255);
    if (lo8 >= 128) lo8 -= 256;
    dd[p] = lo8;
    F = (F - lo8) >> 8;
  }
  dd[0] = (int)F;
  if (bits < 0) {
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) dd[p] = -dd[p];
  }
}

// Digit p of x0 and of x1 as one bf16 pair (x0 in the low half) for every p.
// A digit d 2^(-8 p) has |d| <= 2^7 + 1, at most 8 significant bits, so its
// bf16 is exactly the upper half of its fp32 pattern; float(d) is formed as
// (1.5 2^23 + d) read from its integer pattern minus 1.5 2^23, so that no
// conversion instruction is needed (the conversion pipe runs at a quarter
// of the fp32 rate and limited the slicer).
__device__ __forceinline__ void digit_pairs(double x0, double x1, int e, uint32_t *w) {
  int a[OZ_S], b[OZ_S];
  digit_ints(x0, e, a);
  digit_ints(x1, e, b);
  const float sc[6] = {1.f, 0x1p-8f, 0x1p-16f, 0x1p-24f, 0x1p-32f, 0x1p-40f};
#pragma unroll
  for (int p = 0; p < OZ_S; ++p) {
    const float fa = (__int_as_float(0x4B400000 + a[p]) - 12582912.0f) * sc[p];
    const float fb = (__int_as_float(0x4B400000 + b[p]) - 12582912.0f) * sc[p];
    w[p] = __byte_perm(__float_as_uint(fa), __float_as_uint(fb), 0x7632);
  }
}

// Offsets of column kk of row br (= b rows + r) in the interleaved digit
// layout (see OzDigits): digit p < 4 at blk 64 + 16 p + u, p >= 4 at
// g1 + blk 32 + 16 (p - 4) + u, blk = br KB + kk / 16, u = kk mod 16.
__device__ __forceinline__ long long digit_off(long long blk, int u, int p, long long g1) {
  return p < 4 ? blk * 64 + 16 * p + u : g1 + blk * 32 + 16 * (p - 4) + u;
}

__global__ void __launch_bounds__(256) oz_digits_kernel(OzView v, int rows, long long K,
                                                        const int *__restrict__ ef,
                                                        __nv_bfloat16 *__restrict__ out,
                                                        long long ld, long long g1) {
  __shared__ double s[SR][SK];
  const int b = blockIdx.z;
  // one tile per block: blockIdx.x = row tile + (rows / SR) * column tile
  const long long rtiles = (rows + SR - 1) / SR;
  const long long r0 = ((long long)blockIdx.x % rtiles) * SR, k0 = ((long long)blockIdx.x / rtiles) * SK;
  load_tile(v, b, r0, k0, rows, K, s);
  __syncthreads();
  // one thread per 8 consecutive columns of one row (256 threads = 32 rows x
  // 8 groups): 16-byte stores into each digit slot
  const int r = threadIdx.x / 8, c0 = (threadIdx.x % 8) * KC;
  const long long rr = r0 + r, kk0 = k0 + c0;
  if (rr >= rows || kk0 >= ld) return;
  const int e = row_scale(ef[(long long)b * rows + rr]);
  uint32_t w[OZ_S][KC / 2];
#pragma unroll
  for (int u = 0; u < KC; u += 2) {
    uint32_t wp[OZ_S];
    digit_pairs(s[r][tile_col(r, c0 + u)], s[r][tile_col(r, c0 + u + 1)], e, wp);
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) w[p][u / 2] = wp[p];
  }
  const long long blk = ((long long)b * rows + rr) * (ld / 16) + (kk0 >> 4);
  if (!OZ_IN(blk * 64 + 63, g1, 31)) return;
#pragma unroll
  for (int p = 0; p < OZ_S; ++p)
    *reinterpret_cast<uint4 *>(out + digit_off(blk, (int)(kk0 & 15), p, g1)) =
        make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// ---------------------------------------- K-contiguous sources (fast path) --
// Views whose rows are contiguous along K (cs2 == 1, one k1 segment), with
// 16-byte aligned rows: each thread takes 8 consecutive columns of one row
// (four 16-byte loads) and, in the digit pass, writes 16 bytes to each of the
// six digit slots.  No shared-memory transpose.

__device__ __forceinline__ void load8(const OzView &v, int b, long long r, long long k0,
                                      long long K, double *x) {
  const long long o = b * v.bs + r * v.rs + k0;
  if (!OZ_IN(o + std::min<long long>(KC, K - k0) - 1, v.xlen, 33)) {
#pragma unroll
    for (int u = 0; u < KC; ++u) x[u] = 0.0;
    return;
  }
  if (k0 + KC <= K) {
    if (v.x2) {
      const float4 *p = reinterpret_cast<const float4 *>(v.x2 + o);
#pragma unroll
      for (int u = 0; u < KC / 2; ++u) {
        const float4 f = p[u];
        x[2 * u] = (double)f.x + (double)f.y;
        x[2 * u + 1] = (double)f.z + (double)f.w;
      }
    } else {
      const double2 *p = reinterpret_cast<const double2 *>(v.x + o);
#pragma unroll
      for (int u = 0; u < KC / 2; ++u) {
        const double2 d = p[u];
        x[2 * u] = d.x;
        x[2 * u + 1] = d.y;
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < KC; ++u)
      x[u] = k0 + u < K ? (v.x2 ? (double)v.x2[o + u].x + (double)v.x2[o + u].y : v.x[o + u])
                        : 0.0;
  }
}

// ef[b][r] = max biased exponent over the row; grid (rows * ceil(K / KCB), 1, batch),
// blockIdx.x = r + rows * (KCB-column block); each thread takes KCB / 2048 groups
// of 8 columns, their loads issued together.
constexpr int KCU = 4, KCB = 256 * KC * KCU;
__global__ void __launch_bounds__(256) oz_rowmax_kc_kernel(OzView v, int rows, long long K,
                                                           int *__restrict__ ef) {
  __shared__ int wm[8];
  const int b = blockIdx.z, r = (int)(blockIdx.x % (unsigned)rows);
  const long long kb = (long long)(blockIdx.x / (unsigned)rows) * KCB;
  int m = 0;
  double x[KCU][KC];
#pragma unroll
  for (int g = 0; g < KCU; ++g) {
    const long long k0 = kb + ((long long)g * 256 + threadIdx.x) * KC;
    if (k0 < K) load8(v, b, r, k0, K, x[g]);
    else
#pragma unroll
      for (int u = 0; u < KC; ++u) x[g][u] = 0.0;
  }
#pragma unroll
  for (int g = 0; g < KCU; ++g)
#pragma unroll
    for (int u = 0; u < KC; ++u) m = max(m, ef_of(x[g][u]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = max(m, wm[w]);
    if (m > 0) atomicMax(&ef[(long long)b * rows + r], m);
  }
}

// Digits of 8 consecutive columns per thread over [batch][rows][ld] (zeros in K..ld).
__global__ void __launch_bounds__(256) oz_digits_kc_kernel(OzView v, int rows, long long K,
                                                           const int *__restrict__ ef,
                                                           __nv_bfloat16 *__restrict__ out,
                                                           long long ld, long long g1) {
  // g1 = batch rows ld 4 values: the chunks of 8 columns are g1 / 32
  const long long cpr = ld / KC, total = g1 / 32;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    const long long br = c / cpr, k0 = (c - br * cpr) * KC;
    const int b = (int)(br / rows);
    const long long r = br - (long long)b * rows;
    double x[KC];
    load8(v, b, r, k0, K, x);
    const int e = row_scale(ef[br]);
    uint32_t w[OZ_S][KC / 2];
#pragma unroll
    for (int u = 0; u < KC; u += 2) {
      uint32_t wp[OZ_S];
      digit_pairs(x[u], x[u + 1], e, wp);
#pragma unroll
      for (int p = 0; p < OZ_S; ++p) w[p][u / 2] = wp[p];
    }
    const long long blk = br * (ld / 16) + (k0 >> 4);
    if (!OZ_IN(blk * 64 + 63, g1, 32)) continue;
#pragma unroll
    for (int p = 0; p < OZ_S; ++p)
      *reinterpret_cast<uint4 *>(out + digit_off(blk, (int)(k0 & 15), p, g1)) =
          make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
  }
}

// Short rows (ld <= 256 NG) of the same sources in one pass: one warp per row
// (grid-stride over batch x rows) holds the row in registers, 8 consecutive
// columns per lane per group, reduces the maximum exponent across the warp
// and writes the digits.  Reads the source once; no shared memory.
template <int NG>
__global__ void __launch_bounds__(256) oz_slice_rowwarp_kernel(OzView v, int rows, long long K,
                                                               long long nrows,
                                                               int *__restrict__ ef,
                                                               __nv_bfloat16 *__restrict__ out,
                                                               long long ld, long long g1) {
  const int lane = threadIdx.x & 31;
  const long long wstride = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long br = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; br < nrows;
       br += wstride) {
    const int b = (int)(br / rows);
    const long long r = br - (long long)b * rows;
    double x[NG][KC];
    int m = 0;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const long long k0 = ((long long)g * 32 + lane) * KC;
      if (k0 < K) {
        load8(v, b, r, k0, K, x[g]);
      } else {
#pragma unroll
        for (int u = 0; u < KC; ++u) x[g][u] = 0.0;
      }
#pragma unroll
      for (int u = 0; u < KC; ++u) m = max(m, ef_of(x[g][u]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) ef[br] = m;
    const int e = row_scale(m);
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const long long k0 = ((long long)g * 32 + lane) * KC;
      if (k0 >= ld) continue;
      uint32_t w[OZ_S][KC / 2];
#pragma unroll
      for (int u = 0; u < KC; u += 2) {
        uint32_t wp[OZ_S];
        digit_pairs(x[g][u], x[g][u + 1], e, wp);
#pragma unroll
        for (int p = 0; p < OZ_S; ++p) w[p][u / 2] = wp[p];
      }
      const long long blk = br * (ld / 16) + (k0 >> 4);
      if (!OZ_IN(blk * 64 + 63, g1, 35)) continue;
#pragma unroll
      for (int p = 0; p < OZ_S; ++p)
        *reinterpret_cast<uint4 *>(out + digit_off(blk, (int)(k0 & 15), p, g1)) =
            make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    }
  }
}

// --------------------------------------- row-contiguous sources (rs == 1) --
// ef of rows whose source is contiguous across rows: one thread per row walks
// RK columns (loads coalesced across the warp, no shared memory); grid
// (ceil(rows / 256), ceil(K / RK), batch).
constexpr int RK = 64;
__global__ void __launch_bounds__(256) oz_rowmax_rmaj_kernel(OzView v, int rows, long long K,
                                                             int *__restrict__ ef) {
  const int b = blockIdx.z;
  const long long r = (long long)blockIdx.x * 256 + threadIdx.x;
  const long long k0 = (long long)blockIdx.y * RK;
  if (r >= rows) return;
  long long k1 = k0 / v.k2pad, k2 = k0 - k1 * v.k2pad;
  const int kn = (int)(K - k0 < RK ? K - k0 : RK);
  int m = 0;
#pragma unroll 8
  for (int u = 0; u < kn; ++u) {
    m = max(m, ef_of(view_at(v, b, r, k1, k2)));
    if (++k2 == v.k2pad) {
      k2 = 0;
      ++k1;
    }
  }
  if (m > 0) atomicMax(&ef[(long long)b * rows + r], m);
}

// Short rows (K <= SHORT_K, one K segment) of a row-contiguous source in one
// pass: a block stages 16 whole rows in shared memory (coalesced 128-byte
// reads across the rows), takes each row's maximum there and writes the
// digits along K in 16-byte stores; ef is written, not accumulated.
constexpr int SHORT_K = 256, SHORT_R = 16;
// Row r of column kk sits at s[kk][r ^ ((kk >> 3) & 15)]: with the odd row
// stride, a half warp's 16 rows at one column and the digit pass's 16 column
// groups 8 apart in one row each fall on 16 different 8-byte bank pairs.
__device__ __forceinline__ int short_col(int kk, int r) { return r ^ ((kk >> 3) & 15); }
__global__ void __launch_bounds__(256) oz_slice_short_kernel(OzView v, int rows, long long K,
                                                             int *__restrict__ ef,
                                                             __nv_bfloat16 *__restrict__ out,
                                                             long long ld, long long g1) {
  __shared__ double s[SHORT_K][SHORT_R + 1];
  __shared__ int wm[256 / SHORT_R][SHORT_R];
  __shared__ int es[SHORT_R];
  const int b = blockIdx.z;
  const long long r0 = (long long)blockIdx.x * SHORT_R;
  const int t = threadIdx.x, kn = (int)K;
  // all of a thread's loads are issued before any is stored: the 16 rows of a
  // column are one 128-byte piece and the columns lie far apart, so the
  // pass needs many loads in flight per SM
  constexpr int LPT = SHORT_K * SHORT_R / 256;
  double val[LPT];
#pragma unroll
  for (int i = 0; i < LPT; ++i) {
    const int idx = t + i * 256, r = idx % SHORT_R, kk = idx / SHORT_R;
    val[i] = kk < kn && r0 + r < rows ? view_at(v, b, r0 + r, 0, kk) : 0.0;
  }
#pragma unroll
  for (int i = 0; i < LPT; ++i) {
    const int idx = t + i * 256, r = idx % SHORT_R, kk = idx / SHORT_R;
    if (kk < kn) s[kk][short_col(kk, r)] = val[i];
  }
  __syncthreads();
  {
    const int r = t % SHORT_R, part = t / SHORT_R;
    int m = 0;
    for (int kk = part; kk < kn; kk += 256 / SHORT_R)
      m = max(m, ef_of(s[kk][short_col(kk, r)]));
    wm[part][r] = m;
  }
  __syncthreads();
  if (t < SHORT_R) {
    int m = 0;
    for (int q = 0; q < 256 / SHORT_R; ++q) m = max(m, wm[q][t]);
    es[t] = m;
    if (r0 + t < rows) ef[(long long)b * rows + r0 + t] = m;
  }
  __syncthreads();
  const int cpr = (int)(ld / KC);
  for (int c = t; c < SHORT_R * cpr; c += 256) {
    const int r = c / cpr, k0 = (c - r * cpr) * KC;
    if (r0 + r >= rows) continue;
    const int e = row_scale(es[r]);
    uint32_t w[OZ_S][KC / 2];
#pragma unroll
    for (int u = 0; u < KC; u += 2) {
      uint32_t wp[OZ_S];
      digit_pairs(k0 + u < kn ? s[k0 + u][short_col(k0 + u, r)] : 0.0,
                  k0 + u + 1 < kn ? s[k0 + u + 1][short_col(k0 + u + 1, r)] : 0.0, e, wp);
#pragma unroll
      for (int p = 0; p < OZ_S; ++p) w[p][u / 2] = wp[p];
    }
    const long long blk = ((long long)b * rows + r0 + r) * (ld / 16) + (k0 >> 4);
    if (!OZ_IN(blk * 64 + 63, g1, 34)) continue;
#pragma unroll
    for (int p = 0; p < OZ_S; ++p)
      *reinterpret_cast<uint4 *>(out + digit_off(blk, k0 & 15, p, g1)) =
          make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
  }
}

// ---------------------------------------------------- exchange operand -----
__global__ void oz_exch_gather_kernel(int n, int bk, int nl16, int jtiles, long long kx,
                                      const double *__restrict__ D, int P,
                                      const int *__restrict__ pidx, double *__restrict__ xs,
                                      long long xs_cap) {
  const int rt = blockIdx.y;
  const int mt = rt / jtiles, jt = rt % jtiles;
  const long long lw = (long long)nl16 * KS;
  const int llo = (jt * 16 - bk) & ~7;
  double *dst = xs + (long long)rt * BM * kx;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < BM * kx;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / kx);
    const long long kk = e - (long long)r * kx;
    const int m = mt * 8 + (r >> 4), j = jt * 16 + (r & 15);
    const int k = mt * 8 - bk + (int)(kk / lw), l = llo + (int)(kk % lw);
    double v = 0.0;
    if (m < n && j < n && k >= 0 && k < n && l >= 0 && l < n) {
      const int a = pidx[m * n + k], c = pidx[l * n + j];
      if (a >= 0 && c >= 0 && OZ_IN(a, P, 40) && OZ_IN(c, P, 41)) v = D[(long long)a * P + c];
    }
    if (OZ_IN((long long)rt * BM * kx + e, xs_cap, 42)) dst[e] = v;
  }
}

__global__ void oz_rows_kp_kernel(const double *__restrict__ KP, const int *__restrict__ rowptr,
                                  int n, int na, int W, double *__restrict__ out) {
  const long long tot = (long long)n * na * W;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % W);
    const long long iq = e / W;
    const int q = (int)(iq % na), i = (int)(iq / na);
    const int a = rowptr[i] + c;
    out[e] = a < rowptr[i + 1] ? KP[(long long)a * na + q] : 0.0;
  }
}

__global__ void oz_rows_g_kernel(const double *__restrict__ G, const int *__restrict__ rowptr,
                                 const int *__restrict__ pcol, int n, int W,
                                 double *__restrict__ out) {
  const long long tot = (long long)n * n * W;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % W);
    const long long im = e / W;
    const int m = (int)(im % n), i = (int)(im / n);
    const int a = rowptr[i] + c;
    out[e] = a < rowptr[i + 1] ? G[(long long)pcol[a] * n + m] : 0.0;
  }
}

__global__ void oz_pair_index_kernel(const int *__restrict__ pij, int P, int n,
                                     int *__restrict__ pidx) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < P; a += gridDim.x * blockDim.x)
    if (OZ_IN(pij[a], (long long)n * n, 50)) pidx[pij[a]] = a;
}

__global__ void oz_fold_kernel(const int *__restrict__ prow, const int *__restrict__ pcol,
                               const double *__restrict__ L, int P, int n, int na,
                               double *__restrict__ U) {
  const long long tot = (long long)P * na;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / na), q = (int)(e % na);
    const long long o = ((long long)pcol[a] * n + prow[a]) * na + q;
    if (OZ_IN(o, (long long)n * n * na, 51)) U[o] += 2.0 * L[e];
  }
}

// --------------------------------------------------------------- host ------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;

void load_encode() {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
}

// 4D bf16 map: dims d[0..3] (elements), strides s[0..2] (bytes, of dims 1..3),
// box b[0..3], swizzle of 128 bytes (b[0] = 64) or 64 bytes (b[0] = 32).
cudaError_t make_map4(CUtensorMap *m, const void *base, const cuuint64_t d[4],
                      const cuuint64_t s[3], const cuuint32_t b[4]) {
  if (!g_encode) return cudaErrorNotSupported;
  if ((uintptr_t)base % 16) return cudaErrorInvalidValue;
  for (int k = 0; k < 3; ++k)
    if (s[k] % 16) return cudaErrorInvalidValue;
  if (b[0] != 64 && b[0] != 32) return cudaErrorInvalidValue;
  cuuint64_t dims[4] = {d[0], d[1], d[2], d[3]};
  cuuint64_t strides[3] = {s[0], s[1], s[2]};
  cuuint32_t box[4] = {b[0], b[1], b[2], b[3]};
  cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base),
                              dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              b[0] == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The two maps of a digit operand (digits 0-3 and 4-5, see OzDigits): dims
// (slot width, K blocks, rows, batch), box (width, 1, 128, 1).
cudaError_t digit_maps(CUtensorMap *m0, CUtensorMap *m1, const OzDigits &o) {
  const cuuint64_t kb = (cuuint64_t)(o.ld / 16);
  const __nv_bfloat16 *g1 = o.d + (long long)o.batch * o.rows * o.ld * 4;
  {
    const cuuint64_t d[4] = {64, kb, (cuuint64_t)o.rows, (cuuint64_t)o.batch};
    const cuuint64_t st[3] = {128, kb * 128, kb * 128 * o.rows};
    const cuuint32_t b[4] = {64, 1, BM, 1};
    RS_TRY(make_map4(m0, o.d, d, st, b));
  }
  const cuuint64_t d[4] = {32, kb, (cuuint64_t)o.rows, (cuuint64_t)o.batch};
  const cuuint64_t st[3] = {64, kb * 64, kb * 64 * o.rows};
  const cuuint32_t b[4] = {32, 1, BM, 1};
  return make_map4(m1, g1, d, st, b);
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

cudaError_t prepare() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  RS_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!done[dev]) {
    RS_TRY(cudaFuncSetAttribute(oz_gemm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SMEM));
    RS_TRY(cudaFuncSetAttribute(oz_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SMEM));
    // the launch needs THREADS threads at the kernel's register count
    cudaFuncAttributes fa;
    RS_TRY(cudaFuncGetAttributes(&fa, oz_gemm_kernel<0>));
    if (fa.maxThreadsPerBlock < THREADS) return cudaErrorLaunchOutOfResources;
    done[dev] = true;
  }
  return cudaSuccess;
}

// K splits of a dense product: when its output tiles leave SMs idle, K is
// split so that the rounds of tiles over the SMs times the K steps of a split,
// plus the split partials' extra traffic, is least.  Costs in units of one K
// step of one tile (21 digit products of 128 x 128 x 16, ~0.9 us at the
// tensor rate): a tile's drain and stores ~9 steps; the partials are written
// and read back at ~5.3 MB per step (HBM), plus ~6 steps for the reduction launch.
void plan(const OzGemm &g, int *ksplit, int *kst) {
  const int steps = ceil_div(g.A.K, KS);
  const long long tiles = (long long)ceil_div(g.M, BM) * ceil_div(g.N, BN) * g.batch;
  const long long sms = 152;
  int best_per = steps;
  if (tiles < 4 * sms && steps >= 2) {
    double best = (double)((tiles + sms - 1) / sms) * (steps + 9);
    const double part = (double)g.M * g.N * g.batch * 8.0 / 5.3e6;
    const int maxks = std::min(64, steps);
    for (int ks = 2; ks <= maxks; ++ks) {
      const int per = ceil_div(steps, ks);
      const int kp = ceil_div(steps, per);  // splits actually made
      if (kp != ks) continue;
      const double cost =
          (double)((tiles * kp + sms - 1) / sms) * (per + 9) + (kp + 1) * part + 6.0;
      if (cost < best) {
        best = cost;
        best_per = per;
      }
    }
  }
  *kst = best_per;
  *ksplit = ceil_div(steps, best_per);
}

// Tile order of a dense product.  The CTAs run in waves of one tile per SM
// over consecutive queue entries and read each K window of the waves' row
// tiles of A and column tiles of B about together, so a wave reads from HBM
// the distinct m tiles and n tiles it spans; an operand held whole in L2
// (~64 MB of digits at most) is read once.  m-fastest when that reads less.
bool m_fastest(const OzGemm &g) {
  const long long mt = ceil_div(g.M, BM), nt = ceil_div(g.N, BN), sms = 152;
  const double kb = (double)g.A.K * OZ_S * 2.0;  // digit bytes of one row
  const bool a_l2 = (double)g.M * kb * g.A.batch <= 64e6;
  const bool b_l2 = (double)g.N * kb * g.B.batch <= 64e6;
  const long long wn = std::min(nt, sms), wm = std::min(mt, sms);
  // n fastest: a wave spans min(nt, sms) n tiles and ~sms / nt m tiles
  const double cn = (b_l2 ? 0.0 : (double)wn) + (a_l2 ? 0.0 : (double)ceil_div(sms, wn));
  const double cm = (a_l2 ? 0.0 : (double)wm) + (b_l2 ? 0.0 : (double)ceil_div(sms, wm));
  return cm < cn;
}

}  // namespace

cudaError_t oz_check_fetch(int out[4]) {
  RS_TRY(cudaMemcpyFromSymbol(out, g_check, 4 * sizeof(int)));
#ifdef RSSRI_CHECKS
  long long ctx[12];
  RS_TRY(cudaMemcpyFromSymbol(ctx, g_check_ctx, sizeof(ctx)));
  if (ctx[11])
    fprintf(stderr,
            "view read: b %lld r %lld k1 %lld k2 %lld | bs %lld rs %lld cs1 %lld cs2 %lld k2pad "
            "%lld k2n %lld xlen %lld\n",
            ctx[0], ctx[1], ctx[2], ctx[3], ctx[4], ctx[5], ctx[6], ctx[7], ctx[8], ctx[9], ctx[10]);
#endif
  const int zero[4] = {0, 0, 0, 0};
  return cudaMemcpyToSymbol(g_check, zero, 4 * sizeof(int));
}

int oz_kernel_regs(int *max_threads) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, oz_gemm_kernel<0>) != cudaSuccess) return -1;
  if (max_threads) *max_threads = fa.maxThreadsPerBlock;
  return fa.numRegs;
}

bool oz_available() {
  std::call_once(g_once, load_encode);
  return g_encode != nullptr;
}

cudaError_t oz_slice(const OzView &v, const OzDigits &out, cudaStream_t s) {
  if (out.rows <= 0 || out.K <= 0 || out.batch <= 0) return cudaSuccess;
  if (out.ld < out.K || (out.ld % 16) || v.k2pad <= 0) return cudaErrorInvalidValue;
  // start of the digits 4-5 group (see OzDigits)
  const long long g1 = (long long)out.batch * out.rows * out.ld * 4;
  RS_TRY(cudaMemsetAsync(out.ef, 0, (size_t)out.batch * out.rows * sizeof(int), s));
  if (out.batch > 65535) return cudaErrorInvalidValue;
  const long long rtiles = ((long long)out.rows + SR - 1) / SR;
  // rows contiguous along K, 16-byte aligned: the vectorised path
  const uintptr_t base = v.x2 ? (uintptr_t)v.x2 : (uintptr_t)v.x;
  const long long kcb = (out.K + KCB - 1) / KCB;  // column blocks of the maximum pass
  const bool kc = v.cs2 == 1 && v.k2off == 0 && v.k2pad >= out.K && v.k2n >= out.K &&
                  base % 16 == 0 && v.rs % 2 == 0 && v.bs % 2 == 0 &&
                  kcb * out.rows <= 0x7FFFFFFFLL;
  if (kc && out.ld <= 256 * 4) {
    const long long nrows = (long long)out.batch * out.rows;
    const int grid = (int)std::min<long long>(ceil_div(nrows, 8LL), 152LL * 16);
    if (out.ld <= 256)
      oz_slice_rowwarp_kernel<1><<<grid, 256, 0, s>>>(v, out.rows, out.K, nrows, out.ef, out.d,
                                                      out.ld, g1);
    else if (out.ld <= 512)
      oz_slice_rowwarp_kernel<2><<<grid, 256, 0, s>>>(v, out.rows, out.K, nrows, out.ef, out.d,
                                                      out.ld, g1);
    else
      oz_slice_rowwarp_kernel<4><<<grid, 256, 0, s>>>(v, out.rows, out.K, nrows, out.ef, out.d,
                                                      out.ld, g1);
    ++launch_counter();
    return cudaGetLastError();
  }
  if (kc) {
    dim3 gm((unsigned)(kcb * out.rows), 1, out.batch);
    oz_rowmax_kc_kernel<<<gm, 256, 0, s>>>(v, out.rows, out.K, out.ef);
    ++launch_counter();
    RS_TRY(cudaGetLastError());
    const long long chunks = (long long)out.batch * out.rows * out.ld / KC;
    const int grid = (int)std::min<long long>(ceil_div(chunks, 256LL), 152LL * 16);
    oz_digits_kc_kernel<<<grid, 256, 0, s>>>(v, out.rows, out.K, out.ef, out.d, out.ld, g1);
    ++launch_counter();
    return cudaGetLastError();
  }
  if (v.rs == 1 && v.k2off == 0 && v.k2pad >= out.K && out.K <= SHORT_K && out.ld <= SHORT_K) {
    dim3 g(ceil_div(out.rows, SHORT_R), 1, out.batch);
    oz_slice_short_kernel<<<g, 256, 0, s>>>(v, out.rows, out.K, out.ef, out.d, out.ld, g1);
    ++launch_counter();
    return cudaGetLastError();
  }
  if (v.rs == 1) {
    if (ceil_div(out.K, RK) > 65535) return cudaErrorInvalidValue;
    dim3 gm(ceil_div(out.rows, 256), ceil_div(out.K, RK), out.batch);
    oz_rowmax_rmaj_kernel<<<gm, 256, 0, s>>>(v, out.rows, out.K, out.ef);
  } else {
    const long long tiles = rtiles * ((out.K + SK - 1) / SK);
    if (tiles > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
    dim3 gm((unsigned)tiles, 1, out.batch);
    oz_rowmax_kernel<<<gm, 256, 0, s>>>(v, out.rows, out.K, out.ef);
  }
  ++launch_counter();
  RS_TRY(cudaGetLastError());
  // the digit pass covers the padding columns K..ld too (zeros)
  const long long dtiles = rtiles * ((out.ld + SK - 1) / SK);
  if (dtiles > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  dim3 gd((unsigned)dtiles, 1, out.batch);
  oz_digits_kernel<<<gd, 256, 0, s>>>(v, out.rows, out.K, out.ef, out.d, out.ld, g1);
  ++launch_counter();
  return cudaGetLastError();
}

size_t oz_gemm_work(const OzGemm &g) {
  int ks, kst;
  plan(g, &ks, &kst);
  return ks > 1 ? (size_t)ks * g.batch * g.M * g.N : 0;
}

double oz_gemm_flops(const OzGemm &g) {
  int ks, kst;
  plan(g, &ks, &kst);
  return OZ_PRODUCTS * 2.0 * BM * BN * KS * (double)kst * ks * ceil_div(g.M, BM) *
         ceil_div(g.N, BN) * g.batch;
}

cudaError_t oz_gemm(const OzGemm &g, double *work, size_t work_elems, cudaStream_t s) {
  if (!oz_available()) return cudaErrorNotSupported;
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.A.K != g.B.K || g.A.rows != g.M || g.B.rows != g.N || g.A.batch != g.batch ||
      (g.B.batch != 1 && g.B.batch != g.batch))
    return cudaErrorInvalidValue;
  if (g.A.K <= 0 || (g.alpha != 1.0 && g.alpha != -1.0)) return cudaErrorInvalidValue;
  int ks, kst;
  plan(g, &ks, &kst);
  if (ks > 1 && work_elems < (size_t)ks * g.batch * g.M * g.N) return cudaErrorInvalidValue;
  if ((long long)g.batch * ks > 65535 || ceil_div(g.M, BM) > 65535) return cudaErrorInvalidValue;
  OzParams p;
  std::memset(&p, 0, sizeof(p));
  if (g.A.ld % 16 || g.B.ld % 16) return cudaErrorInvalidValue;
  RS_TRY(digit_maps(&p.ta0, &p.ta1, g.A));
  RS_TRY(digit_maps(&p.tb0, &p.tb1, g.B));
  p.M = g.M;
  p.N = g.N;
  p.kst = kst;
  p.ksplit = ks;
  p.bshared = g.B.batch == 1 && g.batch > 1;
  p.efa = g.A.ef;
  p.efb = g.B.ef;
  p.efa_bs = g.M;
  p.efb_bs = g.N;
  p.neg = g.alpha == -1.0;
  p.C = ks > 1 ? work : g.C;
  p.vec2 = ((uintptr_t)p.C % 16 == 0) &&
           (ks > 1 ? g.N % 2 == 0 : g.ldc % 2 == 0 && (g.batch == 1 || g.sC % 2 == 0));
  p.mfast = m_fastest(g);
  p.ldc = g.ldc;
  p.sC = g.sC;
  p.err = g.err;
  p.ccap = ks > 1 ? (long long)ks * g.batch * g.M * g.N : g.ccap;
  p.efa_cap = (long long)g.A.batch * g.A.rows;
  p.efb_cap = (long long)g.B.batch * g.B.rows;
  p.wait_polls = g.wait_polls;
  RS_TRY(prepare());
  p.ntiles = ceil_div(g.N, BN);
  p.mtiles = ceil_div(g.M, BM);
  const long long tiles = (long long)p.ntiles * p.mtiles * g.batch * ks;
  if (tiles > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  p.tiles = (int)tiles;
  oz_gemm_kernel<0><<<(unsigned)std::min<long long>(tiles, sm_count()), THREADS, SMEM, s>>>(p);
  ++launch_counter();
  RS_TRY(cudaGetLastError());
  if (ks > 1) {
    const long long tot = (long long)g.batch * g.M * g.N;
    oz_reduce_kernel<<<(int)std::min<long long>((tot + 255) / 256, 152 * 8), 256, 0, s>>>(
        work, ks, g.M, g.N, g.batch, g.C, g.ldc, g.sC, g.ccap);
    ++launch_counter();
    RS_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t oz_rows_kp(const double *KP, const int *rowptr, int n, int na, int W, double *out,
                       cudaStream_t s) {
  const long long tot = (long long)n * na * W;
  if (tot <= 0) return cudaSuccess;
  oz_rows_kp_kernel<<<(int)std::min<long long>((tot + 255) / 256, 152 * 16), 256, 0, s>>>(
      KP, rowptr, n, na, W, out);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t oz_rows_g(const double *G, const int *rowptr, const int *pcol, int n, int W,
                      double *out, cudaStream_t s) {
  const long long tot = (long long)n * n * W;
  if (tot <= 0) return cudaSuccess;
  oz_rows_g_kernel<<<(int)std::min<long long>((tot + 255) / 256, 152 * 16), 256, 0, s>>>(
      G, rowptr, pcol, n, W, out);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t oz_pair_index(const int *pij, int P, int n, int *pidx, cudaStream_t s) {
  RS_TRY(cudaMemsetAsync(pidx, 0xFF, (size_t)n * n * sizeof(int), s));
  if (P <= 0) return cudaSuccess;
  oz_pair_index_kernel<<<std::min(ceil_div(P, 256), 1024), 256, 0, s>>>(pij, P, n, pidx);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t oz_fold_direct(const int *prow, const int *pcol, const double *L, int P, int n,
                           int na, double *U, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  const long long tot = (long long)P * na;
  oz_fold_kernel<<<(int)std::min<long long>((tot + 255) / 256, 152 * 16), 256, 0, s>>>(
      prow, pcol, L, P, n, na, U);
  ++launch_counter();
  return cudaGetLastError();
}

OzExch oz_exch_geometry(int n, int na, int bk) {
  OzExch x;
  x.n = n;
  x.na = na;
  x.bk = bk;
  // l window of the 16-wide j tile at j0 (a multiple of 16): from
  // floor8(j0 - bk) = j0 - ceil8(bk) to j0 + 15 + bk, in nl16 steps of 16
  const int c8 = (bk + 7) / 8 * 8;
  x.nl16 = ceil_div(16 + bk + c8, KS);
  x.mtiles = ceil_div(n, 8);
  x.jtiles = ceil_div(n, 16);
  x.kx = (long long)(8 + 2 * bk) * x.nl16 * KS;
  // l' = l + lsh puts every window start j0 - c8 on a 16-column block
  x.lsh = (16 - c8 % 16) % 16;
  x.lb0 = (x.lsh - c8) / 16;  // exact: lsh - c8 is a multiple of 16
  x.ldl = ((long long)n + x.lsh + 15) / 16 * 16;
  return x;
}

double oz_exch_flops(const OzExch &x) {
  return OZ_PRODUCTS * 2.0 * BM * (double)ceil_div(x.na, BN) * BN * x.kx * x.mtiles * x.jtiles;
}

cudaError_t oz_exch_gather(const OzExch &x, const double *D, int P, const int *pidx, double *xs,
                           long long xs_cap, cudaStream_t s) {
  const int tiles = x.mtiles * x.jtiles;
  if (tiles > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)std::min<long long>(ceil_div(BM * x.kx, 256), 64), tiles);
  oz_exch_gather_kernel<<<grid, 256, 0, s>>>(x.n, x.bk, x.nl16, x.jtiles, x.kx, D, P, pidx, xs,
                                             xs_cap);
  ++launch_counter();
  return cudaGetLastError();
}

cudaError_t oz_exch(const OzExch &x, const OzDigits &X, const OzDigits &At, double *T,
                    long long tcap, double alpha, int *err, cudaStream_t s, int wait_polls) {
  if (!oz_available()) return cudaErrorNotSupported;
  const int tiles = x.mtiles * x.jtiles;
  if (X.batch != tiles || X.rows != BM || X.K != x.kx || At.rows != x.na ||
      At.K != (long long)x.n * x.ldl || At.ld != At.K || At.batch != 1 || tiles > 65535 ||
      X.ld % 16 || x.ldl % 16 || (alpha != 1.0 && alpha != -1.0))
    return cudaErrorInvalidValue;
  OzParams p;
  std::memset(&p, 0, sizeof(p));
  RS_TRY(digit_maps(&p.ta0, &p.ta1, X));
  {
    // right operand as (slot, l' block, k, q): a box is one l' block of 128 q rows
    const cuuint64_t lb = (cuuint64_t)(x.ldl / 16);
    const __nv_bfloat16 *g1 = At.d + (long long)x.na * x.n * x.ldl * 4;
    const cuuint64_t d0[4] = {64, lb, (cuuint64_t)x.n, (cuuint64_t)x.na};
    const cuuint64_t s0[3] = {128, lb * 128, lb * 128 * x.n};
    const cuuint32_t b0[4] = {64, 1, 1, BM};
    RS_TRY(make_map4(&p.tb0, At.d, d0, s0, b0));
    const cuuint64_t d1[4] = {32, lb, (cuuint64_t)x.n, (cuuint64_t)x.na};
    const cuuint64_t s1[3] = {64, lb * 64, lb * 64 * x.n};
    const cuuint32_t b1[4] = {32, 1, 1, BM};
    RS_TRY(make_map4(&p.tb1, g1, d1, s1, b1));
  }
  p.M = x.n;
  p.N = x.na;
  p.kst = (int)(x.kx / KS);
  p.ksplit = 1;
  p.efa = X.ef;
  p.efb = At.ef;
  p.neg = alpha == -1.0;
  p.vec2 = ((uintptr_t)T % 16 == 0) && x.na % 2 == 0;
  p.C = T;
  p.bk = x.bk;
  p.lb0 = x.lb0;
  p.nl16 = x.nl16;
  p.jtiles = x.jtiles;
  p.err = err;
  p.ccap = tcap;
  p.efa_cap = (long long)X.batch * X.rows;
  p.efb_cap = (long long)At.batch * At.rows;
  p.wait_polls = wait_polls;
  RS_TRY(prepare());
  p.ntiles = ceil_div(x.na, BN);
  p.mtiles = 1;
  p.tiles = p.ntiles * tiles;
  oz_gemm_kernel<1><<<(unsigned)std::min(p.tiles, sm_count()), THREADS, SMEM, s>>>(p);
  ++launch_counter();
  return cudaGetLastError();
}

}  // namespace rssri
