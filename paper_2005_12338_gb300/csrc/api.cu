// C ABI of librssri: handle, validation and the order of the steps of the
// RS-SRI-GF2 self-energy path (see include/rssri.h for the contract).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "chain_tc.cuh"
#include "cv_mlp.cuh"
#include "dd_df64.cuh"
#include "kernels.cuh"
#include "oz_gemm.cuh"
#include "tc_gemm.cuh"
#include "tc_group.cuh"

using namespace rssri;

namespace {
thread_local char g_err_site[96] = "";
}  // namespace

namespace rssri {
void note_error_site(const char *file, int line) {
  if (g_err_site[0]) return;
  const char *base = std::strrchr(file, '/');
  std::snprintf(g_err_site, sizeof g_err_site, "%s:%d", base ? base + 1 : file, line);
}
}  // namespace rssri

namespace {

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  template <class T> T *as() const { return static_cast<T *>(p); }
};

// Testing: the device allocation (counted from 1 within one API call) that is
// made to fail without calling the allocator; 0 = none (rssri_options.test_fail_alloc).
thread_local int g_fail_alloc_at = 0, g_alloc_count = 0;

struct AllocFailScope {
  explicit AllocFailScope(int k) {
    g_fail_alloc_at = k;
    g_alloc_count = 0;
  }
  ~AllocFailScope() { g_fail_alloc_at = 0; }
};

cudaError_t ensure(DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return cudaSuccess;
  if (g_fail_alloc_at > 0 && ++g_alloc_count == g_fail_alloc_at) return cudaErrorMemoryAllocation;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  RS_TRY(cudaMalloc(&b.p, bytes));
  b.bytes = bytes;
  return cudaSuccess;
}

void release(DevBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

thread_local char g_last_cuda[192] = "";

int map_err(cudaError_t e) {
  if (e == cudaSuccess) return RSSRI_OK;
  std::snprintf(g_last_cuda, sizeof g_last_cuda, "%s%s%s", cudaGetErrorName(e),
                g_err_site[0] ? " at " : "", g_err_site);
  g_err_site[0] = 0;
  if (e == cudaErrorMemoryAllocation) return RSSRI_ERR_OOM;
  return RSSRI_ERR_CUDA;
}

}  // namespace

struct rssri_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev[8] = {};  // 6, 7: the control variate's coefficients
  // results of an enqueued sigma call, copied into pinned host memory:
  // [0..3] the energy scalars, then the tensor-core timeout flag
  double *host_res = nullptr;
  bool pending = false, pending_tc = false;
  int pending_ns = 0;
  bool ready = false;
  bool broken = false;

  // problem
  int n = 0, n_occ = 0, n_aux = 0, n_tau = 0;
  double mu = 0, beta = 0, eps_prime = 0, eps = 0;
  int ptr_kind = RSSRI_PTR_DEVICE;
  const double *eri3 = nullptr, *metric = nullptr, *orb_e = nullptr, *orb_c = nullptr,
               *tau = nullptr, *tau_w = nullptr;
  DevBuf in_eri3, in_metric, in_orb_e, in_orb_c, in_tau, in_tau_w;
  std::vector<double> h_tau_w;

  // setup products
  DevBuf W, nsY, nsZ, nsP, nsT, nsY2, nsZ2, scal, part, flags;
  DevBuf colmax, cnt, cscratch, cnum, csum, spairs, EL, KLs, cnt2, lidx, pij, prow, pcol, rowptr,
      KP, D;
  int P_s = 0, P = 0;
  long long nnz_eri_l = 0, nnz_k_l = 0;
  double k_l_max = 0, ns_resid = 0;
  int ns_iters = 0;
  float t_setup_ms = 0;

  // sigma buffers
  DevBuf theta, Ut, fac, RLp, G, Gb, cs, XG, Cc, Bm, BC, tarr, sarr, e_st, sig_raw, sdd, PG, At,
      T, AP, Gam, L, trdd, tr, res, sig_out, e_pair, gwork, outbuf;
  // learned control variate
  DevBuf cv_params, cv_m, cv_v, cv_grad, cv_ptmp, cv_act, cv_work, cv_X, cv_t, cv_w, cv_stats, cv_c,
      cv_scr, cv_bx, cv_bt, cv_bw, cv_loss;
  bool cv_ready = false, cv_c_ready = false;
  bool pending_cv_c = false;  // the last sampling call computed c
  // double-float copies for the exchange contraction
  DevBuf Dhl, Ahl, KPhl, PGhl, APhl, Gamhl, GGhl;
  // literal estimator: pair gathers / J, aux traces, pair form of the batch
  DevBuf litMP, litT, litMhl;
  // pairs of (ij|A) and of U^T / theta for the double-float factor products
  DevBuf eri_hl, ut_hl;
  // pair copies of the Newton-Schulz operands (double-float metric root)
  DevBuf nsA2, nsB2;
  DevBuf elHl;  // (ij|A)^L rows as pairs (double-float [K]^L)
  // double-float chain: factor pairs, X G and C pairs, (2tI - B) pairs
  DevBuf facHl, xgHl, cHl, bHl;
  bool d_df64_ready = false;
  bool kp_hl_ready = false;  // K_P as pairs (KPhl) made for this setup
  // bf16 chain buffers
  DevBuf hxsl, hy3, hg, hgb, hP, hdc32, hcl32, hdcl16, hxy32, ha6, hct, hdct, hpart, hfold;
  DevBuf hclt, hfl;  // learned control variate on the tensor-core chain: (C^L)^T, F^L per pair
  // the bf16 chain captured as a CUDA graph, valid for the key it was built for
  cudaGraphExec_t chain_graph = nullptr;
  cudaStream_t cap_stream = nullptr;  // captures run here (the legacy stream cannot capture)
  std::vector<uintptr_t> chain_key_ptr;
  std::vector<double> chain_key_w;
  long long chain_graph_launches = 0;
  long long last_ns = 0;
  bool have_sigma = false;
  // The deterministic block (S6, S7) of the last build: G, Gb and Sigma_DD for
  // every tau.  rssri_setup builds it for the orbitals' G with the setup's
  // dd_arith and rssri_sigma reuses it; rssri_sigma_from_g rebuilds it for the
  // caller's G, after which the next rssri_sigma rebuilds the orbitals' block.
  bool block_ok = false, block_from_g = false;
  int setup_arith = RSSRI_DD_FP64;
  bool gg_valid = false;  // GGhl holds the pair split of the current G, Gb
  bool pending_block = false;  // the enqueued sigma call rebuilt the block
  int test_wait_polls = 0;     // rssri_options.test_wait_polls of the current call
  DevBuf sdd0;            // zeros: the block of the plain stochastic-RI estimator
  // the sliced (RSSRI_DD_OZ) block: pair index map, the exchange contraction's
  // left operand and the digits of K_P (setup); per-tau digit buffers
  struct OzBuf {
    DevBuf d, e;
    OzDigits v;
  };
  bool oz_ready = false;
  OzExch oz_geo;
  DevBuf oz_gs, oz_gexp;  // G(tau) 2^-e(tau) as pairs, and e(tau), for K^Q G
  DevBuf oz_pidx, oz_tmp;
  OzBuf ozX, ozKP, ozKPt, ozGb, ozBig0, ozBig1, ozAtP, ozGam;
  OzBuf ozPA, ozPB;  // operands of the setup and factor products (RSSRI_DD_OZ)
  OzBuf ozKPr, ozGr;  // row-batched operands of K^Q G (see oz_rows_kp)
  DevBuf oz_gr;       // G gathered by pair rows, fp64 [n][n][oz_w]
  int oz_w = 0;       // longest row of the pair list, rounded up to 16
  rssri_stats stats{};

  // per-class launch counts and (when profiling) event timings
  struct Rec {
    int cls;
    double gflop, tgflop;
    long long launches;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<cudaEvent_t> evpool;
  size_t ev_used = 0;
  std::vector<Rec> recs;
  long long setup_launches[RSSRI_PROF_NCLASS] = {};
  double setup_ms[RSSRI_PROF_NCLASS] = {}, setup_gflop[RSSRI_PROF_NCLASS] = {},
         setup_tgflop[RSSRI_PROF_NCLASS] = {};
};

namespace {

// Device flags (ints): [4] tensor-core chain timeout, [5] sliced-block timeout,
// [8..10] the double-float range check (flag, running maximum, block count).
int *range_flag(rssri_handle *h) { return h->flags.as<int>() + 8; }

// ------------------------------------------------------------ profiling ----
cudaEvent_t take_event(rssri_handle *h) {
  if (h->ev_used == h->evpool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->evpool.push_back(e);
  }
  return h->evpool[h->ev_used++];
}

// One group of launches of one kernel class; records its launch count and,
// when profiling, CUDA events around it on the handle's stream.
struct Span {
  rssri_handle *h;
  int cls;
  double gflop, tgflop;
  long long l0;
  cudaEvent_t a = nullptr;
  Span(rssri_handle *h_, int c, double gf, double tgf = 0.0)
      : h(h_), cls(c), gflop(gf), tgflop(tgf), l0(launch_counter()) {
    if (h->prof_on) {
      a = take_event(h);
      if (a && cudaEventRecord(a, h->stream) != cudaSuccess) a = nullptr;
    }
  }
  ~Span() {
    cudaEvent_t b = nullptr;
    if (a) {
      b = take_event(h);
      if (b && cudaEventRecord(b, h->stream) != cudaSuccess) b = nullptr;
    }
    h->recs.push_back({cls, gflop, tgflop, launch_counter() - l0, a, b});
  }
};
#define SPAN(cls, gf) Span span_(h, (cls), (gf))
#define SPAN_T(cls, gf, tgf) Span span_(h, (cls), (gf), (tgf))

// Sum the recorded spans (the stream must have completed them) and reset.
void collect(rssri_handle *h, long long *launches, double *ms, double *gflop, double *tgflop) {
  for (int c = 0; c < RSSRI_PROF_NCLASS; ++c) {
    launches[c] = 0;
    ms[c] = 0;
    gflop[c] = 0;
    tgflop[c] = 0;
  }
  for (const auto &r : h->recs) {
    launches[r.cls] += r.launches;
    gflop[r.cls] += r.gflop;
    tgflop[r.cls] += r.tgflop;
    float t = 0;
    if (r.a && r.b && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.cls] += t;
  }
  h->recs.clear();
  h->ev_used = 0;
}

// ----------------------------------------------------------- validation ----
bool finite(double x) { return std::isfinite(x); }

int validate_problem(const rssri_problem *p) {
  if (!p) return RSSRI_ERR_INVALID_ARG;
  if (p->n < 1 || p->n > 4096 || p->n_occ < 1 || p->n_occ > p->n - 1 || p->n_aux < 1 ||
      p->n_aux >= (1 << 20) || p->n_tau < 1)
    return RSSRI_ERR_INVALID_ARG;
  if ((long long)p->n * p->n * (long long)p->n_aux > (1LL << 40)) return RSSRI_ERR_INVALID_ARG;
  if (p->ptr_kind != RSSRI_PTR_DEVICE && p->ptr_kind != RSSRI_PTR_HOST)
    return RSSRI_ERR_INVALID_ARG;
  if (!p->eri3 || !p->metric || !p->orb_e || !p->orb_c || !p->tau || !p->tau_w)
    return RSSRI_ERR_INVALID_ARG;
  if (!finite(p->mu) || !finite(p->beta) || !(p->beta > 0)) return RSSRI_ERR_INVALID_ARG;
  return RSSRI_OK;
}

int validate_options(const rssri_options *o, bool for_sigma) {
  if (!o) return RSSRI_ERR_INVALID_ARG;
  if (!(o->eps_prime >= 0.0 && o->eps_prime <= 1.0) || !(o->eps >= 0.0 && o->eps <= 1.0))
    return RSSRI_ERR_INVALID_ARG;
  if (o->dd_arith != RSSRI_DD_FP64 && o->dd_arith != RSSRI_DD_DF64 && o->dd_arith != RSSRI_DD_OZ)
    return RSSRI_ERR_INVALID_ARG;
  if (o->dd_arith == RSSRI_DD_OZ && !oz_available()) return RSSRI_ERR_INVALID_ARG;
  if (o->test_wait_polls < 0 || o->test_fail_alloc < 0) return RSSRI_ERR_INVALID_ARG;
  if (for_sigma) {
    if (o->n_s < 2 || o->n_s > (1LL << 30) || o->xi_offset < 0 ||
        o->xi_offset + o->n_s >= (1LL << 40))
      return RSSRI_ERR_INVALID_ARG;
    if (o->estimator != RSSRI_EST_CV && o->estimator != RSSRI_EST_SRI &&
        o->estimator != RSSRI_EST_LITERAL)
      return RSSRI_ERR_INVALID_ARG;
    if (o->estimator == RSSRI_EST_LITERAL && (o->precision != RSSRI_PREC_FP64 || o->cv != 0))
      return RSSRI_ERR_INVALID_ARG;
    if (o->precision != RSSRI_PREC_FP64 && o->precision != RSSRI_PREC_BF16 &&
        o->precision != RSSRI_PREC_TF32 && o->precision != RSSRI_PREC_DF64)
      return RSSRI_ERR_INVALID_ARG;
    if (o->pair_batch < 0) return RSSRI_ERR_INVALID_ARG;
    if (o->cv != 0 && o->cv != 1) return RSSRI_ERR_INVALID_ARG;
  }
  return RSSRI_OK;
}

cudaError_t stage(DevBuf &dst, const double *src, size_t count, int kind, cudaStream_t s,
                  const double **out) {
  if (kind == RSSRI_PTR_DEVICE) {
    *out = src;
    return cudaSuccess;
  }
  RS_TRY(ensure(dst, count * sizeof(double)));
  RS_TRY(cudaMemcpyAsync(dst.p, src, count * sizeof(double), cudaMemcpyHostToDevice, s));
  *out = dst.as<double>();
  return cudaSuccess;
}

// Copy a small device value to the host (synchronous on the stream).
template <class T> cudaError_t fetch(T *h, const void *d, cudaStream_t s, size_t count = 1) {
  RS_TRY(cudaMemcpyAsync(h, d, sizeof(T) * count, cudaMemcpyDeviceToHost, s));
  return cudaStreamSynchronize(s);
}

// Every product goes through here: grows the split-K scratch when needed.
cudaError_t gemm(rssri_handle *h, const GemmArgs &g) {
  const size_t need = dgemm_work_elems(g) * sizeof(double);
  if (need > h->gwork.bytes) RS_TRY(ensure(h->gwork, need));
  return dgemm(g, h->gwork.as<double>(), h->gwork.bytes / sizeof(double), h->stream);
}

// A product counted under kernel class `cls` with its 2 M N K batch flops.
cudaError_t gemm_p(rssri_handle *h, int cls, const GemmArgs &g) {
  SPAN(cls, 2.0 * g.M * (double)g.N * g.K * g.batch * 1e-9);
  return gemm(h, g);
}

cudaError_t oz_product(rssri_handle *h, int cls, const OzView &va, int batch, int M,
                       const OzView *vb, int N, long long K, double *C, long long ldc,
                       long long sC, int *err);
OzView oz_rows(const double *x, long long ld, long long K, long long len);
cudaError_t df_gemm_w(rssri_handle *h, const DfGemm &g);
OzView oz_cols(const double *x, long long ld, long long K, long long len);

// ------------------------------------------------------------ S1: V^-1/2 --
// Coupled Newton-Schulz iteration for the inverse square root: with
// Y_0 = V / c, Z_0 = I and T_k = (3 I - Z_k Y_k) / 2, Y_{k+1} = Y_k T_k and
// Z_{k+1} = T_k Z_k converge to (V/c)^{1/2} and (V/c)^{-1/2} whenever the
// spectrum of V/c lies in (0, 1] (c = max row sum of |V| guarantees this for
// an SPD V).  Stops one step after max |Z Y - I| < 1e-8; a non-SPD metric
// never converges and is reported as NOT_SPD.
int metric_inv_sqrt(rssri_handle *h, int *rc, bool df64) {
  cudaStream_t s = h->stream;
  const int na = h->n_aux;
  const size_t bytes = (size_t)na * na * sizeof(double);
  cudaError_t e;
#define RS_CK(x)                     \
  do {                               \
    e = (x);                         \
    if (e != cudaSuccess) { note_error_site(__FILE__, __LINE__); return map_err(e); } \
  } while (0)
  RS_CK(ensure(h->W, bytes));
  RS_CK(ensure(h->nsY, bytes));
  RS_CK(ensure(h->nsZ, bytes));
  RS_CK(ensure(h->nsP, bytes));
  RS_CK(ensure(h->nsT, bytes));
  RS_CK(ensure(h->nsY2, bytes));
  RS_CK(ensure(h->nsZ2, bytes));
  double *Y = h->nsY.as<double>(), *Z = h->nsZ.as<double>(), *Y2 = h->nsY2.as<double>(),
         *Z2 = h->nsZ2.as<double>(), *Pm = h->nsP.as<double>(), *Tm = h->nsT.as<double>();
  double *scal = h->scal.as<double>(), *part = h->part.as<double>();
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(ns_init(h->metric, na, Y, Z, scal, part, s)); }
  if (df64) {
    RS_CK(ensure(h->nsA2, (size_t)na * na * sizeof(float2)));
    RS_CK(ensure(h->nsB2, (size_t)na * na * sizeof(float2)));
  }
  // C = A B (na x na), in fp64 or in double-float on split copies (the
  // coupled iteration keeps the errors of its products as a perturbation of
  // the metric it implies, so it runs in fp64-accurate arithmetic throughout)
  auto mm = [&](const double *A, const double *B, double *C) -> cudaError_t {
    if (!df64) {
      GemmArgs g;
      g.M = g.N = g.K = na;
      g.lda = g.ldb = g.ldc = na;
      g.A = A; g.B = B; g.C = C;
      return gemm_p(h, RSSRI_PROF_SETUP_GEMM, g);
    }
    {
      SPAN(RSSRI_PROF_OTHER, 0.0);
      RS_TRY(to_df64(A, (long long)na * na, h->nsA2.as<float2>(), s, range_flag(h)));
      RS_TRY(to_df64(B, (long long)na * na, h->nsB2.as<float2>(), s, range_flag(h)));
    }
    SPAN(RSSRI_PROF_SETUP_GEMM, 2.0 * na * (double)na * na * 1e-9);
    DfGemm g;
    g.M = g.N = g.K = na;
    g.A = h->nsA2.as<float2>(); g.lda = na;
    g.B = h->nsB2.as<float2>(); g.ldb = na;
    g.C64 = C; g.ldc = na;
    return df_gemm_w(h, g);
  };
  const int max_it = 100;
  double resid = 0;
  bool final_step = false;
  int it = 0;
  for (; it < max_it; ++it) {
    RS_CK(mm(Z, Y, Pm));
    { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(ns_tbuild(Pm, na, Tm, scal, part, s)); }
    RS_CK(fetch(&resid, scal + 1, s));
    if (!std::isfinite(resid) || resid > 1e6) break;
    if (final_step) break;
    if (resid < 1e-8) final_step = true;
    RS_CK(mm(Y, Tm, Y2));
    RS_CK(mm(Tm, Z, Z2));
    std::swap(Y, Y2);
    std::swap(Z, Z2);
  }
  h->ns_iters = it;
  h->ns_resid = resid;
  if (!final_step || !std::isfinite(resid) || resid > 1e-6) {
    *rc = RSSRI_ERR_NOT_SPD;
    return RSSRI_OK;
  }
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(ns_finish(Z, na, scal, h->W.as<double>(), s)); }
  *rc = RSSRI_OK;
  return RSSRI_OK;
#undef RS_CK
}


// S6 and S7 for every tau (defined below).
int build_block(rssri_handle *h, int dd_arith, const double *g_in, const double *gb_in);

}  // namespace

// ====================================================================== ABI

extern "C" {

const char *rssri_last_cuda_error(void) { return g_last_cuda; }

const char *rssri_status_string(int code) {
  switch (code) {
    case RSSRI_OK: return "ok";
    case RSSRI_ERR_INVALID_ARG: return "invalid argument";
    case RSSRI_ERR_NOT_SPD: return "metric is not symmetric positive definite";
    case RSSRI_ERR_NONSYMMETRIC_ERI: return "3-index integrals are not symmetric in (i,j)";
    case RSSRI_ERR_OOM: return "device memory allocation failed";
    case RSSRI_ERR_CUDA: return "CUDA runtime error";
    case RSSRI_ERR_TIMEOUT: return "bounded device wait expired";
    case RSSRI_ERR_NOT_READY: return "rssri_setup has not completed on this handle";
    case RSSRI_ERR_NONFINITE: return "non-finite input or result";
    case RSSRI_ERR_RANGE: return "a double-float operand lies outside the pairs' exponent range";
    default: return "unknown status";
  }
}

int rssri_create(rssri_handle **out, int device, void *stream) {
  if (!out) return RSSRI_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return RSSRI_ERR_CUDA;
  if (device < 0 || device >= ndev) return RSSRI_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return RSSRI_ERR_CUDA;
  rssri_handle *h = new (std::nothrow) rssri_handle();
  if (!h) return RSSRI_ERR_OOM;
  h->device = device;
  h->stream = static_cast<cudaStream_t>(stream);
  for (auto &e : h->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      rssri_destroy(h);
      return RSSRI_ERR_CUDA;
    }
  cudaError_t e = ensure(h->scal, 64 * sizeof(double));
  if (e == cudaSuccess) e = ensure(h->part, 8192 * sizeof(double));
  if (e == cudaSuccess) e = ensure(h->flags, 16 * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&h->host_res, 8 * sizeof(double));
  if (e != cudaSuccess) {
    rssri_destroy(h);
    if (e != cudaSuccess) note_error_site(__FILE__, __LINE__);
    return map_err(e);
  }
  *out = h;
  return RSSRI_OK;
}

void rssri_destroy(rssri_handle *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  DevBuf *bufs[] = {&h->in_eri3, &h->in_metric, &h->in_orb_e, &h->in_orb_c, &h->in_tau,
                    &h->in_tau_w, &h->W, &h->nsY, &h->nsZ, &h->nsP, &h->nsT, &h->nsY2, &h->nsZ2,
                    &h->scal, &h->part, &h->flags, &h->colmax, &h->cnt, &h->cscratch, &h->cnum,
                    &h->csum, &h->spairs, &h->EL, &h->KLs, &h->cnt2, &h->lidx, &h->pij, &h->prow,
                    &h->pcol, &h->rowptr, &h->KP, &h->D, &h->theta, &h->Ut, &h->fac, &h->RLp,
                    &h->G, &h->Gb, &h->cs, &h->XG, &h->Cc, &h->Bm, &h->BC, &h->tarr, &h->sarr,
                    &h->e_st, &h->sig_raw, &h->sdd, &h->PG, &h->At, &h->T, &h->AP, &h->Gam, &h->L,
                    &h->trdd, &h->tr, &h->res, &h->sig_out, &h->e_pair, &h->gwork, &h->outbuf,
                    &h->hxsl, &h->hy3, &h->hg, &h->hgb, &h->hP, &h->hdc32, &h->hcl32,
                    &h->hdcl16, &h->hxy32, &h->ha6, &h->hct, &h->hdct, &h->hpart, &h->hfold, &h->hclt, &h->hfl, &h->Dhl,
                    &h->Ahl, &h->KPhl, &h->PGhl, &h->APhl, &h->Gamhl, &h->GGhl, &h->litMP, &h->litT, &h->litMhl, &h->eri_hl, &h->ut_hl, &h->nsA2, &h->nsB2, &h->elHl, &h->facHl, &h->xgHl, &h->cHl, &h->bHl, &h->cv_params, &h->cv_m, &h->cv_v, &h->cv_grad, &h->cv_ptmp,
                    &h->cv_act, &h->cv_work, &h->cv_X, &h->cv_t, &h->cv_w, &h->cv_stats, &h->cv_c,
                    &h->cv_scr, &h->cv_bx, &h->cv_bt, &h->cv_bw, &h->cv_loss, &h->sdd0, &h->oz_gs, &h->oz_gexp};
  for (DevBuf *b : bufs) release(*b);
  release(h->oz_pidx);
  release(h->oz_tmp);
  release(h->oz_gr);
  for (rssri_handle::OzBuf *o : {&h->ozX, &h->ozKP, &h->ozKPt, &h->ozGb, &h->ozBig0, &h->ozBig1,
                                 &h->ozAtP, &h->ozGam, &h->ozPA, &h->ozPB, &h->ozKPr,
                                 &h->ozGr}) {
    release(o->d);
    release(o->e);
  }
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto e : h->evpool) cudaEventDestroy(e);
  if (h->chain_graph) cudaGraphExecDestroy(h->chain_graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->host_res) cudaFreeHost(h->host_res);
  delete h;
}

int rssri_setup(rssri_handle *h, const rssri_problem *p, const rssri_options *o) {
  if (!h || h->pending) return RSSRI_ERR_INVALID_ARG;
  if (h->broken) return RSSRI_ERR_CUDA;
  int rc = validate_problem(p);
  if (rc) return rc;
  rc = validate_options(o, false);
  if (rc) return rc;
  if (cudaSetDevice(h->device) != cudaSuccess) return RSSRI_ERR_CUDA;
  AllocFailScope alloc_test(o->test_fail_alloc);
  h->test_wait_polls = o->test_wait_polls;
  cudaStream_t s = h->stream;
  h->ready = false;
  h->have_sigma = false;
  h->d_df64_ready = false;
  h->kp_hl_ready = false;
  h->cv_c_ready = false;
  h->block_ok = false;
  h->gg_valid = false;
  h->oz_ready = false;
  const int n = p->n, na = p->n_aux, nt = p->n_tau;
  const long long nn = (long long)n * n;
  cudaError_t e;
#define RS_CK(x)                                       \
  do {                                                 \
    e = (x);                                           \
    if (e != cudaSuccess) {                            \
      note_error_site(__FILE__, __LINE__);             \
      int _r = map_err(e);                             \
      if (_r == RSSRI_ERR_CUDA) h->broken = true;      \
      return _r;                                       \
    }                                                  \
  } while (0)

  // tau grid checks need host copies of the nodes
  std::vector<double> htau(nt), htw(nt);
  if (p->ptr_kind == RSSRI_PTR_HOST) {
    std::memcpy(htau.data(), p->tau, nt * sizeof(double));
    std::memcpy(htw.data(), p->tau_w, nt * sizeof(double));
  } else {
    RS_CK(cudaMemcpyAsync(htau.data(), p->tau, nt * sizeof(double), cudaMemcpyDeviceToHost, s));
    RS_CK(cudaMemcpyAsync(htw.data(), p->tau_w, nt * sizeof(double), cudaMemcpyDeviceToHost, s));
    RS_CK(cudaStreamSynchronize(s));
  }
  for (int k = 0; k < nt; ++k)
    if (!(htau[k] > 0.0 && htau[k] < p->beta) || !std::isfinite(htw[k]))
      return RSSRI_ERR_INVALID_ARG;

  h->recs.clear();
  h->ev_used = 0;
  h->prof_on = o->profile != 0;
  RS_CK(cudaEventRecord(h->ev[0], s));
  h->n = n; h->n_occ = p->n_occ; h->n_aux = na; h->n_tau = nt;
  h->mu = p->mu; h->beta = p->beta; h->ptr_kind = p->ptr_kind;
  h->eps_prime = o->eps_prime; h->eps = o->eps;
  h->h_tau_w = htw;
  RS_CK(stage(h->in_eri3, p->eri3, (size_t)nn * na, p->ptr_kind, s, &h->eri3));
  RS_CK(stage(h->in_metric, p->metric, (size_t)na * na, p->ptr_kind, s, &h->metric));
  RS_CK(stage(h->in_orb_e, p->orb_e, n, p->ptr_kind, s, &h->orb_e));
  RS_CK(stage(h->in_orb_c, p->orb_c, (size_t)nn, p->ptr_kind, s, &h->orb_c));
  RS_CK(stage(h->in_tau, p->tau, nt, p->ptr_kind, s, &h->tau));
  RS_CK(stage(h->in_tau_w, p->tau_w, nt, p->ptr_kind, s, &h->tau_w));

  // input checks: symmetry of (ij|A), finiteness of everything
  int *flags = h->flags.as<int>();
  RS_CK(cudaMemsetAsync(flags, 0, 16 * sizeof(int), s));
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(eri_check(h->eri3, n, na, flags, s)); }
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(nonfinite_check(h->metric, (long long)na * na, flags + 1, s)); }
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(nonfinite_check(h->orb_e, n, flags + 1, s)); }
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(nonfinite_check(h->orb_c, nn, flags + 1, s)); }
  int hflags[2];
  RS_CK(fetch(hflags, flags, s, 2));
  if (hflags[1]) return RSSRI_ERR_NONFINITE;
  if (hflags[0]) return RSSRI_ERR_NONSYMMETRIC_ERI;

  // scratch: split-K partials of the products, per-block partial maxima / row sums
  RS_CK(ensure(h->gwork, (size_t)16 << 20));
  RS_CK(ensure(h->part, (size_t)std::max(8192, na) * sizeof(double)));

  // S1
  int ns_rc = RSSRI_OK;
  rc = metric_inv_sqrt(h, &ns_rc, o->dd_arith != RSSRI_DD_FP64);
  if (rc) { if (rc == RSSRI_ERR_CUDA) h->broken = true; return rc; }
  if (ns_rc) return ns_rc;

  // S2: screen (Eq. 11) and compact the kept pairs
  RS_CK(ensure(h->colmax, n * sizeof(double)));
  RS_CK(ensure(h->cnt, nn * sizeof(int)));
  RS_CK(ensure(h->cscratch, compact_scratch_bytes((int)nn)));
  RS_CK(ensure(h->cnum, 4 * sizeof(int)));
  RS_CK(ensure(h->csum, 4 * sizeof(long long)));
  RS_CK(ensure(h->spairs, nn * sizeof(int)));
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(eri_colmax(h->eri3, n, na, h->colmax.as<double>(), s)); }
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(eri_pair_count(h->eri3, n, na, h->colmax.as<double>(), o->eps_prime, h->cnt.as<int>(), s)); }
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(compact(h->cnt.as<int>(), (int)nn, h->spairs.as<int>(), h->cnum.as<int>(),
                h->csum.as<long long>(), h->cscratch.p, s)); }
  int P_s = 0;
  long long nnz = 0;
  RS_CK(fetch(&P_s, h->cnum.p, s));
  RS_CK(fetch(&nnz, h->csum.p, s));
  h->P_s = P_s;
  h->nnz_eri_l = nnz;

  // S3: K^L rows of the screened pairs (Eq. 12), global max and cut (Eq. 13)
  RS_CK(ensure(h->EL, (size_t)std::max(P_s, 1) * na * sizeof(double)));
  RS_CK(ensure(h->KLs, (size_t)std::max(P_s, 1) * na * sizeof(double)));
  RS_CK(ensure(h->cnt2, (size_t)std::max(P_s, 1) * sizeof(int)));
  RS_CK(ensure(h->lidx, (size_t)std::max(P_s, 1) * sizeof(int)));
  int P = 0;
  long long nnzk = 0;
  double kmax = 0;
  if (P_s > 0) {
    { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(eri_gather_rows(h->eri3, n, na, h->colmax.as<double>(), o->eps_prime,
                          h->spairs.as<int>(), P_s, h->EL.as<double>(), s)); }
    // in IEEE fp64, or in double-float (~1e-14) under the double-float and
    // sliced blocks: the cut of Eq. 13 compares these values
    if (o->dd_arith != RSSRI_DD_FP64) {
      RS_CK(ensure(h->elHl, (size_t)P_s * na * sizeof(float2)));
      RS_CK(ensure(h->nsB2, (size_t)na * na * sizeof(float2)));
      { SPAN(RSSRI_PROF_OTHER, 0.0);
        RS_CK(to_df64(h->EL.as<double>(), (long long)P_s * na, h->elHl.as<float2>(), s, range_flag(h)));
        RS_CK(to_df64(h->W.as<double>(), (long long)na * na, h->nsB2.as<float2>(), s, range_flag(h))); }
      SPAN(RSSRI_PROF_SETUP_GEMM, 2.0 * P_s * (double)na * na * 1e-9);
      DfGemm g;
      g.M = P_s; g.N = na; g.K = na;
      g.A = h->elHl.as<float2>(); g.lda = na;
      g.B = h->nsB2.as<float2>(); g.ldb = na;
      g.C64 = h->KLs.as<double>(); g.ldc = na;
      RS_CK(df_gemm_w(h, g));
    } else {
      GemmArgs g;
      g.M = P_s; g.N = na; g.K = na;
      g.A = h->EL.as<double>(); g.lda = na;
      g.B = h->W.as<double>(); g.ldb = na;
      g.C = h->KLs.as<double>(); g.ldc = na;
      RS_CK(gemm_p(h, RSSRI_PROF_SETUP_GEMM, g));
    }
    double *scal = h->scal.as<double>();
    { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(absmax(h->KLs.as<double>(), (long long)P_s * na, scal + 2, h->part.as<double>(), s)); }
    { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(kl_cut(h->KLs.as<double>(), P_s, na, scal + 2, o->eps, h->cnt2.as<int>(), s)); }
    { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(compact(h->cnt2.as<int>(), P_s, h->lidx.as<int>(), h->cnum.as<int>(),
                  h->csum.as<long long>(), h->cscratch.p, s)); }
    RS_CK(fetch(&P, h->cnum.p, s));
    RS_CK(fetch(&nnzk, h->csum.p, s));
    RS_CK(fetch(&kmax, scal + 2, s));
  }
  h->P = P;
  h->nnz_k_l = nnzk;
  h->k_l_max = kmax;
  RS_CK(ensure(h->pij, (size_t)std::max(P, 1) * sizeof(int)));
  RS_CK(ensure(h->prow, (size_t)std::max(P, 1) * sizeof(int)));
  RS_CK(ensure(h->pcol, (size_t)std::max(P, 1) * sizeof(int)));
  RS_CK(ensure(h->rowptr, (size_t)(n + 1) * sizeof(int)));
  RS_CK(ensure(h->KP, (size_t)std::max(P, 1) * na * sizeof(double)));
  RS_CK(ensure(h->D, (size_t)std::max(P, 1) * std::max(P, 1) * sizeof(double)));
  if (P > 0) {
    { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(gather_int(h->spairs.as<int>(), h->lidx.as<int>(), P, h->pij.as<int>(), s)); }
    { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(gather_rows(h->KLs.as<double>(), h->lidx.as<int>(), P, na, h->KP.as<double>(), s)); }
    // D[a][b] = sum_Q K_P[a][Q] K_P[b][Q] = v^L for the pair of pairs (Eq. 8 on [K]^L),
    // in the arithmetic the deterministic block is asked to use
    if (o->dd_arith == RSSRI_DD_OZ) {
      RS_CK(oz_product(h, RSSRI_PROF_SETUP_GEMM,
                       oz_rows(h->KP.as<double>(), na, na, (long long)P * na), 1, P, nullptr, P,
                       na, h->D.as<double>(), P, 0, h->flags.as<int>() + 5));
      // K_P as pairs for the block's one double-float product (K^Q G)
      RS_CK(ensure(h->KPhl, (size_t)P * na * sizeof(float2)));
      { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(to_df64(h->KP.as<double>(), (long long)P * na, h->KPhl.as<float2>(), s, range_flag(h))); }
      h->kp_hl_ready = true;
    } else if (o->dd_arith != RSSRI_DD_FP64) {
      RS_CK(ensure(h->Dhl, (size_t)P * P * sizeof(float2)));
      RS_CK(ensure(h->KPhl, (size_t)P * na * sizeof(float2)));
      { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(to_df64(h->KP.as<double>(), (long long)P * na, h->KPhl.as<float2>(), s, range_flag(h))); }
      {
        SPAN(RSSRI_PROF_SETUP_GEMM, 2.0 * P * (double)P * na * 1e-9);
        DfGemm g;
        g.M = P; g.N = P; g.K = na;
        g.A = h->KPhl.as<float2>(); g.lda = na;
        g.B = h->KPhl.as<float2>(); g.ldb = na; g.transB = 1;
        g.C64 = h->D.as<double>(); g.ldc = P;
        RS_CK(df_gemm_w(h, g));
      }
      { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(to_df64(h->D.as<double>(), (long long)P * P, h->Dhl.as<float2>(), s, range_flag(h))); }
      h->d_df64_ready = true;
      h->kp_hl_ready = true;
    } else {
      GemmArgs g;
      g.M = P; g.N = P; g.K = na;
      g.A = h->KP.as<double>(); g.lda = na;
      g.B = h->KP.as<double>(); g.ldb = na; g.transB = 1;
      g.C = h->D.as<double>(); g.ldc = P;
      RS_CK(gemm_p(h, RSSRI_PROF_SETUP_GEMM, g));
    }
  }
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(pair_csr(h->pij.as<int>(), P, n, h->rowptr.as<int>(), h->prow.as<int>(),
                 h->pcol.as<int>(), s)); }
  // S6, S7: G(tau), G(beta - tau) and the deterministic block for every tau,
  // cached for every sampling call on this setup (they do not depend on the draws)
  h->setup_arith = o->dd_arith;
  rc = build_block(h, o->dd_arith, nullptr, nullptr);
  if (rc) { if (rc == RSSRI_ERR_CUDA) h->broken = true; return rc; }
  RS_CK(cudaEventRecord(h->ev[1], s));
  RS_CK(cudaEventSynchronize(h->ev[1]));
  {
    int range = 0;
    RS_CK(fetch(&range, range_flag(h), s));
    if (range) return RSSRI_ERR_RANGE;
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
  h->t_setup_ms = ms;
  collect(h, h->setup_launches, h->setup_ms, h->setup_gflop, h->setup_tgflop);
  h->ready = true;
  return RSSRI_OK;
#undef RS_CK
}

}  // extern "C"

namespace {

// S6 for all tau: G(tau) = -C_v e^{-(e_v-mu)tau} C_v^T, Gb(tau) = -C_o e^{(e_o-mu)tau} C_o^T.
cudaError_t build_green(rssri_handle *h) {
  cudaStream_t s = h->stream;
  const int n = h->n, no = h->n_occ, nv = n - no, nt = h->n_tau;
  const long long nn = (long long)n * n;
  RS_TRY(ensure(h->cs, (size_t)nt * n * std::max(no, nv) * sizeof(double)));
  for (int occ = 0; occ < 2; ++occ) {
    const int off = occ ? 0 : no, m = occ ? no : nv;
    double *out = occ ? h->Gb.as<double>() : h->G.as<double>();
    { SPAN(RSSRI_PROF_GREEN, 0.0); RS_TRY(green_scale(h->orb_c, h->orb_e, n, off, m, h->mu, h->tau, nt, occ ? 1 : -1,
                       h->cs.as<double>(), s)); }
    GemmArgs g;
    g.M = n; g.N = n; g.K = m; g.batch = nt;
    g.A = h->cs.as<double>(); g.lda = m; g.sA = (long long)n * m;
    g.B = h->orb_c + off; g.ldb = n; g.transB = 1; g.sB = 0;
    g.C = out; g.ldc = n; g.sC = nn;
    g.alpha = -1.0;
    RS_TRY(gemm_p(h, RSSRI_PROF_GREEN, g));
  }
  return cudaSuccess;
}

// S7 for one tau: the deterministic block, Eq. 20 on v^L = sum_Q K^Q K^Q with
// K = [K]^L.  With PG^Q = K^Q G, At^Q = Gb K^Q G, Gamma_QQ' = Tr(K^Q G K^Q' Gb),
// L^Q = sum_Q' Gamma_QQ' K^Q' and T^Q = sum_Q' K^Q' At^Q K^Q' (built in pair
// space from D = v^L):  Sigma_DD = sum_Q K^Q G (2 L^Q - T^Q).
cudaError_t sigma_dd_tau(rssri_handle *h, const double *G, const double *Gb, double *out) {
  cudaStream_t s = h->stream;
  const int n = h->n, na = h->n_aux, P = h->P;
  const long long nn = (long long)n * n;
  if (P == 0) return cudaMemsetAsync(out, 0, nn * sizeof(double), s);
  double *PG = h->PG.as<double>(), *At = h->At.as<double>(), *T = h->T.as<double>();
  // PG[i][m][Q] = sum_{k in row i} K_P[(i,k)][Q] G[k][m]
  { SPAN(RSSRI_PROF_DD_GEMM, 2.0 * n * (double)na * P * 1e-9); RS_TRY(dgemm_segmented(n, n, na, h->rowptr.as<int>(), h->pcol.as<int>(), G, n,
                         h->KP.as<double>(), na, PG, na, (long long)n * na, s)); }
  // At[k][(l,Q)] = sum_m Gb[k][m] PG[m][(l,Q)]
  {
    GemmArgs g;
    g.M = n; g.N = n * na; g.K = n;
    g.A = Gb; g.lda = n;
    g.B = PG; g.ldb = (long long)n * na;
    g.C = At; g.ldc = (long long)n * na;
    RS_TRY(gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  // T[m][Q][j] = sum_{a in row m, b in row j} D[a][b] At[(col a, col b)][Q]
  { SPAN(RSSRI_PROF_DD_SPMM, 2.0 * na * (double)P * P * 1e-9); RS_TRY(dd_exchange_spmm(h->rowptr.as<int>(), h->pcol.as<int>(), h->D.as<double>(), P, At, n, na,
                          T, s)); }
  // Gamma = K_P^T At_P, At_P the rows of At at the kept pairs
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_TRY(gather_rows(At, h->pij.as<int>(), P, na, h->AP.as<double>(), s)); }
  {
    GemmArgs g;
    g.M = na; g.N = na; g.K = P;
    g.A = h->KP.as<double>(); g.lda = na; g.transA = 1;
    g.B = h->AP.as<double>(); g.ldb = na;
    g.C = h->Gam.as<double>(); g.ldc = na;
    RS_TRY(gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  // L[a][Q] = sum_Q' K_P[a][Q'] Gamma[Q][Q']
  {
    GemmArgs g;
    g.M = P; g.N = na; g.K = na;
    g.A = h->KP.as<double>(); g.lda = na;
    g.B = h->Gam.as<double>(); g.ldb = na; g.transB = 1;
    g.C = h->L.as<double>(); g.ldc = na;
    RS_TRY(gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_TRY(dd_fold_direct(h->prow.as<int>(), h->pcol.as<int>(), h->L.as<double>(), P, n, na, T, s)); }
  // Sigma_DD = -PG_view [n x (n na)] * T_view [(n na) x n]
  {
    GemmArgs g;
    g.M = n; g.N = n; g.K = n * na;
    g.A = PG; g.lda = (long long)n * na;
    g.B = T; g.ldb = n;
    g.C = out; g.ldc = n;
    g.alpha = -1.0;
    RS_TRY(gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  return cudaSuccess;
}

// A double-float product with the handle's split-over-K scratch (no span).
cudaError_t df_gemm_w(rssri_handle *h, const DfGemm &g) {
  const size_t need = df_gemm_work(g) * sizeof(double);
  if (need > h->gwork.bytes) RS_TRY(ensure(h->gwork, need));
  return df_gemm(g, h->gwork.as<double>(), h->gwork.bytes / sizeof(double), h->stream);
}

// A double-float product counted under kernel class `cls`.
cudaError_t df_gemm_c(rssri_handle *h, int cls, const DfGemm &g) {
  SPAN(cls, df_gemm_flops(g) * 1e-9);
  const size_t need = df_gemm_work(g) * sizeof(double);
  if (need > h->gwork.bytes) RS_TRY(ensure(h->gwork, need));
  return df_gemm(g, h->gwork.as<double>(), h->gwork.bytes / sizeof(double), h->stream);
}

// A double-float product counted under the deterministic-block GEMM class.
cudaError_t df_gemm_p(rssri_handle *h, const DfGemm &g) {
  SPAN(RSSRI_PROF_DD_GEMM, df_gemm_flops(g) * 1e-9);
  const size_t need = df_gemm_work(g) * sizeof(double);
  if (need > h->gwork.bytes) RS_TRY(ensure(h->gwork, need));
  return df_gemm(g, h->gwork.as<double>(), h->gwork.bytes / sizeof(double), h->stream);
}

// The same block in double-float arithmetic (fp32 pairs, fp64 totals every 256
// terms).  Operands are split into (hi, lo) pairs once: D and K_P at setup, G
// and Gb for all tau before the loop (Ghl, Gbhl), PG and At by the products
// that form them, Gamma and T after their fp64 reductions.
cudaError_t sigma_dd_tau_df64(rssri_handle *h, const float2 *Ghl, const float2 *Gbhl,
                              double *out) {
  cudaStream_t s = h->stream;
  const int n = h->n, na = h->n_aux, P = h->P;
  const long long nn = (long long)n * n;
  if (P == 0) return cudaMemsetAsync(out, 0, nn * sizeof(double), s);
  float2 *PGhl = h->PGhl.as<float2>(), *Ahl = h->Ahl.as<float2>();
  const float2 *KPhl = h->KPhl.as<float2>();
  double *T = h->T.as<double>();
  // PG[i][m][Q] = sum_{k in row i} K_P[(i,k)][Q] G[k][m]
  { SPAN(RSSRI_PROF_DD_GEMM, 2.0 * n * (double)na * P * 1e-9);
    RS_TRY(df_gemm_segmented(n, n, na, h->rowptr.as<int>(), h->pcol.as<int>(), Ghl, n, KPhl, na,
                             PGhl, na, (long long)n * na, s)); }
  // At[k][(l,Q)] = sum_m Gb[k][m] PG[m][(l,Q)], written as pairs
  {
    DfGemm g;
    g.M = n; g.N = n * na; g.K = n;
    g.A = Gbhl; g.lda = n;
    g.B = PGhl; g.ldb = (long long)n * na;
    g.C2 = Ahl; g.ldc = (long long)n * na;
    RS_TRY(df_gemm_p(h, g));
  }
  // T[m][Q][j] = sum_{a in row m, b in row j} D[a][b] At[(col a, col b)][Q]
  { SPAN(RSSRI_PROF_DD_SPMM, 2.0 * na * (double)P * P * 1e-9);
    RS_TRY(dd_exchange_spmm_df64(h->rowptr.as<int>(), h->pcol.as<int>(), h->Dhl.as<float2>(), P,
                                 Ahl, n, na, T, s)); }
  // Gamma = K_P^T At_P, At_P the rows of At at the kept pairs
  { SPAN(RSSRI_PROF_OTHER, 0.0);
    RS_TRY(gather_rows_f2(Ahl, h->pij.as<int>(), P, na, h->APhl.as<float2>(), s)); }
  {
    DfGemm g;
    g.M = na; g.N = na; g.K = P;
    g.A = KPhl; g.lda = na; g.transA = 1;
    g.B = h->APhl.as<float2>(); g.ldb = na;
    g.C64 = h->Gam.as<double>(); g.ldc = na;
    RS_TRY(df_gemm_p(h, g));
  }
  { SPAN(RSSRI_PROF_OTHER, 0.0);
    RS_TRY(to_df64(h->Gam.as<double>(), (long long)na * na, h->Gamhl.as<float2>(), s)); }
  // L[a][Q] = sum_Q' K_P[a][Q'] Gamma[Q][Q']
  {
    DfGemm g;
    g.M = P; g.N = na; g.K = na;
    g.A = KPhl; g.lda = na;
    g.B = h->Gamhl.as<float2>(); g.ldb = na; g.transB = 1;
    g.C64 = h->L.as<double>(); g.ldc = na;
    RS_TRY(df_gemm_p(h, g));
  }
  { SPAN(RSSRI_PROF_OTHER, 0.0);
    RS_TRY(dd_fold_direct(h->prow.as<int>(), h->pcol.as<int>(), h->L.as<double>(), P, n, na, T, s));
    // At is no longer needed: its pair buffer takes T
    RS_TRY(to_df64(T, nn * na, Ahl, s)); }
  // Sigma_DD = -PG_view [n x (n na)] * T_view [(n na) x n], symmetric (G, Gb
  // and every K^Q are): the tiles below the diagonal are mirrored
  {
    DfGemm g;
    g.M = n; g.N = n; g.K = n * na;
    g.A = PGhl; g.lda = (long long)n * na;
    g.B = Ahl; g.ldb = n;
    g.C64 = out; g.ldc = n;
    g.alpha = -1.0;
    g.sym = 1;
    RS_TRY(df_gemm_p(h, g));
  }
  return cudaSuccess;
}

// ------------------------------------------- the sliced (RSSRI_DD_OZ) block --
// A digit buffer for batch x rows x K values (rows padded to ld = K rounded up to 16).
cudaError_t oz_make(rssri_handle::OzBuf &b, int batch, int rows, long long K) {
  OzDigits v;
  v.batch = batch;
  v.rows = rows;
  v.K = K;
  v.ld = (K + 15) / 16 * 16;
  RS_TRY(ensure(b.d, oz_digit_elems(v) * sizeof(__nv_bfloat16)));
  RS_TRY(ensure(b.e, (size_t)batch * rows * sizeof(int)));
  v.d = b.d.as<__nv_bfloat16>();
  v.ef = b.e.as<int>();
  b.v = v;
  return cudaSuccess;
}

cudaError_t oz_slice_p(rssri_handle *h, const OzView &v, const OzDigits &o) {
  SPAN(RSSRI_PROF_SLICE, 0.0);
  return oz_slice(v, o, h->stream);
}

// An fp64-accurate product on the tensor cores, counted under `cls`.
cudaError_t oz_gemm_p(rssri_handle *h, int cls, const OzGemm &g_in) {
  OzGemm g = g_in;
  g.wait_polls = h->test_wait_polls;
  const double alg = 2.0 * g.M * (double)g.N * g.A.K * g.batch;
  SPAN_T(cls, alg * 1e-9, oz_gemm_flops(g) * 1e-9);
  const size_t need = oz_gemm_work(g) * sizeof(double);
  if (need > h->gwork.bytes) RS_TRY(ensure(h->gwork, need));
  return oz_gemm(g, h->gwork.as<double>(), h->gwork.bytes / sizeof(double), h->stream);
}

// C[b sC + i ldc + j] = sum_k A_b(i, k) B(j, k), fp64-accurate on the tensor
// cores (digit slicing), for slicer views A (batch x M x K) and B (N x K,
// shared by the batch; null: B is A with batch 1).  The digit buffers grow
// as needed.  err: device flag of the bounded waits.
cudaError_t oz_product(rssri_handle *h, int cls, const OzView &va, int batch, int M,
                       const OzView *vb, int N, long long K, double *C, long long ldc,
                       long long sC, int *err) {
  RS_TRY(oz_make(h->ozPA, batch, M, K));
  RS_TRY(oz_slice_p(h, va, h->ozPA.v));
  OzGemm g;
  g.A = h->ozPA.v;
  if (vb) {
    RS_TRY(oz_make(h->ozPB, 1, N, K));
    RS_TRY(oz_slice_p(h, *vb, h->ozPB.v));
    g.B = h->ozPB.v;
  } else {
    g.B = h->ozPA.v;
  }
  g.M = M; g.N = N; g.batch = batch;
  g.C = C; g.ldc = ldc; g.sC = sC;
  g.ccap = (long long)(batch - 1) * sC + (long long)(M - 1) * ldc + N;
  g.err = err;
  return oz_gemm_p(h, cls, g);
}

// Slicer views of a row-major matrix (rows of K at stride ld) and of the
// transpose of one (element (j, k) = x[k ld + j]).
OzView oz_rows(const double *x, long long ld, long long K, long long len) {
  OzView v;
  v.x = x; v.rs = ld; v.cs2 = 1; v.k2pad = v.k2n = K; v.xlen = len;
  return v;
}
OzView oz_cols(const double *x, long long ld, long long K, long long len) {
  OzView v;
  v.x = x; v.rs = 1; v.cs2 = ld; v.k2pad = v.k2n = K; v.xlen = len;
  return v;
}

// Setup of the sliced block: the pair index map, the band half-width, the
// exchange contraction's left operand (from D) and the digits of K_P and K_P^T.
int oz_setup(rssri_handle *h) {
  cudaStream_t s = h->stream;
  const int n = h->n, na = h->n_aux, P = h->P;
  cudaError_t e;
#define RS_CK(x)                     \
  do {                               \
    e = (x);                         \
    if (e != cudaSuccess) { note_error_site(__FILE__, __LINE__); return map_err(e); } \
  } while (0)
  RS_CK(ensure(h->oz_pidx, (size_t)n * n * sizeof(int)));
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(oz_pair_index(h->pij.as<int>(), P, n, h->oz_pidx.as<int>(), s)); }
  // band half-width of the kept pairs
  std::vector<int> hp(P);
  RS_CK(fetch(hp.data(), h->pij.p, s, P));
  int bk = 0;
  for (int a = 0; a < P; ++a) bk = std::max(bk, std::abs(hp[a] / n - hp[a] % n));
  h->oz_geo = oz_exch_geometry(n, na, bk);
  const OzExch &x = h->oz_geo;
  const int tiles = x.mtiles * x.jtiles;
  if (tiles > 65535) return RSSRI_ERR_INVALID_ARG;
  RS_CK(ensure(h->oz_tmp, (size_t)tiles * 128 * x.kx * sizeof(double)));
  { SPAN(RSSRI_PROF_OTHER, 0.0);
    RS_CK(oz_exch_gather(x, h->D.as<double>(), P, h->oz_pidx.as<int>(), h->oz_tmp.as<double>(),
                         (long long)tiles * 128 * x.kx, s)); }
  RS_CK(oz_make(h->ozX, tiles, 128, x.kx));
  {
    OzView v;
    v.x = h->oz_tmp.as<double>();
    v.bs = 128 * x.kx; v.rs = x.kx; v.cs2 = 1; v.k2pad = v.k2n = x.kx;
    v.xlen = (long long)tiles * 128 * x.kx;
    RS_CK(oz_slice_p(h, v, h->ozX.v));
  }
  // K_P [P][na]: digits with rows a (for L) and rows Q (for Gamma)
  RS_CK(oz_make(h->ozKP, 1, P, na));
  RS_CK(oz_make(h->ozKPt, 1, na, P));
  {
    OzView v;
    v.x = h->KP.as<double>();
    v.rs = na; v.cs2 = 1; v.k2pad = v.k2n = na; v.xlen = (long long)P * na;
    RS_CK(oz_slice_p(h, v, h->ozKP.v));
    OzView t;
    t.x = h->KP.as<double>();
    t.rs = 1; t.cs2 = na; t.k2pad = t.k2n = P; t.xlen = (long long)P * na;
    RS_CK(oz_slice_p(h, t, h->ozKPt.v));
  }
  // K_P by rows i of the pair list, padded to W: the right operand of K^Q G
  {
    std::vector<int> rp(n + 1);
    RS_CK(fetch(rp.data(), h->rowptr.p, s, n + 1));
    int wmax = 1;
    for (int i = 0; i < n; ++i) wmax = std::max(wmax, rp[i + 1] - rp[i]);
    h->oz_w = (wmax + 15) / 16 * 16;
    const int W = h->oz_w;
    const long long len = (long long)n * na * W;
    RS_CK(ensure(h->oz_tmp, std::max(h->oz_tmp.bytes, (size_t)len * sizeof(double))));
    { SPAN(RSSRI_PROF_OTHER, 0.0);
      RS_CK(oz_rows_kp(h->KP.as<double>(), h->rowptr.as<int>(), n, na, W, h->oz_tmp.as<double>(), s)); }
    RS_CK(oz_make(h->ozKPr, n, na, W));
    OzView v;
    v.x = h->oz_tmp.as<double>();
    v.bs = (long long)na * W; v.rs = W; v.cs2 = 1; v.k2pad = v.k2n = W; v.xlen = len;
    RS_CK(oz_slice_p(h, v, h->ozKPr.v));
  }
  RS_CK(cudaStreamSynchronize(s));
  release(h->oz_tmp);
  h->oz_ready = true;
  return RSSRI_OK;
#undef RS_CK
}

// S7 for one tau with every dense product and the exchange contraction on
// the tensor cores (sliced fp64-accurate products), the segmented K^Q G in
// double-float.  With T stored negated by the contraction, U = 2 L - T and
// Sigma_DD = sum_Q PG^Q U^Q, PG^Q = K^Q G (see sigma_dd_tau).
cudaError_t sigma_dd_tau_oz(rssri_handle *h, const double *Gt, const double *Gb, double *out) {
  cudaStream_t s = h->stream;
  const int n = h->n, na = h->n_aux, P = h->P;
  const long long nn = (long long)n * n, nna = nn * na;
  if (P == 0) return cudaMemsetAsync(out, 0, nn * sizeof(double), s);
  const OzExch &x = h->oz_geo;
  int *err = h->flags.as<int>() + 5;
  double *PG = h->PG.as<double>();
  // T (the exchange's output) takes At's buffer once At's rows at the kept
  // pairs are gathered and At is sliced
  double *At = h->At.as<double>(), *T = At;
  // PG[i][m][Q] = sum_{k in row i} K_P[(i,k)][Q] G[k][m]: batched over the rows i of the
  // pair list, K = the row's pairs (padded to W), both operands sliced
  {
    const int W = h->oz_w;
    { SPAN(RSSRI_PROF_OTHER, 0.0);
      RS_TRY(oz_rows_g(Gt, h->rowptr.as<int>(), h->pcol.as<int>(), n, W, h->oz_gr.as<double>(), s)); }
    OzView v;
    v.x = h->oz_gr.as<double>();
    v.bs = (long long)n * W; v.rs = W; v.cs2 = 1; v.k2pad = v.k2n = W;
    v.xlen = (long long)n * n * W;
    RS_TRY(oz_slice_p(h, v, h->ozGr.v));
    OzGemm g;
    g.A = h->ozGr.v; g.B = h->ozKPr.v;
    g.M = n; g.N = na; g.batch = n;
    g.C = PG; g.ldc = na; g.sC = (long long)n * na; g.ccap = nna; g.err = err;
    RS_TRY(oz_gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  // At[k][(l,Q)] = sum_m Gb[k][m] PG[m][(l,Q)]
  OzDigits &dGb = h->ozGb.v;
  { OzView v; v.x = Gb; v.rs = n; v.cs2 = 1; v.k2pad = v.k2n = n; v.xlen = nn;
    RS_TRY(oz_slice_p(h, v, dGb)); }
  OzDigits dPGb = h->ozBig0.v;
  dPGb.rows = (int)(n * (long long)na); dPGb.K = n; dPGb.ld = (n + 15) / 16 * 16;
  { OzView v; v.x = PG; v.rs = 1; v.cs2 = (long long)n * na; v.k2pad = v.k2n = n;
    v.xlen = nna;
    RS_TRY(oz_slice_p(h, v, dPGb)); }
  {
    OzGemm g;
    g.A = dGb; g.B = dPGb; g.M = n; g.N = (int)(n * (long long)na);
    g.C = At; g.ldc = (long long)n * na; g.ccap = nna; g.err = err;
    RS_TRY(oz_gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  // the exchange contraction: T[j][m][Q] = -sum D[(m,k),(l,j)] At[k][l][Q]
  OzDigits dAt = h->ozBig1.v;
  dAt.rows = na; dAt.K = (long long)n * x.ldl; dAt.ld = dAt.K;
  { OzView v; v.x = At; v.rs = 1; v.cs1 = (long long)n * na; v.cs2 = na; v.k2pad = x.ldl;
    v.k2off = x.lsh;
    v.k2n = n; v.xlen = nna;
    RS_TRY(oz_slice_p(h, v, dAt)); }
  // At_P: the rows of At at the kept pairs (for Gamma below)
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_TRY(gather_rows(At, h->pij.as<int>(), P, na, h->AP.as<double>(), s)); }
  { SPAN_T(RSSRI_PROF_DD_SPMM, 2.0 * na * (double)P * P * 1e-9, oz_exch_flops(x) * 1e-9);
    RS_TRY(oz_exch(x, h->ozX.v, dAt, T, nna, -1.0, err, s, h->test_wait_polls)); }
  // Gamma = K_P^T At_P
  { OzView v; v.x = h->AP.as<double>(); v.rs = 1; v.cs2 = na; v.k2pad = v.k2n = P;
    v.xlen = (long long)P * na;
    RS_TRY(oz_slice_p(h, v, h->ozAtP.v)); }
  {
    OzGemm g;
    g.A = h->ozKPt.v; g.B = h->ozAtP.v; g.M = na; g.N = na;
    g.C = h->Gam.as<double>(); g.ldc = na; g.ccap = (long long)na * na; g.err = err;
    RS_TRY(oz_gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  // L[a][Q] = sum_Q' K_P[a][Q'] Gamma[Q][Q']
  { OzView v; v.x = h->Gam.as<double>(); v.rs = na; v.cs2 = 1; v.k2pad = v.k2n = na;
    v.xlen = (long long)na * na;
    RS_TRY(oz_slice_p(h, v, h->ozGam.v)); }
  {
    OzGemm g;
    g.A = h->ozKP.v; g.B = h->ozGam.v; g.M = P; g.N = na;
    g.C = h->L.as<double>(); g.ldc = na; g.ccap = (long long)P * na; g.err = err;
    RS_TRY(oz_gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  // U = 2 L - T at the kept pairs (T already negated)
  { SPAN(RSSRI_PROF_OTHER, 0.0);
    RS_TRY(oz_fold_direct(h->prow.as<int>(), h->pcol.as<int>(), h->L.as<double>(), P, n, na, T, s)); }
  // Sigma_DD[i][j] = sum_{(m,Q)} PG[i][m][Q] U[j][m][Q]
  OzDigits dU = h->ozBig0.v;
  const long long kmq = (long long)n * na;  // the contraction index (m, Q)
  dU.rows = n; dU.K = kmq; dU.ld = (kmq + 15) / 16 * 16;
  { OzView v; v.x = T; v.rs = (long long)n * na; v.cs2 = 1; v.k2pad = v.k2n = dU.K;
    v.xlen = nna;
    RS_TRY(oz_slice_p(h, v, dU)); }
  OzDigits dPGa = h->ozBig1.v;
  dPGa.rows = n; dPGa.K = kmq; dPGa.ld = (kmq + 15) / 16 * 16;
  { OzView v; v.x = PG; v.rs = (long long)n * na; v.cs2 = 1; v.k2pad = v.k2n = dPGa.K;
    v.xlen = nna;
    RS_TRY(oz_slice_p(h, v, dPGa)); }
  {
    OzGemm g;
    g.A = dPGa; g.B = dU; g.M = n; g.N = n;
    g.C = out; g.ldc = n; g.ccap = nn; g.err = err;
    RS_TRY(oz_gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  return cudaSuccess;
}

size_t dd_work_need(rssri_handle *h) {
  const int n = h->n, na = h->n_aux, P = std::max(h->P, 1);
  size_t w = 0;
  GemmArgs g;
  g.M = na; g.N = na; g.K = P; w = std::max(w, dgemm_work_elems(g));
  g.M = P; g.N = na; g.K = na; w = std::max(w, dgemm_work_elems(g));
  g.M = n; g.N = n; g.K = n * na; w = std::max(w, dgemm_work_elems(g));
  g.M = n; g.N = n * na; g.K = n; w = std::max(w, dgemm_work_elems(g));
  return w;
}

// The pair copies of D and K_P used by the double-float block (made once per setup).
cudaError_t ensure_d_df64(rssri_handle *h) {
  if (h->d_df64_ready || h->P == 0) return cudaSuccess;
  const int P = h->P, na = h->n_aux;
  RS_TRY(ensure(h->Dhl, (size_t)P * P * sizeof(float2)));
  RS_TRY(ensure(h->KPhl, (size_t)P * na * sizeof(float2)));
  SPAN(RSSRI_PROF_OTHER, 0.0);
  RS_TRY(to_df64(h->D.as<double>(), (long long)P * P, h->Dhl.as<float2>(), h->stream, range_flag(h)));
  RS_TRY(to_df64(h->KP.as<double>(), (long long)P * na, h->KPhl.as<float2>(), h->stream, range_flag(h)));
  h->d_df64_ready = true;
  h->kp_hl_ready = true;
  return cudaSuccess;
}

// K_P as pairs only (the sliced block's K^Q G product).
cudaError_t ensure_kp_df64(rssri_handle *h) {
  if (h->kp_hl_ready || h->P == 0) return cudaSuccess;
  RS_TRY(ensure(h->KPhl, (size_t)h->P * h->n_aux * sizeof(float2)));
  SPAN(RSSRI_PROF_OTHER, 0.0);
  RS_TRY(to_df64(h->KP.as<double>(), (long long)h->P * h->n_aux, h->KPhl.as<float2>(), h->stream,
                 range_flag(h)));
  h->kp_hl_ready = true;
  return cudaSuccess;
}

// The pair split of G and Gb for every tau (double-float block and chain).
cudaError_t ensure_gg(rssri_handle *h) {
  if (h->gg_valid) return cudaSuccess;
  const long long nn = (long long)h->n * h->n, nt = h->n_tau;
  RS_TRY(ensure(h->GGhl, (size_t)2 * nt * nn * sizeof(float2)));
  SPAN(RSSRI_PROF_OTHER, 0.0);
  // one conversion per tau point: the range check holds per matrix
  for (long long t = 0; t < nt; ++t) {
    RS_TRY(to_df64(h->G.as<double>() + t * nn, nn, h->GGhl.as<float2>() + t * nn, h->stream,
                   range_flag(h)));
    RS_TRY(to_df64(h->Gb.as<double>() + t * nn, nn, h->GGhl.as<float2>() + (nt + t) * nn,
                   h->stream, range_flag(h)));
  }
  h->gg_valid = true;
  return cudaSuccess;
}

// S6 and S7 for every tau point: G(tau) and G(beta - tau) from the orbitals
// (Eq. 17) or copied from the caller (g_in, gb_in: [n_tau][n][n] of the
// problem's pointer kind), then Sigma_DD(tau) (Eq. 20 on v^L = sum_Q
// [K^Q]^L [K^Q]^L, the deterministic terms of Eq. 25) in the arithmetic
// dd_arith.  The results stay in the handle (G, Gb, sdd) for the sampling calls.
int build_block(rssri_handle *h, int dd_arith, const double *g_in, const double *gb_in) {
  cudaStream_t s = h->stream;
  const int n = h->n, na = h->n_aux, nt = h->n_tau, P = h->P;
  const long long nn = (long long)n * n;
  h->block_ok = false;
  h->gg_valid = false;
  cudaError_t e;
#define RS_CK(x)                     \
  do {                               \
    e = (x);                         \
    if (e != cudaSuccess) { note_error_site(__FILE__, __LINE__); return map_err(e); } \
  } while (0)
  RS_CK(ensure(h->G, (size_t)nt * nn * sizeof(double)));
  RS_CK(ensure(h->Gb, (size_t)nt * nn * sizeof(double)));
  RS_CK(ensure(h->sdd, (size_t)nt * nn * sizeof(double)));
  const bool dd_df64 = P > 0 && dd_arith == RSSRI_DD_DF64;
  const bool dd_oz = P > 0 && dd_arith == RSSRI_DD_OZ;
  if (P > 0) {
    if (dd_oz) {
      // the exchange operand first (its fp64 gather is freed before the
      // per-tau buffers are made), then the per-tau buffers; T shares At's
      if (!h->oz_ready) {
        const int rc = oz_setup(h);
        if (rc) return rc;
      }
      RS_CK(ensure(h->PG, (size_t)nn * na * sizeof(double)));
      RS_CK(ensure(h->oz_gr, (size_t)nn * h->oz_w * sizeof(double)));
      RS_CK(oz_make(h->ozGr, n, n, h->oz_w));
      RS_CK(ensure(h->At, (size_t)nn * na * sizeof(double)));
      RS_CK(ensure(h->AP, (size_t)P * na * sizeof(double)));
      // the largest per-tau digit operand: n*na rows of ld16(n), n rows of ld16(n*na), or
      // na rows of n*ldl
      const long long ld_n = (n + 15) / 16 * 16, ld_kmq = ((long long)n * na + 15) / 16 * 16;
      const long long big = std::max({(long long)n * na * ld_n, (long long)n * ld_kmq,
                                      (long long)na * n * h->oz_geo.ldl});
      RS_CK(oz_make(h->ozGb, 1, n, n));
      RS_CK(oz_make(h->ozBig0, 1, 1, big));
      RS_CK(oz_make(h->ozBig1, 1, 1, big));
      RS_CK(ensure(h->ozBig0.e, (size_t)std::max<long long>(nn * na, n) * sizeof(int)));
      RS_CK(ensure(h->ozBig1.e, (size_t)std::max<long long>(na, n) * sizeof(int)));
      h->ozBig0.v.ef = h->ozBig0.e.as<int>();
      h->ozBig1.v.ef = h->ozBig1.e.as<int>();
      RS_CK(oz_make(h->ozAtP, 1, na, P));
      RS_CK(oz_make(h->ozGam, 1, na, na));
    } else if (!dd_df64) {  // the double-float block keeps these as pairs
      RS_CK(ensure(h->PG, (size_t)nn * na * sizeof(double)));
      RS_CK(ensure(h->At, (size_t)nn * na * sizeof(double)));
      RS_CK(ensure(h->AP, (size_t)P * na * sizeof(double)));
    }
    if (!dd_oz) RS_CK(ensure(h->T, (size_t)nn * na * sizeof(double)));
    RS_CK(ensure(h->L, (size_t)P * na * sizeof(double)));
    RS_CK(ensure(h->Gam, (size_t)na * na * sizeof(double)));
    RS_CK(ensure(h->gwork, std::max(h->gwork.bytes, dd_work_need(h) * 8)));
    if (dd_df64) {
      RS_CK(ensure(h->Ahl, (size_t)nn * na * sizeof(float2)));
      RS_CK(ensure(h->PGhl, (size_t)nn * na * sizeof(float2)));
      RS_CK(ensure(h->APhl, (size_t)P * na * sizeof(float2)));
      RS_CK(ensure(h->Gamhl, (size_t)na * na * sizeof(float2)));
      RS_CK(ensure_d_df64(h));
    }
  }
  double *G = h->G.as<double>(), *Gb = h->Gb.as<double>();
  // S6
  if (g_in) {
    const cudaMemcpyKind k = h->ptr_kind == RSSRI_PTR_HOST ? cudaMemcpyHostToDevice
                                                           : cudaMemcpyDeviceToDevice;
    RS_CK(cudaMemcpyAsync(G, g_in, nt * nn * sizeof(double), k, s));
    RS_CK(cudaMemcpyAsync(Gb, gb_in, nt * nn * sizeof(double), k, s));
  } else {
    RS_CK(build_green(h));
  }
  // S7 per tau
  if (dd_df64) RS_CK(ensure_gg(h));
  for (int t = 0; t < nt; ++t) {
    double *out = h->sdd.as<double>() + t * nn;
    if (dd_oz) {
      RS_CK(sigma_dd_tau_oz(h, G + t * nn, Gb + t * nn, out));
    } else if (dd_df64)
      RS_CK(sigma_dd_tau_df64(h, h->GGhl.as<float2>() + t * nn,
                              h->GGhl.as<float2>() + (nt + t) * nn, out));
    else
      RS_CK(sigma_dd_tau(h, G + t * nn, Gb + t * nn, out));
  }
  if (dd_oz) {
    // a bounded wait of the tensor-core kernels that gave up
    int fl = 0;
    RS_CK(fetch(&fl, h->flags.as<int>() + 5, s));
    if (fl) return RSSRI_ERR_TIMEOUT;
#ifdef RSSRI_CHECKS
    int chk[4];
    RS_CK(oz_check_fetch(chk));
    if (chk[0]) {
      std::fprintf(stderr, "rssri bounds check %d failed at oz_gemm.cu:%d, index %lld\n", chk[0],
                   chk[1], ((long long)chk[3] << 32) | (unsigned)chk[2]);
      return RSSRI_ERR_CUDA;
    }
#endif
  }
  h->block_ok = true;
  h->block_from_g = g_in != nullptr;
  return RSSRI_OK;
#undef RS_CK
}

// S8 on the tensor cores (bf16 or tf32 operands, fp32 accumulation), all
// sample pairs at once, tau points in chunks of tc tau per stage:
//   P = [R^S; R^L] G,  dC = P_S R' + P_L R'^S,  C^L = P_L R'^L,
//   [X; Y] = [dC; C^L] Gb,  fold (traces, energy, 2 dt I - X, 2 t^L I - Y, C^T, dC^T),
//   sum_x (2 dt I - X) C + (2 t^L I - Y) dC  (one contraction over the pairs).
// sig[t] = sdd[t] + that sum / n_s.  e_st accumulates the pair energies.
// Each stage of a chunk (all its tau points, all pairs) is one persistent
// launch of tc_group: its products go into one device work queue of tiles.
// The launches are issued into a CUDA graph once and the graph is replayed
// while the shapes, buffers and tau weights stay the same.
struct ChainBufs {
  int kind;  // TcKind of the operands
  int wait_polls;  // testing (see TcGemm)
  const double *cvc;  // coefficients c [n_tau][n][n] of the learned control variate, or null
  void *clt;          // (C^L)^T operands [tc][ns][n][ldp] (control variate)
  float *fl;          // F^L per pair [tc][ns][n][n] fp32 (control variate)
  size_t es;  // operand element size
  int tc;     // tau points per chunk
  // per chunk slot j < tc (buffers hold tc slots):
  void *xsl, *y3, *gh, *gbh, *P, *dcl, *a6, *ct, *dct;
  float *dc32, *cl32, *xy32, *part;
  double *fold;
  int bpc, groups;
};

// The products of the chain's stages for tau points [t0, t0 + c) (slot j = t - t0).
void chain_stage_probs(rssri_handle *h, const ChainBufs &b, int ns, int t0, int c, int stage,
                       std::vector<TcProb> &out) {
  const int n = h->n;
  const int ldp = (n + 7) / 8 * 8;
  const long long nn = (long long)n * n, mat = (long long)n * ldp;
  auto at = [&](void *p, long long e) { return static_cast<void *>(static_cast<char *>(p) + e * b.es); };
  auto op = [&](const void *p, long long sb, int rows) {
    TcOperand t;
    t.ptr = p;
    t.ld = ldp;
    t.sb = sb;
    t.rows = rows;
    return t;
  };
  out.clear();
  if (stage == 0) {  // P = [R^S; R^L] G for every tau of the chunk: batch over tau
    TcProb g;
    g.M = 2 * ns * n; g.N = n; g.K[0] = n; g.batch = c;
    g.A[0] = op(b.xsl, 0, 2 * ns * n); g.B[0] = op(at(b.gh, (long long)t0 * mat), mat, n);
    g.cop = b.P; g.ldcop = ldp;
    out.push_back(g);
  } else if (stage == 1) {  // dC = P_S R' + P_L R'^S and C^L = P_L R'^L per tau
    for (int j = 0; j < c; ++j) {
      void *Pj = at(b.P, (long long)j * 2 * ns * mat);
      TcProb g;
      g.M = n; g.N = n; g.batch = ns; g.nseg = 2; g.K[0] = g.K[1] = n;
      g.A[0] = op(Pj, mat, n); g.B[0] = op(b.y3, mat, n);
      g.A[1] = op(at(Pj, ns * mat), mat, n); g.B[1] = op(at(b.y3, ns * mat), mat, n);
      g.c32 = b.dc32 + (long long)j * ns * nn;
      g.cop = at(b.dcl, (long long)j * 2 * ns * mat); g.ldcop = ldp;
      out.push_back(g);
      TcProb l;
      l.M = n; l.N = n; l.batch = ns; l.K[0] = n;
      l.A[0] = op(at(Pj, ns * mat), mat, n); l.B[0] = op(at(b.y3, 2 * ns * mat), mat, n);
      l.c32 = b.cl32 + (long long)j * ns * nn;
      l.cop = at(b.dcl, ((long long)j * 2 * ns + ns) * mat); l.ldcop = ldp;
      out.push_back(l);
    }
  } else if (stage == 2) {  // [X; Y] = [dC; C^L] Gb for every tau: batch over tau
    TcProb g;
    g.M = 2 * ns * n; g.N = n; g.K[0] = n; g.batch = c;
    g.A[0] = op(b.dcl, 2 * ns * mat, 2 * ns * n);
    g.B[0] = op(at(b.gbh, (long long)t0 * mat), mat, n);
    g.c32 = b.xy32;
    out.push_back(g);
  } else if (stage == 3) {  // sum over pairs of (2 dt I - X) C + (2 t^L I - Y) dC per tau
    for (int j = 0; j < c; ++j) {
      void *A6 = at(b.a6, (long long)j * 2 * ns * mat);
      TcProb g;
      g.M = n; g.N = n; g.batch = ns; g.bpc = b.bpc; g.nseg = 2; g.K[0] = g.K[1] = n;
      g.A[0] = op(A6, mat, n); g.B[0] = op(at(b.ct, (long long)j * ns * mat), mat, n);
      g.A[1] = op(at(A6, ns * mat), mat, n); g.B[1] = op(at(b.dct, (long long)j * ns * mat), mat, n);
      g.c32 = b.part + (long long)j * b.groups * nn;
      out.push_back(g);
    }
  } else {  // F^L = (2 t^L I - Y) C^L per pair and tau (learned control variate)
    for (int j = 0; j < c; ++j) {
      TcProb g;
      g.M = n; g.N = n; g.batch = ns; g.K[0] = n;
      g.A[0] = op(at(b.a6, ((long long)j * 2 * ns + ns) * mat), mat, n);
      g.B[0] = op(at(b.clt, (long long)j * ns * mat), mat, n);
      g.c32 = b.fl + (long long)j * ns * nn;
      out.push_back(g);
    }
  }
}

cudaError_t issue_chain_tc(rssri_handle *h, cudaStream_t s, int ns, const double *G,
                           const double *Gb, const double *sdd, double *sig, int *err,
                           const ChainBufs &b) {
  const int n = h->n, nt = h->n_tau;
  const int ldp = (n + 7) / 8 * 8;
  const long long nn = (long long)n * n, mat = (long long)n * ldp;
  RS_TRY(chain_factors(b.kind, h->fac.as<double>(), ns, n, ldp, b.xsl, b.y3, s));
  RS_TRY(chain_matrices(b.kind, G, nt, n, ldp, b.gh, s));
  RS_TRY(chain_matrices(b.kind, Gb, nt, n, ldp, b.gbh, s));
  const double ne = 2.0 * h->n_occ;
  auto at = [&](void *p, long long e) { return static_cast<void *>(static_cast<char *>(p) + e * b.es); };
  std::vector<TcProb> probs;
  for (int t0 = 0; t0 < nt; t0 += b.tc) {
    const int c = std::min(b.tc, nt - t0);
    for (int stage = 0; stage < 3; ++stage) {
      chain_stage_probs(h, b, ns, t0, c, stage, probs);
      RS_TRY(tc_group(b.kind, probs.data(), (int)probs.size(), err, s, b.wait_polls));
    }
    for (int j = 0; j < c; ++j)
      RS_TRY(fold_tc(b.kind, b.xy32 + (long long)j * 2 * ns * nn, b.dc32 + (long long)j * ns * nn,
                     b.cl32 + (long long)j * ns * nn, ns, n, ldp, h->h_tau_w[t0 + j], ne,
                     at(b.a6, (long long)j * 2 * ns * mat), at(b.ct, (long long)j * ns * mat),
                     at(b.dct, (long long)j * ns * mat),
                     b.cvc ? at(b.clt, (long long)j * ns * mat) : nullptr, h->e_st.as<double>(),
                     b.fold + (long long)j * ns * ceil_div(n, 32) * 4, s));
    chain_stage_probs(h, b, ns, t0, c, 3, probs);
    RS_TRY(tc_group(b.kind, probs.data(), (int)probs.size(), err, s, b.wait_polls));
    for (int j = 0; j < c; ++j)
      RS_TRY(reduce_tc(b.part + (long long)j * b.groups * nn, b.groups, n, sdd + (t0 + j) * nn,
                       (double)ns, sig + (t0 + j) * nn, s));
    if (b.cvc) {
      chain_stage_probs(h, b, ns, t0, c, 4, probs);
      RS_TRY(tc_group(b.kind, probs.data(), (int)probs.size(), err, s, b.wait_polls));
      for (int j = 0; j < c; ++j)
        RS_TRY(cv_tc_apply(b.fl + (long long)j * ns * nn, ns, n, b.cvc + (t0 + j) * nn,
                           sdd + (t0 + j) * nn, Gb + (t0 + j) * nn, h->h_tau_w[t0 + j], ne,
                           sig + (t0 + j) * nn, h->e_st.as<double>(), s));
    }
  }
  return cudaSuccess;
}

cudaError_t chain_tc(rssri_handle *h, int kind, int ns, const double *G, const double *Gb,
                     const double *sdd, double *sig, int *err, const double *cvc) {
  cudaStream_t s = h->stream;
  const int n = h->n, nt = h->n_tau;
  const int ldp = (n + 7) / 8 * 8;
  const long long nn = (long long)n * n, mat = (long long)n * ldp;
  ChainBufs b;
  b.kind = kind;
  b.wait_polls = h->test_wait_polls;
  b.cvc = cvc;
  b.clt = nullptr;
  b.fl = nullptr;
  b.es = kind == TC_BF16 ? sizeof(__nv_bfloat16) : sizeof(float);
  const size_t b16 = b.es;
  b.bpc = std::max(1, ceil_div(ns, 152));
  b.groups = ceil_div(ns, b.bpc);
  // tau points per chunk: as many as fit a scratch budget of 8 GB (at least 1)
  const size_t per_tau = 2 * ns * mat * b16 /*P*/ + 2 * ns * nn * 4 /*dC, C^L fp32*/ +
                         2 * ns * mat * b16 /*dcl*/ + 2 * ns * nn * 4 /*X, Y*/ +
                         2 * ns * mat * b16 /*a6*/ + 2 * ns * mat * b16 /*ct, dct*/ +
                         (size_t)b.groups * nn * 4 /*part*/ +
                         (cvc ? ns * mat * b16 + ns * nn * 4 : 0);
  b.tc = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::min(nt, 12),
                                                   ((size_t)8 << 30) / per_tau));
  const int tc = b.tc;
  RS_TRY(ensure(h->hxsl, 2 * ns * mat * b16));
  RS_TRY(ensure(h->hy3, 3 * ns * mat * b16));
  RS_TRY(ensure(h->hg, nt * mat * b16));
  RS_TRY(ensure(h->hgb, nt * mat * b16));
  RS_TRY(ensure(h->hP, (size_t)tc * 2 * ns * mat * b16));
  RS_TRY(ensure(h->hdc32, (size_t)tc * ns * nn * sizeof(float)));
  RS_TRY(ensure(h->hcl32, (size_t)tc * ns * nn * sizeof(float)));
  RS_TRY(ensure(h->hdcl16, (size_t)tc * 2 * ns * mat * b16));
  RS_TRY(ensure(h->hxy32, (size_t)tc * 2 * ns * nn * sizeof(float)));
  RS_TRY(ensure(h->ha6, (size_t)tc * 2 * ns * mat * b16));
  RS_TRY(ensure(h->hct, (size_t)tc * ns * mat * b16));
  RS_TRY(ensure(h->hdct, (size_t)tc * ns * mat * b16));
  RS_TRY(ensure(h->hpart, (size_t)tc * b.groups * nn * sizeof(float)));
  RS_TRY(ensure(h->hfold, (size_t)tc * ns * ceil_div(n, 32) * 4 * sizeof(double)));
  if (cvc) {
    RS_TRY(ensure(h->hclt, (size_t)tc * ns * mat * b16));
    RS_TRY(ensure(h->hfl, (size_t)tc * ns * nn * sizeof(float)));
    b.clt = h->hclt.p;
    b.fl = h->hfl.as<float>();
  }
  b.xsl = h->hxsl.p; b.y3 = h->hy3.p; b.gh = h->hg.p; b.gbh = h->hgb.p; b.P = h->hP.p;
  b.dcl = h->hdcl16.p; b.a6 = h->ha6.p; b.ct = h->hct.p; b.dct = h->hdct.p;
  b.dc32 = h->hdc32.as<float>(); b.cl32 = h->hcl32.as<float>(); b.xy32 = h->hxy32.as<float>();
  b.part = h->hpart.as<float>();
  b.fold = h->hfold.as<double>();
  RS_TRY(tc_prepare());
  // the graph is keyed on every pointer and value baked into its launches
  std::vector<uintptr_t> key = {(uintptr_t)kind, (uintptr_t)b.wait_polls, (uintptr_t)ns, (uintptr_t)n,
                                (uintptr_t)nt, (uintptr_t)h->n_occ, (uintptr_t)tc,
                                (uintptr_t)G, (uintptr_t)Gb, (uintptr_t)sig, (uintptr_t)err,
                                (uintptr_t)cvc, (uintptr_t)b.clt, (uintptr_t)b.fl,
                                (uintptr_t)h->fac.p, (uintptr_t)h->e_st.p, (uintptr_t)sdd};
  for (DevBuf *d : {&h->hxsl, &h->hy3, &h->hg, &h->hgb, &h->hP, &h->hdc32, &h->hcl32, &h->hdcl16,
                    &h->hxy32, &h->ha6, &h->hct, &h->hdct, &h->hpart, &h->hfold})
    key.push_back((uintptr_t)d->p);
  if (!h->chain_graph || key != h->chain_key_ptr || h->h_tau_w != h->chain_key_w) {
    if (h->chain_graph) cudaGraphExecDestroy(h->chain_graph);
    h->chain_graph = nullptr;
    // tune the N tile of every stage's product shape (outside the capture;
    // each shape is tuned once per process)
    if (!b.wait_polls) {
      std::vector<TcProb> probs;
      for (int stage = 0; stage < (cvc ? 5 : 4); ++stage) {
        chain_stage_probs(h, b, ns, 0, std::min(tc, nt), stage, probs);
        tc_group_tune(kind, probs[0], err, s);
      }
      RS_TRY(cudaStreamSynchronize(s));
      RS_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    }
    cudaGraph_t graph = nullptr;
    if (!h->cap_stream) RS_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    RS_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const long long l0 = launch_counter();
    const cudaError_t ei = issue_chain_tc(h, h->cap_stream, ns, G, Gb, sdd, sig, err, b);
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
    const long long captured = launch_counter() - l0;
    launch_counter() = l0;  // captured, not yet run
    if (ei != cudaSuccess || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return ei != cudaSuccess ? ei : ec;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t eg = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    RS_TRY(eg);
    h->chain_graph = exec;
    h->chain_key_ptr = key;
    h->chain_key_w = h->h_tau_w;
    h->chain_graph_launches = captured;
  }
  SPAN_T(RSSRI_PROF_CHAIN_GEMM, 18.0 * ns * (double)n * n * n * nt * 1e-9,
         18.0 * ns * (double)n * n * n * nt * 1e-9);
  RS_TRY(cudaGraphLaunch(h->chain_graph, s));
  launch_counter() += h->chain_graph_launches;
  return cudaSuccess;
}

// Coefficients c(tau, i, j) of the trained network for the current G and Sigma_DD.
constexpr int CV_CHUNK = 65536;

size_t cv_work_floats(int batch) {
  const int m = std::max(batch, 2048);
  return cv_tc_work_floats() + std::max({sgemm_work_floats(CV_HIDDEN, CV_HIDDEN, m),
                   sgemm_work_floats(CV_HIDDEN, CV_NFEAT, m), sgemm_work_floats(1, CV_HIDDEN, m),
                   (size_t)1024});
}

cudaError_t cv_compute_c(rssri_handle *h, const double *G, const double *Gb) {
  cudaStream_t s = h->stream;
  const int n = h->n, nt = h->n_tau;
  const long long nn = (long long)n * n, total = nn * nt;
  RS_TRY(ensure(h->cv_X, total * CV_NFEAT * sizeof(float)));
  RS_TRY(ensure(h->cv_scr, (3 * nt + n + 1) * sizeof(double)));
  RS_TRY(ensure(h->cv_c, total * sizeof(double)));
  RS_TRY(ensure(h->cv_act, cv_act_floats(CV_CHUNK) * sizeof(float)));
  RS_TRY(ensure(h->cv_work, cv_work_floats(CV_CHUNK) * sizeof(float)));
  SPAN(RSSRI_PROF_OTHER, 0.0);
  RS_TRY(cv_features(h->sdd.as<double>(), G, Gb, h->tau, h->beta, h->KP.as<double>(),
                     h->rowptr.as<int>(), h->n_aux, n, nt, h->cv_scr.as<double>(),
                     h->cv_X.as<float>(), s));
  for (long long m0 = 0; m0 < total; m0 += CV_CHUNK) {
    const int m = (int)std::min<long long>(CV_CHUNK, total - m0);
    RS_TRY(cv_forward(h->cv_params.as<float>(), h->cv_X.as<float>() + m0 * CV_NFEAT, m,
                      h->cv_act.as<float>(), h->cv_work.as<float>(), s));
    RS_TRY(cv_coefficients(h->cv_act.as<float>() + 6LL * m * CV_HIDDEN, m,
                           h->cv_c.as<double>() + m0, s));
  }
  return cudaSuccess;
}

// The cross terms of the literal estimator (Eq. 25 with D exact inside each
// bracket) for one tau and one batch of cnt sample pairs.  Phi is bilinear,
// so Phi(D, S') + Phi(S, D) = sum_{y = R', R'^L} (+-) sum_Q F(K^Q, y) +
// sum_{x = R, R^L} (+-) sum_Q F(x, K^Q) with K^Q = [K^Q]^L, and
//   sum_Q F(K^Q, y) = (2 J_y - X_y) G y,   M_y = G y Gb,
//   sum_Q F(x, K^Q) = x G (2 J'_x - X'_x), M'_x = Gb x G,
// where for a matrix M: J = sum_Q Tr(K^Q M) K^Q (direct; K^Q symmetric, so
// Tr(K^Q M) = sum over kept pairs of K_P M) and X = sum_Q K^Q M K^Q, the
// exchange build X_mj = sum_{a in row m, b in row j} v^L_ab M[col a][col b]
// in pair space (the same contraction as the deterministic block's with the
// aux index replaced by the batch of matrices).  The four sides are batched
// as s = side * cnt + x; the result is added to the first chain slot of BC
// and to the pair energies.  XG, Cc, Bm are free scratch here.
cudaError_t literal_cross(rssri_handle *h, const rssri_options *o, int t, int x0, int cnt,
                          const double *Gt, const double *Gbt, double *XG, double *Cc, double *Bm,
                          double *BC) {
  cudaStream_t s = h->stream;
  const int n = h->n, na = h->n_aux, ns = (int)o->n_s, P = h->P;
  const long long nn = (long long)n * n;
  const int S = 4 * cnt;
  const double *fac = h->fac.as<double>();
  auto factor = [&](int set, int kind) { return fac + ((2LL * set + kind) * ns + x0) * nn; };
  // sides: 0 = y R' (+), 1 = y R'^L (-), 2 = x R (+), 3 = x R^L (-)
  double *M = Cc, *tmp = XG;
  for (int side = 0; side < 4; ++side) {
    const bool yside = side < 2;
    const double *F = yside ? factor(1, side) : factor(0, side - 2);
    GemmArgs g;
    g.M = n; g.N = n; g.K = n; g.batch = cnt;
    g.lda = g.ldb = g.ldc = n;
    double *tm = tmp + (long long)side * cnt * nn, *mm = M + (long long)side * cnt * nn;
    // y side: M = G y Gb; x side: M = Gb x G
    g.A = yside ? Gt : Gbt; g.sA = 0; g.B = F; g.sB = nn; g.C = tm; g.sC = nn;
    RS_TRY(gemm_p(h, RSSRI_PROF_CHAIN_GEMM, g));
    g.A = tm; g.sA = nn; g.B = yside ? Gbt : Gt; g.sB = 0; g.C = mm; g.sC = nn;
    RS_TRY(gemm_p(h, RSSRI_PROF_CHAIN_GEMM, g));
  }
  double *Mt = Bm;  // [k][l][s]
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_TRY(lit_qfast(M, S, nn, Mt, s)); }
  // direct: tQ = K_P^T M_P, J_P = K_P tQ
  double *MP = h->litMP.as<double>(), *tQ = h->litT.as<double>();
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_TRY(gather_rows(Mt, h->pij.as<int>(), P, S, MP, s)); }
  {
    GemmArgs g;
    g.M = na; g.N = S; g.K = P;
    g.A = h->KP.as<double>(); g.lda = na; g.transA = 1;
    g.B = MP; g.ldb = S;
    g.C = tQ; g.ldc = S;
    RS_TRY(gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  {
    GemmArgs g;
    g.M = P; g.N = S; g.K = na;
    g.A = h->KP.as<double>(); g.lda = na;
    g.B = tQ; g.ldb = S;
    g.C = MP; g.ldc = S;  // J_P overwrites the gathered M_P
    RS_TRY(gemm_p(h, RSSRI_PROF_DD_GEMM, g));
  }
  // exchange: Tk[m][s][j] = sum_{a in row m, b in row j} D[a][b] Mt[(col a, col b)][s]
  double *Tk = XG;
  {
    SPAN(RSSRI_PROF_DD_SPMM, 2.0 * S * (double)P * P * 1e-9);
    if (o->dd_arith != RSSRI_DD_FP64) {
      RS_TRY(to_df64(Mt, S * nn, h->litMhl.as<float2>(), s));
      RS_TRY(dd_exchange_spmm_df64(h->rowptr.as<int>(), h->pcol.as<int>(), h->Dhl.as<float2>(), P,
                                   h->litMhl.as<float2>(), n, S, Tk, s));
    } else {
      RS_TRY(dd_exchange_spmm(h->rowptr.as<int>(), h->pcol.as<int>(), h->D.as<double>(), P, Mt, n,
                              S, Tk, s));
    }
  }
  // W[s] = 2 J_s - X_s
  double *W = Cc;
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_TRY(lit_w(Tk, S, n, MP, h->pij.as<int>(), P, W, s)); }
  // Z: y side (W G) y, x side (x G) W
  double *Z = XG;
  for (int side = 0; side < 4; ++side) {
    const bool yside = side < 2;
    const double *F = yside ? factor(1, side) : factor(0, side - 2);
    GemmArgs g;
    g.M = n; g.N = n; g.K = n; g.batch = cnt;
    g.lda = g.ldb = g.ldc = n;
    double *tm = Bm + (long long)side * cnt * nn, *zz = Z + (long long)side * cnt * nn;
    const double *ww = W + (long long)side * cnt * nn;
    if (yside) {
      g.A = ww; g.sA = nn; g.B = Gt; g.sB = 0; g.C = tm; g.sC = nn;
      RS_TRY(gemm_p(h, RSSRI_PROF_CHAIN_GEMM, g));
      g.A = tm; g.sA = nn; g.B = F; g.sB = nn; g.C = zz; g.sC = nn;
      RS_TRY(gemm_p(h, RSSRI_PROF_CHAIN_GEMM, g));
    } else {
      g.A = F; g.sA = nn; g.B = Gt; g.sB = 0; g.C = tm; g.sC = nn;
      RS_TRY(gemm_p(h, RSSRI_PROF_CHAIN_GEMM, g));
      g.A = tm; g.sA = nn; g.B = ww; g.sB = nn; g.C = zz; g.sC = nn;
      RS_TRY(gemm_p(h, RSSRI_PROF_CHAIN_GEMM, g));
    }
  }
  SPAN(RSSRI_PROF_OTHER, 0.0);
  return lit_add(Z, cnt, n, Gbt, h->h_tau_w[t], 2.0 * h->n_occ, BC,
                 h->e_st.as<double>() + x0, s);
}

// Enqueues S4-S10 on the handle's stream; the energies and the tensor-core
// flag are copied into the handle's pinned host buffer, read by finish_sigma.
int issue_sigma(rssri_handle *h, const rssri_options *o, const double *g_in, const double *gb_in,
                double *sigma, double *e_pair, bool collect_stats) {
  if (!h) return RSSRI_ERR_INVALID_ARG;
  if (h->broken) return RSSRI_ERR_CUDA;
  if (!h->ready) return RSSRI_ERR_NOT_READY;
  if (h->pending) return RSSRI_ERR_INVALID_ARG;  // one enqueued call per handle
  int rc = validate_options(o, true);
  if (rc) return rc;
  if (!sigma && !collect_stats) return RSSRI_ERR_INVALID_ARG;
  const bool use_cv = o->cv != 0;
  if ((use_cv || collect_stats) && o->estimator != RSSRI_EST_CV) return RSSRI_ERR_INVALID_ARG;
  if (collect_stats && o->precision != RSSRI_PREC_FP64 && o->precision != RSSRI_PREC_DF64)
    return RSSRI_ERR_INVALID_ARG;
  if (use_cv && !h->cv_ready) return RSSRI_ERR_NOT_READY;
  if (cudaSetDevice(h->device) != cudaSuccess) return RSSRI_ERR_CUDA;
  AllocFailScope alloc_test(o->test_fail_alloc);
  h->test_wait_polls = o->test_wait_polls;
  cudaStream_t s = h->stream;
  const int n = h->n, na = h->n_aux, nt = h->n_tau;
  const int ns = (int)o->n_s;
  const long long nn = (long long)n * n;
  const bool sri = o->estimator == RSSRI_EST_SRI;
  const bool literal = o->estimator == RSSRI_EST_LITERAL;
  const int P = sri ? 0 : h->P;
  const int nb = (o->pair_batch > 0) ? (int)std::min<long long>(o->pair_batch, ns) : ns;
  const int has_l = sri ? 0 : 1;
  // chain kinds (X, Y): 0 = (R, R'), 1 = (R^L, R'^L); the literal estimator
  // adds 2 = (R, R'^L) and 3 = (R^L, R'), which enter with a minus sign
  const int nkind = literal ? 4 : 1 + has_l;
  const int nbat2 = nb * nkind;
  // tensor-core chain (bf16 or tf32 operands) instead of the fp64 one
  const bool bf16 = o->precision == RSSRI_PREC_BF16 || o->precision == RSSRI_PREC_TF32;
  const int tc_kind = o->precision == RSSRI_PREC_TF32 ? TC_TF32 : TC_BF16;
  if (bf16 && (n < 16 || !tc_available())) return RSSRI_ERR_INVALID_ARG;
  // the chain in double-float (fp64-accurate) instead of IEEE fp64
  const bool chain_df64 = o->precision == RSSRI_PREC_DF64;
  cudaError_t e;
#define RS_CK(x)                                       \
  do {                                                 \
    e = (x);                                           \
    if (e != cudaSuccess) {                            \
      note_error_site(__FILE__, __LINE__);             \
      int _r = map_err(e);                             \
      if (_r == RSSRI_ERR_CUDA) h->broken = true;      \
      return _r;                                       \
    }                                                  \
  } while (0)

  h->recs.clear();
  h->ev_used = 0;
  h->prof_on = o->profile != 0;
  RS_CK(cudaMemsetAsync(range_flag(h), 0, 3 * sizeof(int), s));
  // bounded-wait flags of the tensor-core kernels: 4 sampling, 5 block
  RS_CK(cudaMemsetAsync(h->flags.as<int>() + 4, 0, 2 * sizeof(int), s));
  RS_CK(cudaEventRecord(h->ev[2], s));
  // ---- buffers
  RS_CK(ensure(h->sig_raw, (size_t)nt * nn * sizeof(double)));
  RS_CK(ensure(h->sig_out, (size_t)nt * nn * sizeof(double)));
  RS_CK(ensure(h->trdd, nt * sizeof(double)));
  RS_CK(ensure(h->tr, nt * sizeof(double)));
  RS_CK(ensure(h->res, 8 * sizeof(double)));
  RS_CK(ensure(h->theta, (size_t)2 * ns * na * sizeof(double)));
  RS_CK(ensure(h->Ut, (size_t)2 * ns * na * sizeof(double)));
  RS_CK(ensure(h->fac, (size_t)4 * ns * nn * sizeof(double)));  // [set][kind][xi][n][n]
  RS_CK(ensure(h->RLp, (size_t)2 * ns * std::max(h->P, 1) * sizeof(double)));
  if (!bf16) {
    if (chain_df64) {
      RS_CK(ensure(h->facHl, (size_t)4 * ns * nn * sizeof(float2)));
      RS_CK(ensure(h->xgHl, (size_t)nbat2 * nn * sizeof(float2)));
      RS_CK(ensure(h->cHl, (size_t)nbat2 * nn * sizeof(float2)));
      RS_CK(ensure(h->bHl, (size_t)nbat2 * nn * sizeof(float2)));
    } else {
      RS_CK(ensure(h->XG, (size_t)nbat2 * nn * sizeof(double)));
      RS_CK(ensure(h->Cc, (size_t)nbat2 * nn * sizeof(double)));
    }
    RS_CK(ensure(h->Bm, (size_t)nbat2 * nn * sizeof(double)));
    RS_CK(ensure(h->BC, (size_t)nbat2 * nn * sizeof(double)));
  }
  RS_CK(ensure(h->tarr, nbat2 * sizeof(double)));
  RS_CK(ensure(h->sarr, nbat2 * sizeof(double)));
  RS_CK(ensure(h->e_st, ns * sizeof(double)));
  RS_CK(ensure(h->e_pair, ns * sizeof(double)));
  if (literal && P > 0) {
    RS_CK(ensure(h->litMP, (size_t)P * nbat2 * sizeof(double)));
    RS_CK(ensure(h->litT, (size_t)na * nbat2 * sizeof(double)));
    if (o->dd_arith != RSSRI_DD_FP64) {
      RS_CK(ensure(h->litMhl, (size_t)nbat2 * nn * sizeof(float2)));
      RS_CK(ensure_d_df64(h));
    }
  }

  // ---- S6, S7: the cached block of the setup, or a new one for the caller's G
  h->pending_block = g_in || !h->block_ok || h->block_from_g;
  if (g_in) {
    rc = build_block(h, o->dd_arith, g_in, gb_in);
    if (rc) { if (rc == RSSRI_ERR_CUDA) h->broken = true; return rc; }
  } else if (!h->block_ok || h->block_from_g) {
    rc = build_block(h, h->setup_arith, nullptr, nullptr);
    if (rc) { if (rc == RSSRI_ERR_CUDA) h->broken = true; return rc; }
  }
  double *G = h->G.as<double>(), *Gb = h->Gb.as<double>();
  // the block the estimator adds to: Sigma_DD, or zero for plain stochastic RI
  const double *sdd = h->sdd.as<double>();
  if (sri) {
    RS_CK(ensure(h->sdd0, (size_t)nt * nn * sizeof(double)));
    RS_CK(cudaMemsetAsync(h->sdd0.p, 0, (size_t)nt * nn * sizeof(double), s));
    sdd = h->sdd0.as<double>();
  }
  if (chain_df64) RS_CK(ensure_gg(h));
  RS_CK(cudaEventRecord(h->ev[3], s));

  // ---- S4: theta, theta' and U^T = theta W (W symmetric)
  double *theta = h->theta.as<double>(), *Ut = h->Ut.as<double>(), *fac = h->fac.as<double>();
  for (int set = 0; set < 2; ++set)
    { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(rademacher(o->seed, set, o->xi_offset, ns, na, theta + (long long)set * ns * na, s)); }
  // the factor products in the block's arithmetic: IEEE fp64, double-float
  // (operands split into pairs first), or sliced on the tensor cores
  // (sliced only under a bf16 / tf32 chain, which rounds R and R^L to 8 or
  // 11 bits anyway: the sliced products carry ~1e-12 of their row scales,
  // which an fp64-accurate chain would see in R^S = R - R^L)
  const bool fac_oz = o->dd_arith == RSSRI_DD_OZ && bf16;
  const bool fac_df64 = o->dd_arith != RSSRI_DD_FP64 && !fac_oz;
  int *tc_err = h->flags.as<int>() + 4;
  if (fac_oz) {
    OzView vt = oz_rows(theta, na, na, 2LL * ns * na);
    vt.bs = (long long)ns * na;
    const OzView vw = oz_cols(h->W.as<double>(), na, na, (long long)na * na);
    RS_CK(oz_product(h, RSSRI_PROF_FACTOR_GEMM, vt, 2, ns, &vw, na, na, Ut, na,
                     (long long)ns * na, tc_err));
  } else {
    GemmArgs g;
    g.M = ns; g.N = na; g.K = na; g.batch = 2;
    g.A = theta; g.lda = na; g.sA = (long long)ns * na;
    g.B = h->W.as<double>(); g.ldb = na; g.sB = 0;
    g.C = Ut; g.ldc = na; g.sC = (long long)ns * na;
    RS_CK(gemm_p(h, RSSRI_PROF_FACTOR_GEMM, g));
  }
  // ---- S5: R[set][xi][ij] = sum_A U^T[xi][A] (ij|A); R^L from the kept pairs
  if (fac_oz) {
    // (ij|A) sliced in blocks of rows, so that its digits stay within ~3 GB
    OzView vu = oz_rows(Ut, na, na, 2LL * ns * na);
    vu.bs = (long long)ns * na;
    RS_CK(oz_make(h->ozPA, 2, ns, na));
    RS_CK(oz_slice_p(h, vu, h->ozPA.v));
    const long long ldk = ((long long)na + 15) / 16 * 16;
    const long long chunk = std::max<long long>(128, ((1LL << 28) / ldk) / 128 * 128);
    for (long long r0 = 0; r0 < nn; r0 += chunk) {
      const int rows = (int)std::min(chunk, nn - r0);
      const OzView ve = oz_rows(h->eri3 + r0 * na, na, na, (long long)rows * na);
      RS_CK(oz_make(h->ozPB, 1, rows, na));
      RS_CK(oz_slice_p(h, ve, h->ozPB.v));
      OzGemm g;
      g.A = h->ozPA.v; g.B = h->ozPB.v;
      g.M = ns; g.N = rows; g.batch = 2;
      g.C = fac + r0; g.ldc = nn; g.sC = 2LL * ns * nn;  // kind 0 of each set
      g.ccap = 4LL * ns * nn - r0;
      g.err = tc_err;
      RS_CK(oz_gemm_p(h, RSSRI_PROF_FACTOR_GEMM, g));
    }
  } else if (fac_df64) {
    RS_CK(ensure(h->eri_hl, (size_t)nn * na * sizeof(float2)));
    RS_CK(ensure(h->ut_hl, (size_t)2 * ns * na * sizeof(float2)));
    {
      SPAN(RSSRI_PROF_OTHER, 0.0);
      RS_CK(to_df64(h->eri3, nn * na, h->eri_hl.as<float2>(), s, range_flag(h)));
      RS_CK(to_df64(Ut, 2LL * ns * na, h->ut_hl.as<float2>(), s, range_flag(h)));
    }
    SPAN(RSSRI_PROF_FACTOR_GEMM, 2.0 * 2 * ns * (double)nn * na * 1e-9);
    DfGemm g;
    g.M = ns; g.N = (int)nn; g.K = na; g.batch = 2;
    g.A = h->ut_hl.as<float2>(); g.lda = na; g.sA = (long long)ns * na;
    g.B = h->eri_hl.as<float2>(); g.ldb = na; g.transB = 1; g.sB = 0;
    g.C64 = fac; g.ldc = nn; g.sC = 2LL * ns * nn;  // kind 0 of each set
    RS_CK(df_gemm_w(h, g));
  } else {
    GemmArgs g;
    g.M = ns; g.N = (int)nn; g.K = na; g.batch = 2;
    g.A = Ut; g.lda = na; g.sA = (long long)ns * na;
    g.B = h->eri3; g.ldb = na; g.transB = 1; g.sB = 0;
    g.C = fac; g.ldc = nn; g.sC = 2LL * ns * nn;  // kind 0 of each set
    RS_CK(gemm_p(h, RSSRI_PROF_FACTOR_GEMM, g));
  }
  for (int set = 0; set < 2; ++set) {
    double *rl = fac + (2LL * set + 1) * ns * nn;
    RS_CK(cudaMemsetAsync(rl, 0, (size_t)ns * nn * sizeof(double), s));
  }
  if (P > 0 && fac_oz) {
    OzView vt = oz_rows(theta, na, na, 2LL * ns * na);
    vt.bs = (long long)ns * na;
    const OzView vk = oz_rows(h->KP.as<double>(), na, na, (long long)P * na);
    RS_CK(oz_product(h, RSSRI_PROF_FACTOR_GEMM, vt, 2, ns, &vk, P, na, h->RLp.as<double>(), P,
                     (long long)ns * P, tc_err));
  } else if (P > 0 && fac_df64) {
    // theta is +-1, exact as a pair; K_P was split at setup
    { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(to_df64(theta, 2LL * ns * na, h->ut_hl.as<float2>(), s, range_flag(h))); }
    SPAN(RSSRI_PROF_FACTOR_GEMM, 2.0 * 2 * ns * (double)P * na * 1e-9);
    DfGemm g;
    g.M = ns; g.N = P; g.K = na; g.batch = 2;
    g.A = h->ut_hl.as<float2>(); g.lda = na; g.sA = (long long)ns * na;
    g.B = h->KPhl.as<float2>(); g.ldb = na; g.transB = 1; g.sB = 0;
    g.C64 = h->RLp.as<double>(); g.ldc = P; g.sC = (long long)ns * P;
    RS_CK(df_gemm_w(h, g));
  } else if (P > 0) {
    GemmArgs g;
    g.M = ns; g.N = P; g.K = na; g.batch = 2;
    g.A = theta; g.lda = na; g.sA = (long long)ns * na;
    g.B = h->KP.as<double>(); g.ldb = na; g.transB = 1; g.sB = 0;
    g.C = h->RLp.as<double>(); g.ldc = P; g.sC = (long long)ns * P;
    RS_CK(gemm_p(h, RSSRI_PROF_FACTOR_GEMM, g));
  }
  if (P > 0) {
    for (int set = 0; set < 2; ++set)
      { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(scatter_pairs(h->RLp.as<double>() + (long long)set * ns * P, ns, P, h->pij.as<int>(),
                          nn, nn, fac + (2LL * set + 1) * ns * nn, s)); }
  }

  if (chain_df64) {
    SPAN(RSSRI_PROF_OTHER, 0.0);
    RS_CK(to_df64(fac, 4LL * ns * nn, h->facHl.as<float2>(), s, range_flag(h)));
  }

  // ---- learned control variate: coefficients, or statistics for training
  // c depends on the network and the setup's G, Sigma_DD and [K]^L only, not on
  // the draws: computed once per setup (or caller G) and parameter set
  h->pending_cv_c = false;
  if (use_cv && (!h->cv_c_ready || h->pending_block)) {
    RS_CK(cudaEventRecord(h->ev[6], s));
    RS_CK(cv_compute_c(h, G, Gb));
    RS_CK(cudaEventRecord(h->ev[7], s));
    h->cv_c_ready = true;
    h->pending_cv_c = true;
  }
  if (collect_stats) {
    RS_CK(ensure(h->cv_stats, (size_t)nt * 5 * nn * sizeof(double)));
    RS_CK(cudaMemsetAsync(h->cv_stats.p, 0, (size_t)nt * 5 * nn * sizeof(double), s));
  }

  // ---- S8: chains per tau and batch of sample pairs
  RS_CK(cudaMemsetAsync(h->e_st.p, 0, ns * sizeof(double), s));
  const double ne = 2.0 * h->n_occ;
  double *XG = h->XG.as<double>(), *Cc = h->Cc.as<double>(), *Bm = h->Bm.as<double>(),
         *BC = h->BC.as<double>();
  if (bf16) {
    RS_CK(chain_tc(h, tc_kind, ns, G, Gb, sdd, h->sig_raw.as<double>(), tc_err,
                   use_cv ? h->cv_c.as<double>() : nullptr));
  }
  for (int t = 0; t < nt && !bf16; ++t) {
    const double *Gt = G + t * nn, *Gbt = Gb + t * nn;
    double *sig = h->sig_raw.as<double>() + t * nn;
    for (int x0 = 0; x0 < ns; x0 += nb) {
      const int cnt = std::min(nb, ns - x0);
      // the batch is [kind][x]
      if (chain_df64) {
        // the same products on (hi, lo) pairs: X G and C = X G Y kept as pairs,
        // B = C Gb in fp64 for the fold
        const float2 *fh = h->facHl.as<float2>();
        const float2 *Gh = h->GGhl.as<float2>() + t * nn, *Gbh = h->GGhl.as<float2>() + (nt + t) * nn;
        for (int kind = 0; kind < nkind; ++kind) {
          const int xk = (kind == 0 || kind == 2) ? 0 : 1, yk = (kind == 0 || kind == 3) ? 0 : 1;
          const float2 *X = fh + ((0LL * 2 + xk) * ns + x0) * nn;
          const float2 *Y = fh + ((1LL * 2 + yk) * ns + x0) * nn;
          float2 *xg = h->xgHl.as<float2>() + (long long)kind * cnt * nn;
          float2 *c = h->cHl.as<float2>() + (long long)kind * cnt * nn;
          DfGemm g;
          g.M = n; g.N = n; g.K = n; g.batch = cnt;
          g.lda = g.ldb = g.ldc = n;
          g.A = X; g.sA = nn; g.B = Gh; g.sB = 0; g.C2 = xg; g.sC = nn;   // X G
          RS_CK(df_gemm_c(h, RSSRI_PROF_CHAIN_GEMM, g));
          g.A = xg; g.sA = nn; g.B = Y; g.sB = nn; g.C2 = c; g.sC = nn;   // C = X G Y
          RS_CK(df_gemm_c(h, RSSRI_PROF_CHAIN_GEMM, g));
          g.A = c; g.sA = nn; g.B = Gbh; g.sB = 0; g.C2 = nullptr;        // B = C Gb
          g.C64 = Bm + (long long)kind * cnt * nn; g.sC = nn;
          RS_CK(df_gemm_c(h, RSSRI_PROF_CHAIN_GEMM, g));
        }
      }
      for (int kind = 0; kind < nkind && !chain_df64; ++kind) {
        const int xk = (kind == 0 || kind == 2) ? 0 : 1, yk = (kind == 0 || kind == 3) ? 0 : 1;
        const double *X = fac + ((0LL * 2 + xk) * ns + x0) * nn;
        const double *Y = fac + ((1LL * 2 + yk) * ns + x0) * nn;
        double *xg = XG + (long long)kind * cnt * nn, *c = Cc + (long long)kind * cnt * nn,
               *bm = Bm + (long long)kind * cnt * nn;
        GemmArgs g;
        g.M = n; g.N = n; g.K = n; g.batch = cnt;
        g.lda = g.ldb = g.ldc = n;
        g.A = X; g.sA = nn; g.B = Gt; g.sB = 0; g.C = xg; g.sC = nn;   // X G
        RS_CK(gemm_p(h, RSSRI_PROF_CHAIN_GEMM, g));
        g.A = xg; g.sA = nn; g.B = Y; g.sB = nn; g.C = c; g.sC = nn;   // C = X G Y
        RS_CK(gemm_p(h, RSSRI_PROF_CHAIN_GEMM, g));
        g.A = c; g.sA = nn; g.B = Gbt; g.sB = 0; g.C = bm; g.sC = nn;  // B = C Gb
        RS_CK(gemm_p(h, RSSRI_PROF_CHAIN_GEMM, g));
      }
      const int tot = cnt * nkind;
      // t = Tr B, s2 = Tr B B, B <- +-(2 t I - B)
      { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(chain_fold(Bm, tot, literal ? 2 * cnt : cnt, n, h->tarr.as<double>(), h->sarr.as<double>(),
                                                      chain_df64 ? h->bHl.as<float2>() : nullptr, s)); }
      if (chain_df64) {
        DfGemm g;
        g.M = n; g.N = n; g.K = n; g.batch = tot;
        g.lda = g.ldb = g.ldc = n;
        g.A = h->bHl.as<float2>(); g.sA = nn; g.B = h->cHl.as<float2>(); g.sB = nn;
        g.C64 = BC; g.sC = nn;  // (2tI - B) C
        RS_CK(df_gemm_c(h, RSSRI_PROF_CHAIN_GEMM, g));
      } else {
        GemmArgs g;
        g.M = n; g.N = n; g.K = n; g.batch = tot;
        g.lda = g.ldb = g.ldc = n;
        g.A = Bm; g.sA = nn; g.B = Cc; g.sB = nn; g.C = BC; g.sC = nn;  // (2tI - B) C
        RS_CK(gemm_p(h, RSSRI_PROF_CHAIN_GEMM, g));
      }
      if (literal && P > 0)
        RS_CK(literal_cross(h, o, t, x0, cnt, Gt, Gbt, XG, Cc, Bm, BC));
      if (collect_stats) {
        SPAN(RSSRI_PROF_OTHER, 0.0);
        RS_CK(cv_stats(BC, cnt, n, h->cv_stats.as<double>() + (long long)t * 5 * nn, s));
      }
      if (use_cv) {
        SPAN(RSSRI_PROF_OTHER, 0.0);
        const double *ct = h->cv_c.as<double>() + t * nn;
        RS_CK(cv_accumulate(BC, cnt, n, (double)ns, sdd + t * nn, ct, x0 == 0,
                            sig, s));
        RS_CK(cv_pair_energy(BC, cnt, n, ct, Gbt, h->tarr.as<double>(), h->sarr.as<double>(),
                             h->h_tau_w[t], ne, h->e_st.as<double>() + x0, s));
      } else {
        { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(sigma_accumulate(BC, cnt, nkind, n, (double)ns, sdd + t * nn,
                               x0 == 0, sig, s)); }
        { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(pair_energy(h->tarr.as<double>(), h->sarr.as<double>(), cnt, nkind, literal ? 2 : 1, h->h_tau_w[t], ne,
                          h->e_st.as<double>() + x0, s)); }
      }
    }
  }
  // ---- S10 and S9
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(symmetrize(h->sig_raw.as<double>(), n, nt, h->sig_out.as<double>(), s)); }
  if (use_cv) {
    SPAN(RSSRI_PROF_OTHER, 0.0);
    RS_CK(trace_prod_w(sdd, Gb, h->cv_c.as<double>(), n, nt,
                       h->trdd.as<double>(), s));
  } else {
    SPAN(RSSRI_PROF_OTHER, 0.0);
    RS_CK(trace_prod(sdd, Gb, n, nt, h->trdd.as<double>(), s));
  }
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(trace_prod(h->sig_out.as<double>(), Gb, n, nt, h->tr.as<double>(), s)); }
  { SPAN(RSSRI_PROF_OTHER, 0.0); RS_CK(energy_finalize(h->tau_w, h->trdd.as<double>(), h->tr.as<double>(), nt, ne,
                        h->e_st.as<double>(), ns, h->e_pair.as<double>(), h->res.as<double>(), s)); }
  const cudaMemcpyKind dk = h->ptr_kind == RSSRI_PTR_HOST ? cudaMemcpyDeviceToHost
                                                          : cudaMemcpyDeviceToDevice;
  if (sigma) RS_CK(cudaMemcpyAsync(sigma, h->sig_out.p, nt * nn * sizeof(double), dk, s));
  if (e_pair) RS_CK(cudaMemcpyAsync(e_pair, h->e_pair.p, ns * sizeof(double), dk, s));
  RS_CK(cudaEventRecord(h->ev[4], s));
  RS_CK(cudaMemcpyAsync(h->host_res, h->res.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  RS_CK(cudaMemcpyAsync(reinterpret_cast<int *>(h->host_res + 4), tc_err, sizeof(int),
                        cudaMemcpyDeviceToHost, s));
  RS_CK(cudaMemcpyAsync(reinterpret_cast<int *>(h->host_res + 5), range_flag(h), sizeof(int),
                        cudaMemcpyDeviceToHost, s));
  RS_CK(cudaEventRecord(h->ev[5], s));
  h->pending = true;
  h->pending_tc = bf16;
  h->pending_ns = ns;
  return RSSRI_OK;
#undef RS_CK
}

// Waits for the enqueued call and returns its energies and statistics.
int finish_sigma(rssri_handle *h, double *e_corr, double *e_stderr, rssri_stats *st) {
  if (!h || !h->pending) return RSSRI_ERR_INVALID_ARG;
  h->pending = false;
  if (cudaSetDevice(h->device) != cudaSuccess) return RSSRI_ERR_CUDA;
  const cudaError_t e = cudaEventSynchronize(h->ev[5]);
  if (e != cudaSuccess) {
    const int r = map_err(e);
    if (r == RSSRI_ERR_CUDA) h->broken = true;
    return r;
  }
  const double *res = h->host_res;
  const int tc_flag = *reinterpret_cast<const int *>(h->host_res + 4);
  if (tc_flag) return RSSRI_ERR_TIMEOUT;
  if (*reinterpret_cast<const int *>(h->host_res + 5)) return RSSRI_ERR_RANGE;
  h->last_ns = h->pending_ns;
  h->have_sigma = true;
  float t_dd = 0, t_samp = 0;
  cudaEventElapsedTime(&t_dd, h->ev[2], h->ev[3]);
  cudaEventElapsedTime(&t_samp, h->ev[3], h->ev[4]);
  rssri_stats &S = h->stats;
  S.n_pairs_screened = h->P_s;
  S.nnz_eri_l = h->nnz_eri_l;
  S.n_pairs_large = h->P;
  S.nnz_k_l = h->nnz_k_l;
  S.k_l_max = h->k_l_max;
  S.metric_iterations = h->ns_iters;
  S.metric_residual = h->ns_resid;
  S.e_dd = res[0];
  S.e_corr = res[1];
  S.e_stderr = res[3];
  S.t_setup_ms = h->t_setup_ms;
  S.t_green_dd_ms = h->pending_block ? t_dd : 0.0;
  S.t_sample_ms = t_samp;
  float t_cv = 0;
  if (h->pending_cv_c) cudaEventElapsedTime(&t_cv, h->ev[6], h->ev[7]);
  S.t_cv_c_ms = t_cv;
  long long pl[RSSRI_PROF_NCLASS];
  double pm[RSSRI_PROF_NCLASS], pg[RSSRI_PROF_NCLASS], pt[RSSRI_PROF_NCLASS];
  collect(h, pl, pm, pg, pt);
  S.kernel_launches = 0;
  for (int c = 0; c < RSSRI_PROF_NCLASS; ++c) {
    S.prof_launches[c] = pl[c] + h->setup_launches[c];
    S.prof_ms[c] = pm[c] + h->setup_ms[c];
    S.prof_gflop[c] = pg[c] + h->setup_gflop[c];
    S.prof_tensor_gflop[c] = pt[c] + h->setup_tgflop[c];
    S.kernel_launches += S.prof_launches[c];
  }
  if (e_corr) *e_corr = res[1];
  if (e_stderr) *e_stderr = res[3];
  if (st) *st = S;
  if (!std::isfinite(res[1]) || !std::isfinite(res[3])) return RSSRI_ERR_NONFINITE;
  return RSSRI_OK;
}

int run_sigma(rssri_handle *h, const rssri_options *o, const double *g_in, const double *gb_in,
              double *sigma, double *e_pair, double *e_corr, double *e_stderr, rssri_stats *st,
              bool collect_stats = false) {
  const int rc = issue_sigma(h, o, g_in, gb_in, sigma, e_pair, collect_stats);
  if (rc) return rc;
  return finish_sigma(h, e_corr, e_stderr, st);
}

}  // namespace

extern "C" {

int rssri_sigma(rssri_handle *h, const rssri_options *o, double *sigma, double *e_pair,
                double *e_corr, double *e_stderr, rssri_stats *st) {
  return run_sigma(h, o, nullptr, nullptr, sigma, e_pair, e_corr, e_stderr, st);
}

int rssri_sigma_from_g(rssri_handle *h, const rssri_options *o, const double *g, const double *gb,
                       double *sigma, double *e_pair, double *e_corr, double *e_stderr,
                       rssri_stats *st) {
  if (!g || !gb) return RSSRI_ERR_INVALID_ARG;
  return run_sigma(h, o, g, gb, sigma, e_pair, e_corr, e_stderr, st);
}

int rssri_sigma_async(rssri_handle *h, const rssri_options *o, double *sigma, double *e_pair) {
  if (!sigma) return RSSRI_ERR_INVALID_ARG;
  return issue_sigma(h, o, nullptr, nullptr, sigma, e_pair, false);
}

int rssri_sigma_wait(rssri_handle *h, double *e_corr, double *e_stderr, rssri_stats *st) {
  return finish_sigma(h, e_corr, e_stderr, st);
}

int rssri_sigma_batch(rssri_handle *const *hs, int count, const rssri_options *o,
                      double *const *sigma, double *const *e_pair, double *e_corr,
                      double *e_stderr) {
  if (count < 0 || (count > 0 && (!hs || !sigma))) return RSSRI_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    for (int j = 0; j < i; ++j)
      if (hs[i] == hs[j]) return RSSRI_ERR_INVALID_ARG;
  int first = RSSRI_OK, issued = 0;
  for (; issued < count; ++issued) {
    const int rc = issue_sigma(hs[issued], o, nullptr, nullptr, sigma[issued],
                               e_pair ? e_pair[issued] : nullptr, false);
    if (rc) {
      first = rc;
      break;
    }
  }
  // every enqueued call is waited for, also after a failure
  for (int i = 0; i < issued; ++i) {
    const int rc = finish_sigma(hs[i], e_corr ? e_corr + i : nullptr,
                                e_stderr ? e_stderr + i : nullptr, nullptr);
    if (rc && first == RSSRI_OK) first = rc;
  }
  return first;
}

int rssri_cv_train(rssri_handle *h, const rssri_options *o, const float *init_params, int steps,
                   int batch, float lr, double *loss_before, double *loss_after) {
  if (!h || h->pending || !o || !init_params || steps < 0 || batch < 1 || batch > CV_CHUNK ||
      !(lr > 0.f))
    return RSSRI_ERR_INVALID_ARG;
  if (h->broken) return RSSRI_ERR_CUDA;
  if (!h->ready) return RSSRI_ERR_NOT_READY;
  rssri_options ot = *o;
  ot.cv = 0;
  int rc = run_sigma(h, &ot, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, true);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  const int n = h->n, nt = h->n_tau, ns = (int)o->n_s;
  const long long nn = (long long)n * n, total = nn * nt;
  const int E = (int)std::min<long long>(CV_CHUNK, total);
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
    return e == cudaSuccess;
  };
  const size_t pb = CV_NPARAM * sizeof(float);
  ck(ensure(h->cv_params, pb));
  ck(ensure(h->cv_m, pb));
  ck(ensure(h->cv_v, pb));
  ck(ensure(h->cv_grad, pb));
  ck(ensure(h->cv_X, total * CV_NFEAT * sizeof(float)));
  ck(ensure(h->cv_t, total * sizeof(float)));
  ck(ensure(h->cv_w, total * sizeof(float)));
  ck(ensure(h->cv_scr, (3 * nt + n + 1) * sizeof(double)));
  ck(ensure(h->cv_act, cv_act_floats(std::max(batch, E)) * sizeof(float)));
  ck(ensure(h->cv_work, cv_work_floats(std::max(batch, E)) * sizeof(float)));
  ck(ensure(h->cv_bx, (size_t)std::max(batch, E) * CV_NFEAT * sizeof(float)));
  ck(ensure(h->cv_bt, (size_t)std::max(batch, E) * sizeof(float)));
  ck(ensure(h->cv_bw, (size_t)std::max(batch, E) * sizeof(float)));
  ck(ensure(h->cv_loss, 4 * sizeof(float)));
  if (e != cudaSuccess) { note_error_site(__FILE__, __LINE__); return map_err(e); }
  float *P = h->cv_params.as<float>(), *X = h->cv_X.as<float>(), *T = h->cv_t.as<float>(),
        *Wt = h->cv_w.as<float>(), *act = h->cv_act.as<float>(), *work = h->cv_work.as<float>(),
        *bx = h->cv_bx.as<float>(), *bt = h->cv_bt.as<float>(), *bw = h->cv_bw.as<float>(),
        *grad = h->cv_grad.as<float>(), *loss = h->cv_loss.as<float>();
  ck(cv_features(h->sdd.as<double>(), h->G.as<double>(), h->Gb.as<double>(), h->tau, h->beta,
                 h->KP.as<double>(), h->rowptr.as<int>(), h->n_aux, n, nt,
                 h->cv_scr.as<double>(), X, s));
  ck(cv_targets(h->cv_stats.as<double>(), n, nt, ns, T, Wt, s));
  ck(cudaMemcpyAsync(P, init_params, pb, cudaMemcpyHostToDevice, s));
  ck(cudaMemsetAsync(h->cv_m.p, 0, pb, s));
  ck(cudaMemsetAsync(h->cv_v.p, 0, pb, s));
  // fixed evaluation set: the first E elements
  auto eval = [&](double *out) {
    ck(cv_forward(P, X, E, act, work, s));
    ck(cv_backward(P, X, E, T, Wt, act, grad, loss, work, s));
    float l = 0;
    ck(cudaMemcpyAsync(&l, loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    if (out) *out = l;
  };
  eval(loss_before);
  // minibatches: elements (start + k stride) mod total, stride coprime to total
  long long stride = 1000003 % total;
  if (stride < 1) stride = 1;
  auto gcd = [](long long a, long long b) {
    while (b) {
      const long long t2 = a % b;
      a = b;
      b = t2;
    }
    return a;
  };
  while (gcd(stride, total) != 1) ++stride;
  for (int step = 1; step <= steps && e == cudaSuccess; ++step) {
    const long long start = ((long long)(step - 1) * batch) % total;
    ck(cv_gather(X, CV_NFEAT, total, start, stride, batch, bx, s));
    ck(cv_gather(T, 1, total, start, stride, batch, bt, s));
    ck(cv_gather(Wt, 1, total, start, stride, batch, bw, s));
    ck(cv_forward(P, bx, batch, act, work, s));
    ck(cv_backward(P, bx, batch, bt, bw, act, grad, nullptr, work, s));
    ck(cv_adam(P, grad, h->cv_m.as<float>(), h->cv_v.as<float>(), (int)CV_NPARAM, lr, step, s));
  }
  eval(loss_after);
  if (e != cudaSuccess) { note_error_site(__FILE__, __LINE__); return map_err(e); }
  h->cv_ready = true;
  h->cv_c_ready = false;
  return RSSRI_OK;
}

int rssri_cv_set_params(rssri_handle *h, const float *params) {
  if (!h || h->pending || !params) return RSSRI_ERR_INVALID_ARG;
  if (h->broken) return RSSRI_ERR_CUDA;
  if (cudaSetDevice(h->device) != cudaSuccess) return RSSRI_ERR_CUDA;
  cudaError_t e = ensure(h->cv_params, CV_NPARAM * sizeof(float));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->cv_params.p, params, CV_NPARAM * sizeof(float), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) {
    h->cv_ready = true;
    h->cv_c_ready = false;
  }
  if (e != cudaSuccess) note_error_site(__FILE__, __LINE__);
  return map_err(e);
}

int rssri_cv_loss_grad(rssri_handle *h, const float *x, const float *target, const float *weight,
                       int m, const float *params, float *loss, float *grad) {
  if (!h || h->pending || !x || !target || !weight || !params || !loss || !grad || m < 1 ||
      m > CV_CHUNK)
    return RSSRI_ERR_INVALID_ARG;
  if (h->broken) return RSSRI_ERR_CUDA;
  if (cudaSetDevice(h->device) != cudaSuccess) return RSSRI_ERR_CUDA;
  cudaStream_t s = h->stream;
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t v) {
    if (e == cudaSuccess) e = v;
  };
  const size_t pb = CV_NPARAM * sizeof(float);
  ck(ensure(h->cv_ptmp, pb));
  ck(ensure(h->cv_grad, pb));
  ck(ensure(h->cv_act, std::max(h->cv_act.bytes, cv_act_floats(m) * sizeof(float))));
  ck(ensure(h->cv_work, std::max(h->cv_work.bytes, cv_work_floats(m) * sizeof(float))));
  ck(ensure(h->cv_bx, std::max(h->cv_bx.bytes, (size_t)m * CV_NFEAT * sizeof(float))));
  ck(ensure(h->cv_bt, std::max(h->cv_bt.bytes, (size_t)m * sizeof(float))));
  ck(ensure(h->cv_bw, std::max(h->cv_bw.bytes, (size_t)m * sizeof(float))));
  ck(ensure(h->cv_loss, 4 * sizeof(float)));
  if (e != cudaSuccess) { note_error_site(__FILE__, __LINE__); return map_err(e); }
  ck(cudaMemcpyAsync(h->cv_ptmp.p, params, pb, cudaMemcpyHostToDevice, s));
  ck(cudaMemcpyAsync(h->cv_bx.p, x, (size_t)m * CV_NFEAT * sizeof(float), cudaMemcpyHostToDevice, s));
  ck(cudaMemcpyAsync(h->cv_bt.p, target, (size_t)m * sizeof(float), cudaMemcpyHostToDevice, s));
  ck(cudaMemcpyAsync(h->cv_bw.p, weight, (size_t)m * sizeof(float), cudaMemcpyHostToDevice, s));
  ck(cv_forward(h->cv_ptmp.as<float>(), h->cv_bx.as<float>(), m, h->cv_act.as<float>(),
                h->cv_work.as<float>(), s));
  ck(cv_backward(h->cv_ptmp.as<float>(), h->cv_bx.as<float>(), m, h->cv_bt.as<float>(),
                 h->cv_bw.as<float>(), h->cv_act.as<float>(), h->cv_grad.as<float>(),
                 h->cv_loss.as<float>(), h->cv_work.as<float>(), s));
  ck(cudaMemcpyAsync(loss, h->cv_loss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
  ck(cudaMemcpyAsync(grad, h->cv_grad.p, pb, cudaMemcpyDeviceToHost, s));
  ck(cudaStreamSynchronize(s));
  if (e != cudaSuccess) note_error_site(__FILE__, __LINE__);
  return map_err(e);
}

int rssri_buffer_bytes(rssri_handle *h, int which, size_t *bytes) {
  if (!h || h->pending || !bytes) return RSSRI_ERR_INVALID_ARG;
  *bytes = 0;
  if (!h->ready) return RSSRI_ERR_NOT_READY;
  const size_t d = sizeof(double);
  const size_t nn = (size_t)h->n * h->n, na = h->n_aux, nt = h->n_tau, ns = h->last_ns;
  switch (which) {
    case RSSRI_BUF_W: *bytes = na * na * d; break;
    case RSSRI_BUF_COLMAX: *bytes = h->n * d; break;
    case RSSRI_BUF_ERI_L: *bytes = nn * na * d; break;
    case RSSRI_BUF_K_L: *bytes = nn * na * d; break;
    case RSSRI_BUF_THETA: *bytes = h->have_sigma ? 2 * ns * na * d : 0; break;
    case RSSRI_BUF_R:
    case RSSRI_BUF_R_L: *bytes = h->have_sigma ? 2 * ns * nn * d : 0; break;
    case RSSRI_BUF_G:
    case RSSRI_BUF_GB:
    case RSSRI_BUF_SIGMA_DD: *bytes = h->block_ok ? nt * nn * d : 0; break;
    case RSSRI_BUF_SIGMA_RAW: *bytes = h->have_sigma ? nt * nn * d : 0; break;
    case RSSRI_BUF_CV_PARAMS: *bytes = h->cv_ready ? CV_NPARAM * sizeof(float) : 0; break;
    case RSSRI_BUF_CV_C: *bytes = h->cv_c_ready ? nt * nn * d : 0; break;
    default: return RSSRI_ERR_INVALID_ARG;
  }
  return *bytes ? RSSRI_OK : RSSRI_ERR_NOT_READY;
}

int rssri_export(rssri_handle *h, int which, void *dst, size_t bytes, int dst_kind) {
  size_t need = 0;
  int rc = rssri_buffer_bytes(h, which, &need);
  if (rc) return rc;
  if (!dst || bytes != need || (dst_kind != RSSRI_PTR_DEVICE && dst_kind != RSSRI_PTR_HOST))
    return RSSRI_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return RSSRI_ERR_CUDA;
  cudaStream_t s = h->stream;
  const cudaMemcpyKind k = dst_kind == RSSRI_PTR_HOST ? cudaMemcpyDeviceToHost
                                                      : cudaMemcpyDeviceToDevice;
  const size_t nn = (size_t)h->n * h->n, na = h->n_aux, ns = h->last_ns;
  cudaError_t e = cudaSuccess;
  auto copy = [&](void *d, const void *src, size_t b) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, src, b, k, s);
  };
  char *out = static_cast<char *>(dst);
  switch (which) {
    case RSSRI_BUF_W: copy(dst, h->W.p, bytes); break;
    case RSSRI_BUF_COLMAX: copy(dst, h->colmax.p, bytes); break;
    case RSSRI_BUF_ERI_L:
    case RSSRI_BUF_K_L: {
      // dense [n][n][n_aux], zero outside the listed pairs
      const bool eri = which == RSSRI_BUF_ERI_L;
      const int P = eri ? h->P_s : h->P;
      const int *idx = eri ? h->spairs.as<int>() : h->pij.as<int>();
      const double *rows = eri ? h->EL.as<double>() : h->KP.as<double>();
      e = ensure(h->outbuf, bytes);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->outbuf.p, 0, bytes, s);
      if (e == cudaSuccess && P > 0) {
        // scatter rows: treat each row of n_aux doubles as one element of width na
        std::vector<int> hidx(P);
        e = cudaMemcpyAsync(hidx.data(), idx, P * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (int p = 0; p < P && e == cudaSuccess; ++p)
          e = cudaMemcpyAsync(h->outbuf.as<double>() + (size_t)hidx[p] * na, rows + (size_t)p * na,
                              na * sizeof(double), cudaMemcpyDeviceToDevice, s);
      }
      copy(dst, h->outbuf.p, bytes);
      break;
    }
    case RSSRI_BUF_THETA: copy(dst, h->theta.p, bytes); break;
    case RSSRI_BUF_R:
    case RSSRI_BUF_R_L: {
      const int kind = which == RSSRI_BUF_R ? 0 : 1;
      for (int set = 0; set < 2; ++set)
        copy(out + set * ns * nn * sizeof(double),
             h->fac.as<double>() + (2 * set + kind) * ns * nn, ns * nn * sizeof(double));
      break;
    }
    case RSSRI_BUF_G: copy(dst, h->G.p, bytes); break;
    case RSSRI_BUF_GB: copy(dst, h->Gb.p, bytes); break;
    case RSSRI_BUF_SIGMA_DD: copy(dst, h->sdd.p, bytes); break;
    case RSSRI_BUF_SIGMA_RAW: copy(dst, h->sig_raw.p, bytes); break;
    case RSSRI_BUF_CV_PARAMS: copy(dst, h->cv_params.p, bytes); break;
    case RSSRI_BUF_CV_C: copy(dst, h->cv_c.p, bytes); break;
    default: return RSSRI_ERR_INVALID_ARG;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) note_error_site(__FILE__, __LINE__);
  return map_err(e);
}

}  // extern "C"
