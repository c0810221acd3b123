// Learned control variate kernels (see cv_mlp.cu).
#pragma once

#include <algorithm>

#include "common.cuh"

namespace rssri {

constexpr int CV_NFEAT = 10, CV_HIDDEN = 256;
constexpr long long CV_NPARAM =
    (long long)CV_HIDDEN * CV_NFEAT + CV_HIDDEN + 2LL * (CV_HIDDEN * CV_HIDDEN + CV_HIDDEN) +
    CV_HIDDEN + 1;

// fp32 C = alpha op(A) op(B) + beta C; work (may be null) of sgemm_work_floats
// floats enables a split over K with a fixed-order reduction.
size_t sgemm_work_floats(int M, int N, int K);
cudaError_t sgemm(int M, int N, int K, const float *A, long long lda, int ta, const float *B,
                  long long ldb, int tb, float *C, long long ldc, float alpha, float beta,
                  float *work, cudaStream_t s);

// Activations of m rows: [Z0 A0 Z1 A1 Z2 A2] (m x 256 each), y (m), dy (m),
// then the bf16 operands of the tensor-core hidden layers.
size_t cv_act_floats(int m);
// Floats of `work` that the tensor-core hidden layers use (bf16 weights and
// weight-gradient partials); the fp32 products' split-K scratch follows them.
size_t cv_tc_work_floats();
// Forward: y = MLP(X) - 1 in act (see cv_act_floats), X [m][10].
cudaError_t cv_forward(const float *params, const float *X, int m, float *act, float *work,
                       cudaStream_t s);
// After cv_forward: loss = sum w (1 + y - t)^2 / sum w and its gradient.
cudaError_t cv_backward(const float *params, const float *X, int m, const float *target,
                        const float *weight, float *act, float *grad, float *loss, float *work,
                        cudaStream_t s);
cudaError_t cv_adam(float *p, const float *g, float *m, float *v, int n, float lr, int step,
                    cudaStream_t s);
// stats [5][n*n] += sums over the pair batch of F, F^L, F^2, (F^L)^2, F F^L.
cudaError_t cv_stats(const double *BC, int nh, int n, double *stats, cudaStream_t s);
// target c* and weight Var(F^L) per (tau, i, j) from stats [nt][5][n*n].
cudaError_t cv_targets(const double *stats, int n, int nt, int ns, float *target, float *weight,
                       cudaStream_t s);
// Feature rows X [nt*n*n][10]; scratch of 3*nt + n + 1 doubles.
cudaError_t cv_features(const double *sdd, const double *G, const double *Gb, const double *tau,
                        double beta, const double *KP, const int *rowptr, int naux, int n, int nt,
                        double *scratch, float *X, cudaStream_t s);
// dst[k] = src[(start + k stride) mod total] (rows of `cols` floats), k < m.
cudaError_t cv_gather(const float *src, int cols, long long total, long long start,
                      long long stride, int m, float *dst, cudaStream_t s);
// sig = (init ? c o base : sig) + sum_x (BC[x] + c o BC[nh+x]) / ns.
cudaError_t cv_accumulate(const double *BC, int nh, int n, double ns, const double *base,
                          const double *c, int init, double *sig, cudaStream_t s);
// e_st[x] += -w ((2 t_x^2 - s2_x) - Tr((c o F^L_x) Gb)) / ne with BC[nh+x] = -F^L_x.
cudaError_t cv_pair_energy(const double *BC, int nh, int n, const double *c, const double *gb,
                           const double *t, const double *s2, double w, double ne, double *e_st,
                           cudaStream_t s);
// out[t] = sum_ij W[t][i][j] X[t][i][j] Y[t][j][i]
cudaError_t trace_prod_w(const double *X, const double *Y, const double *W, int n, int nt,
                         double *out, cudaStream_t s);
// c = 1 + y in fp64.
cudaError_t cv_coefficients(const float *y, long long m, double *c, cudaStream_t s);

}  // namespace rssri
