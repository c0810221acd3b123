// Element-wise kernels of the tensor-core chain (see chain_tc.cu).  Operand
// buffers hold the product kind's type (TcKind: bf16, or fp32 rounded to tf32).
#pragma once

#include "common.cuh"

namespace rssri {

// From fac = [set][kind R, R^L][x][n][n] fp64: xsl = [R^S; R^L] and
// y3 = [R'; R'^S; R'^L], each [ns][n][ldp] (zero columns n..ldp-1).
cudaError_t chain_factors(int kind, const double *fac, int ns, int n, int ldp, void *xsl,
                          void *y3, cudaStream_t s);
// dst[c][i][j] = src[c][i][j] in the operand type with row stride ldp (zero padding).
cudaError_t chain_matrices(int kind, const double *src, int cnt, int n, int ldp, void *dst,
                           cudaStream_t s);
// Per sample pair: traces, the energy increment (weight w, N_e = ne), and the
// operands of the final contraction: a6 = [2 dt I - X; 2 t^L I - Y],
// ct = (C^L + dC)^T, dct = dC^T, all [.][n][ldp].  part: scratch of
// ns * ceil(n/32) * 4 doubles.
// clt (may be null): (C^L)^T as well, the right operand of F^L = (2 t^L I - Y) C^L
// used by the learned control variate.
cudaError_t fold_tc(int kind, const float *xy, const float *dc, const float *cl, int ns, int n,
                    int ldp, double w, double ne, void *a6, void *ct, void *dct, void *clt,
                    double *e_st, double *part, cudaStream_t s);
// The learned control variate on the tensor-core chain (Eq. 25 with the large
// part weighted element-wise by c): with fl[x] = F(R^L, R'^L) of pair x (fp32),
//   sig += (1 - c) o (mean_x fl[x] - sdd)           (fixed order over x),
//   e_st[x] += -(w / ne) sum_ij (1 - c_ij) fl[x]_ij gb_ji.
cudaError_t cv_tc_apply(const float *fl, int ns, int n, const double *c, const double *sdd,
                        const double *gb, double w, double ne, double *sig, double *e_st,
                        cudaStream_t s);
// sig = base + (sum over groups of part) / ns, groups summed in order in fp64.
cudaError_t reduce_tc(const float *part, int groups, int n, const double *base, double ns,
                      double *sig, cudaStream_t s);

}  // namespace rssri
