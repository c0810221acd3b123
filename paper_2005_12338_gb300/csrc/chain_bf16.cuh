// Element-wise kernels of the bf16 tensor-core chain (see chain_bf16.cu).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace rssri {

// From fac = [set][kind R, R^L][x][n][n] fp64: xsl = [R^S; R^L] and
// y3 = [R'; R'^S; R'^L], each [ns][n][ldp] bf16 (zero columns n..ldp-1).
cudaError_t bf16_factors(const double *fac, int ns, int n, int ldp, __nv_bfloat16 *xsl,
                         __nv_bfloat16 *y3, cudaStream_t s);
// dst[c][i][j] = bf16(src[c][i][j]) with row stride ldp (zero padding).
cudaError_t bf16_matrices(const double *src, int cnt, int n, int ldp, __nv_bfloat16 *dst,
                          cudaStream_t s);
// Per sample pair: traces, the energy increment (weight w, N_e = ne), and the
// bf16 operands of the final contraction: a6 = [2 dt I - X; 2 t^L I - Y],
// ct = (C^L + dC)^T, dct = dC^T, all [.][n][ldp].  part: scratch of
// ns * ceil(n/32) * 4 doubles.
cudaError_t fold_bf16(const float *xy, const float *dc, const float *cl, int ns, int n, int ldp,
                      double w, double ne, __nv_bfloat16 *a6, __nv_bfloat16 *ct,
                      __nv_bfloat16 *dct, double *e_st, double *part, cudaStream_t s);
// sig = base + (sum over groups of part) / ns, groups summed in order in fp64.
cudaError_t reduce_bf16(const float *part, int groups, int n, const double *base, double ns,
                        double *sig, cudaStream_t s);

}  // namespace rssri
