// Launchers of the non-GEMM kernels of librssri (one per step of the path).
#pragma once

#include "common.cuh"

namespace rssri {

// ------------------------------------------------------------ S1 helpers --
// c = max_i sum_j |V_ij| (an upper bound of the largest eigenvalue);
// Y = V / c, Z = I.  scal[0] receives c.
cudaError_t ns_init(const double *V, int na, double *Y, double *Z, double *scal,
                    double *part, cudaStream_t s);
// T = (3 I - P) / 2 and scal[1] = max |P - I|.
cudaError_t ns_tbuild(const double *P, int na, double *T, double *scal, double *part,
                      cudaStream_t s);
// W = (Z + Z^T) / (2 sqrt(c)), c = scal[0].
cudaError_t ns_finish(const double *Z, int na, const double *scal, double *W, cudaStream_t s);

// ------------------------------------------------------------ S2: screen --
// flags[0] |= 1 if (ij|A) != (ji|A) somewhere; flags[1] |= 1 on NaN/Inf.
cudaError_t eri_check(const double *eri3, int n, int naux, int *flags, cudaStream_t s);
// colmax[j] = max_{i,A} |(ij|A)| (row j of the symmetric tensor).
cudaError_t eri_colmax(const double *eri3, int n, int naux, double *colmax, cudaStream_t s);
// cnt[i*n+j] = #{A : |(ij|A)| >= (eps'/n) min(M_i, M_j)}.
cudaError_t eri_pair_count(const double *eri3, int n, int naux, const double *colmax,
                           double eps_prime, int *cnt, cudaStream_t s);
// Rows of (ij|A)^L for the listed pairs (linear index i*n+j), zeros below threshold.
cudaError_t eri_gather_rows(const double *eri3, int n, int naux, const double *colmax,
                            double eps_prime, const int *pairs, int P, double *out,
                            cudaStream_t s);

// Stream compaction: idx = ascending positions with cnt[pos] > 0, out[0] = how
// many (int), sum64[0] = sum of cnt (long long).  scratch >= compact_scratch(len).
size_t compact_scratch_bytes(int len);
cudaError_t compact(const int *cnt, int len, int *idx, int *count, long long *sum64,
                    void *scratch, cudaStream_t s);

// ---------------------------------------------------------------- S3 ------
// out[0] = max |x| over len elements (exact; order-independent).
cudaError_t absmax(const double *x, long long len, double *out, double *part, cudaStream_t s);
// Zero entries of the P x naux rows with |x| < eps * kmax[0]; cnt[p] = non-zeros left.
cudaError_t kl_cut(double *rows, int P, int naux, const double *kmax, double eps, int *cnt,
                   cudaStream_t s);
// dst[r][:] = src[idx[r]][:] (row length ncols).
cudaError_t gather_rows(const double *src, const int *idx, int P, int ncols, double *dst,
                        cudaStream_t s);
// dst[r] = vals[idx[r]]
cudaError_t gather_int(const int *vals, const int *idx, int P, int *dst, cudaStream_t s);
// From sorted linear pair indices ij = i*n+j: row pointers (n+1), row and column of each pair.
cudaError_t pair_csr(const int *pair_ij, int P, int n, int *rowptr, int *prow, int *pcol,
                     cudaStream_t s);
// dst (ns x n*n, pre-zeroed) [x][pair_ij[p]] = src[x][p]
cudaError_t scatter_pairs(const double *src, int ns, int P, const int *pair_ij, long long nn,
                          long long dst_stride, double *dst, cudaStream_t s);

// ---------------------------------------------------------------- S4 ------
// theta[x][q] = +-1 from SplitMix64(seed ^ (set<<60 | (xi_offset+x)<<20 | q)).
cudaError_t rademacher(unsigned long long seed, int set, long long xi_offset, int ns, int naux,
                       double *theta, cudaStream_t s);

// ---------------------------------------------------------------- S6 ------
// cs[t][i][a] = C[i][off+a] * exp(sign * (e[off+a] - mu) * tau[t]), a < m.
cudaError_t green_scale(const double *C, const double *e, int n, int off, int m, double mu,
                        const double *tau, int ntau, int sign, double *cs, cudaStream_t s);

// ---------------------------------------------------------------- S7 ------
// T[m][q][j] = sum_{a in row m} sum_{b in row j} D[a*P+b] * At[(col[a]*n+col[b])*naux+q]
cudaError_t dd_exchange_spmm(const int *rowptr, const int *pcol, const double *D, int P,
                             const double *At, int n, int naux, double *T, cudaStream_t s);
// T[m][q][pcol[a]] -= 2 L[a][q] for every kept pair a = (m, pcol[a]).
cudaError_t dd_fold_direct(const int *prow, const int *pcol, const double *L, int P, int n,
                           int naux, double *T, cudaStream_t s);

// ---------------------------------------------------------------- S8 ------
// Per batch entry b (n x n): t[b] = Tr B, s2[b] = Tr(B B), then
// B <- sgn (2 t I - B) with sgn = +1 for b < npos, -1 otherwise; when Bhl is
// given the result goes there as (hi, lo) float pairs and B is left as is.
cudaError_t chain_fold(double *Bm, int nb, int npos, int n, double *t, double *s2,
                       float2 *Bhl, cudaStream_t s);
// sig[i][j] (+)= sum_x sum_{k < nkind} BC[k nh + x][i][j] / ns_div;
// init: sig = base + ..., else sig += ...
cudaError_t sigma_accumulate(const double *BC, int nh, int nkind, int n, double ns_div,
                             const double *base, int init, double *sig, cudaStream_t s);
// e_st[x] += -w * ((2 t[x]^2 - s2[x]) - (2 t[nh+x]^2 - s2[nh+x])) / ne (second if has_l).
// e_st[x] += -(w/ne) sum_k (+-)(2 t[k][x]^2 - s2[k][x]), kinds k < kpos with +.
cudaError_t pair_energy(const double *t, const double *s2, int nh, int nkind, int kpos, double w,
                        double ne, double *e_st, cudaStream_t s);
// Literal estimator helpers.  out[e][s] = in[s][e] (e < nn, s < S).
cudaError_t lit_qfast(const double *in, int S, long long nn, double *out, cudaStream_t s);
// W[s][m][j] = -Tk[m][s][j] + 2 JP[a][s] at the kept pairs a = (m, j).
cudaError_t lit_w(const double *Tk, int S, int n, const double *JP, const int *pij, int P,
                  double *W, cudaStream_t s);
// F0[x] += Z[0][x] - Z[1][x] + Z[2][x] - Z[3][x]; e_st[x] += -w Tr(that Gb) / ne.
cudaError_t lit_add(const double *Z, int cnt, int n, const double *Gb, double w, double ne,
                    double *F0, double *e_st, cudaStream_t s);

// ---------------------------------------------------------------- S9 ------
// out[t] = sum_ij X[t][i][j] Y[t][j][i]
cudaError_t trace_prod(const double *X, const double *Y, int n, int ntau, double *out,
                       cudaStream_t s);
// e_dd = -sum_t w_t trdd[t] / ne, e = -sum_t w_t tr[t] / ne, e_pair[x] = e_dd + e_st[x],
// res = {e_dd, e, mean(e_pair), std(e_pair)/sqrt(ns)}.
cudaError_t energy_finalize(const double *tau_w, const double *trdd, const double *tr, int ntau,
                            double ne, const double *e_st, int ns, double *e_pair, double *res,
                            cudaStream_t s);

// --------------------------------------------------------------- S10 ------
cudaError_t symmetrize(const double *in, int n, int ntau, double *out, cudaStream_t s);

// -------------------------------------------------------------- misc ------
cudaError_t nonfinite_check(const double *x, long long len, int *flag, cudaStream_t s);

}  // namespace rssri
