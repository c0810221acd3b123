"""Learned control variate for the RS-SRI estimator, plain fp64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The deterministic large part of Eq. 25 gives a control variate with an
exactly known mean: for independent theta, theta',
E[F(R^L, R'^L)] = Sigma_DD (Eq. 20 on v^L = sum_Q [K^Q]^L [K^Q]^L).  Hence for
any coefficient matrix c(tau) chosen independently of the draws it is used
with,

    Sigma_c = mean_xi F(R, R') - c o (mean_xi F(R^L, R'^L) - Sigma_DD)

is an unbiased estimate of the RI self-energy (o: element-wise product);
c = 1 is the default estimator.  Per element the variance is smallest at
c* = Cov(F, F^L) / Var(F^L).  A small MLP predicts c from orbital-pair
features; it is fitted, on an independent training run, by minimising the
weighted squared distance to c* with weights Var(F^L), which is the
estimator's variance up to a constant.

Features of element (i, j) at tau (all dimensionless):
  0 |i - j| / N
  1 ln(tau) / ln(beta)
  2 Sigma_DD_ij(tau) / max |Sigma_DD(tau)|
  3 G_ii(tau) / max_k |G_kk(tau)|,      4 G_jj(tau) / same
  5 Gb_ii(tau) / max_k |Gb_kk(tau)|,    6 Gb_jj(tau) / same
  7 r_i / max r,  8 r_j / max r,  r_i = Frobenius norm of [K^L]_{i, :, :}
  9 1 if i == j else 0
Network: 10 -> 256 -> 256 -> 256 -> 1, SiLU activations, output c = 1 + y.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 10
HIDDEN = 256


def cv_sigma(f_sum, fl_sum, n_s, sigma_dd, c):
    """Sigma_c from the sums over samples of F and F^L (one tau point)."""
    return f_sum / n_s - c * (fl_sum / n_s - sigma_dd)


def cv_optimal(f, fl):
    """Per-element c* = Cov(F, F^L) / Var(F^L) and Var(F^L) from samples
    f, fl of shape [N_s, ...]."""
    n = f.shape[0]
    mf, ml = f.mean(0), fl.mean(0)
    cov = ((f - mf) * (fl - ml)).sum(0) / (n - 1)
    var = ((fl - ml) ** 2).sum(0) / (n - 1)
    c = np.where(var > 0, cov / np.where(var > 0, var, 1.0), 1.0)
    return c, var


def features(sigma_dd, g, gb, tau, beta, row_norm):
    """Feature rows [N*N, 10] for one tau point (element (i, j) at row i*N + j)."""
    n = g.shape[0]
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    dg, dgb = np.diag(g), np.diag(gb)
    sdd_max = np.abs(sigma_dd).max()
    gmax, gbmax, rmax = np.abs(dg).max(), np.abs(dgb).max(), row_norm.max()
    f = np.empty((n, n, N_FEAT))
    f[..., 0] = np.abs(i - j) / n
    f[..., 1] = np.log(tau) / np.log(beta)
    f[..., 2] = sigma_dd / sdd_max if sdd_max > 0 else 0.0
    f[..., 3] = dg[i] / gmax
    f[..., 4] = dg[j] / gmax
    f[..., 5] = dgb[i] / gbmax
    f[..., 6] = dgb[j] / gbmax
    f[..., 7] = row_norm[i] / rmax if rmax > 0 else 0.0
    f[..., 8] = row_norm[j] / rmax if rmax > 0 else 0.0
    f[..., 9] = (i == j).astype(float)
    return f.reshape(n * n, N_FEAT)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def mlp_forward(params, x):
    """params: list of (W [out, in], b [out]); returns (c, cache)."""
    a = x
    cache = []
    for k, (w, b) in enumerate(params):
        z = a @ w.T + b
        cache.append((a, z))
        a = silu(z) if k < len(params) - 1 else z
    return 1.0 + a[:, 0], cache


def mlp_loss_grad(params, x, target, weight):
    """Loss sum(w (c - c*)^2) / sum(w) and its gradient by backpropagation."""
    c, cache = mlp_forward(params, x)
    sw = weight.sum()
    loss = float((weight * (c - target) ** 2).sum() / sw)
    d = (2.0 * weight * (c - target) / sw)[:, None]  # dL/dy, y = c - 1
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        a, z = cache[k]
        dz = d if k == len(params) - 1 else d * silu_grad(z)
        grads[k] = (dz.T @ a, dz.sum(0))
        d = dz @ params[k][0]
    return loss, grads


def init_params(seed: int = 0):
    """He-style initialisation of the hidden layers; zero output layer (c = 1)."""
    rng = np.random.default_rng(seed)
    sizes = [N_FEAT, HIDDEN, HIDDEN, HIDDEN, 1]
    params = []
    for k in range(4):
        fan_in = sizes[k]
        w = rng.standard_normal((sizes[k + 1], fan_in)) * np.sqrt(2.0 / fan_in)
        if k == 3:
            w[:] = 0.0
        params.append((w, np.zeros(sizes[k + 1])))
    return params
