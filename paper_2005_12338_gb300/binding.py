"""ctypes binding of librssri (include/*.h): argument marshalling only.

Every computation runs in the CUDA library.  There is no CPU fallback: if the
library cannot be loaded, `lib()` raises.  The functions keep the C names;
`Handle` wraps them for callers holding torch CUDA tensors (device pointers)
or numpy arrays (host pointers).  torch supplies device memory and the
stream; no torch type crosses the C ABI.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# RSSRI_CHECKS=1: the build whose kernels check their own indices (see build.py)
LIB_PATH = os.path.join(HERE, "librssri_checks.so" if os.environ.get("RSSRI_CHECKS", "") == "1"
                        else "librssri.so")

RSSRI_PTR_DEVICE, RSSRI_PTR_HOST = 0, 1
RSSRI_EST_CV, RSSRI_EST_SRI, RSSRI_EST_LITERAL = 0, 1, 2
RSSRI_PREC_FP64, RSSRI_PREC_BF16, RSSRI_PREC_TF32, RSSRI_PREC_DF64 = 0, 1, 2, 3
RSSRI_DD_FP64, RSSRI_DD_DF64, RSSRI_DD_OZ = 0, 1, 2
BUF = dict(W=0, COLMAX=1, ERI_L=2, K_L=3, THETA=4, R=5, R_L=6, G=7, GB=8, SIGMA_DD=9,
           SIGMA_RAW=10, CV_PARAMS=11, CV_C=12)
RSSRI_CV_NPARAM = 134657
PROF_CLASSES = ["chain_gemm", "dd_spmm", "dd_gemm", "factor_gemm", "setup_gemm", "green", "other",
                "slice"]
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "NOT_SPD", -3: "NONSYMMETRIC_ERI", -4: "OOM",
          -5: "CUDA", -6: "TIMEOUT", -7: "NOT_READY", -8: "NONFINITE", -9: "RANGE"}


class rssri_problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_occ", C.c_int32), ("n_aux", C.c_int32),
                ("n_tau", C.c_int32), ("ptr_kind", C.c_int32), ("reserved0", C.c_int32),
                ("eri3", C.c_void_p), ("metric", C.c_void_p), ("orb_e", C.c_void_p),
                ("orb_c", C.c_void_p), ("tau", C.c_void_p), ("tau_w", C.c_void_p),
                ("mu", C.c_double), ("beta", C.c_double)]


class rssri_options(C.Structure):
    _fields_ = [("eps_prime", C.c_double), ("eps", C.c_double), ("n_s", C.c_int64),
                ("seed", C.c_uint64), ("xi_offset", C.c_int64), ("estimator", C.c_int32),
                ("precision", C.c_int32), ("pair_batch", C.c_int64), ("profile", C.c_int32),
                ("dd_arith", C.c_int32), ("cv", C.c_int32), ("test_wait_polls", C.c_int32),
                ("test_fail_alloc", C.c_int32), ("reserved0", C.c_int32)]


class rssri_stats(C.Structure):
    _fields_ = [("n_pairs_screened", C.c_int64), ("nnz_eri_l", C.c_int64),
                ("n_pairs_large", C.c_int64), ("nnz_k_l", C.c_int64), ("k_l_max", C.c_double),
                ("metric_iterations", C.c_int32), ("reserved0", C.c_int32),
                ("metric_residual", C.c_double), ("e_dd", C.c_double), ("e_corr", C.c_double),
                ("e_stderr", C.c_double), ("t_setup_ms", C.c_double),
                ("t_green_dd_ms", C.c_double), ("t_sample_ms", C.c_double),
                ("kernel_launches", C.c_int64), ("prof_launches", C.c_int64 * 8),
                ("prof_ms", C.c_double * 8), ("prof_gflop", C.c_double * 8),
                ("prof_tensor_gflop", C.c_double * 8), ("t_cv_c_ms", C.c_double)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            if k.startswith("reserved"):
                continue
            v = getattr(self, k)
            d[k] = list(v) if k.startswith("prof_") else v
        return d


_LIB = None

# name -> (restype, argtypes); every function declared in include/*.h
SIGNATURES = {
    "rssri_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "rssri_destroy": (None, [C.c_void_p]),
    "rssri_status_string": (C.c_char_p, [C.c_int]),
    "rssri_last_cuda_error": (C.c_char_p, []),
    "rssri_setup": (C.c_int, [C.c_void_p, C.POINTER(rssri_problem), C.POINTER(rssri_options)]),
    "rssri_sigma": (C.c_int, [C.c_void_p, C.POINTER(rssri_options), C.c_void_p, C.c_void_p,
                              C.POINTER(C.c_double), C.POINTER(C.c_double),
                              C.POINTER(rssri_stats)]),
    "rssri_sigma_from_g": (C.c_int, [C.c_void_p, C.POINTER(rssri_options), C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(rssri_stats)]),
    "rssri_sigma_async": (C.c_int, [C.c_void_p, C.POINTER(rssri_options), C.c_void_p,
                                    C.c_void_p]),
    "rssri_sigma_wait": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(rssri_stats)]),
    "rssri_sigma_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(rssri_options),
                                    C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "rssri_buffer_bytes": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_size_t)]),
    "rssri_export": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_int]),
    "rssri_energy_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                      C.c_int, C.c_void_p, C.c_void_p]),
    "rssri_cv_train": (C.c_int, [C.c_void_p, C.POINTER(rssri_options), C.c_void_p, C.c_int,
                                 C.c_int, C.c_float, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]),
    "rssri_cv_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rssri_cv_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_void_p, C.c_void_p, C.c_void_p]),
    # include/rssri_peak.h
    "rssri_peak_measure": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]),
}
RSSRI_PEAK_DFMA, RSSRI_PEAK_DMMA, RSSRI_PEAK_FFMA = 0, 1, 2
RSSRI_STATIC_MAX_TAU = 4096


def lib() -> C.CDLL:
    """Load librssri.so (built by `paper_2005_12338_gb300.build`)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2005_12338_gb300.build` "
                "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class RssriError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().rssri_status_string(code).decode()
        if code in (-4, -5):  # OOM, CUDA: name the runtime error
            msg += ": " + lib().rssri_last_cuda_error().decode()
        super().__init__(f"{where}: {STATUS.get(code, code)} ({msg})")
        self.code = code


def check(code: int, where: str):
    if code != 0:
        raise RssriError(code, where)


def _ptr(x):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be float64 and C-contiguous")
        return x.ctypes.data
    import torch  # device memory comes from torch
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("tensors must be float64 and contiguous")
        return x.data_ptr()
    raise TypeError(type(x))


class Handle:
    """One librssri handle on a CUDA device and stream (torch's current one by default)."""

    def __init__(self, device: int = 0, stream=None):
        self._h = C.c_void_p()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.device = device
        check(lib().rssri_create(C.byref(self._h), device, C.c_void_p(stream)), "rssri_create")
        self._keep = None
        self._pending = None
        self.kind = RSSRI_PTR_DEVICE
        self.n = self.n_tau = self.n_aux = 0

    def close(self):
        if self._h:
            lib().rssri_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def options(eps_prime=0.02, eps=1e-3, n_s=64, seed=0, xi_offset=0, estimator=RSSRI_EST_CV,
                pair_batch=0, profile=0, precision=RSSRI_PREC_FP64,
                dd_arith=RSSRI_DD_FP64, cv=0, test_wait_polls=0,
                test_fail_alloc=0) -> rssri_options:
        return rssri_options(eps_prime, eps, n_s, seed & ((1 << 64) - 1), xi_offset, estimator,
                             precision, pair_batch, profile, dd_arith, cv, test_wait_polls,
                             test_fail_alloc, 0)

    def setup(self, eri3, metric, orb_e, orb_c, tau, tau_w, n_occ: int, mu: float, beta: float,
              opts: rssri_options):
        """rssri_setup.  Arrays: all torch CUDA float64 tensors or all numpy float64."""
        host = isinstance(eri3, np.ndarray)
        n, _, n_aux = eri3.shape
        self.kind = RSSRI_PTR_HOST if host else RSSRI_PTR_DEVICE
        p = rssri_problem(n, n_occ, n_aux, int(tau.shape[0]), self.kind, 0,
                          _ptr(eri3), _ptr(metric), _ptr(orb_e), _ptr(orb_c), _ptr(tau),
                          _ptr(tau_w), float(mu), float(beta))
        self._keep = (eri3, metric, orb_e, orb_c, tau, tau_w)  # device arrays are referenced
        self.n, self.n_aux, self.n_tau = n, n_aux, int(tau.shape[0])
        check(lib().rssri_setup(self._h, C.byref(p), C.byref(opts)), "rssri_setup")

    def sigma(self, opts: rssri_options, sigma_out, e_pair_out=None, g=None, gb=None):
        """rssri_sigma (or rssri_sigma_from_g when g, gb are given).

        sigma_out: [n_tau][n][n] float64 (same memory kind as the problem).
        Returns (e_corr, e_stderr, stats dict)."""
        e = C.c_double()
        se = C.c_double()
        st = rssri_stats()
        if g is None:
            rc = lib().rssri_sigma(self._h, C.byref(opts), _ptr(sigma_out), _ptr(e_pair_out),
                                   C.byref(e), C.byref(se), C.byref(st))
            check(rc, "rssri_sigma")
        else:
            rc = lib().rssri_sigma_from_g(self._h, C.byref(opts), _ptr(g), _ptr(gb),
                                          _ptr(sigma_out), _ptr(e_pair_out), C.byref(e),
                                          C.byref(se), C.byref(st))
            check(rc, "rssri_sigma_from_g")
        return e.value, se.value, st.as_dict()

    def sigma_async(self, opts: rssri_options, sigma_out, e_pair_out=None):
        """rssri_sigma_async: enqueue and return; keep the outputs alive until sigma_wait."""
        self._pending = (opts, sigma_out, e_pair_out)
        check(lib().rssri_sigma_async(self._h, C.byref(opts), _ptr(sigma_out),
                                      _ptr(e_pair_out)), "rssri_sigma_async")

    def sigma_wait(self):
        """rssri_sigma_wait; returns (e_corr, e_stderr, stats dict)."""
        e, se, st = C.c_double(), C.c_double(), rssri_stats()
        rc = lib().rssri_sigma_wait(self._h, C.byref(e), C.byref(se), C.byref(st))
        self._pending = None
        check(rc, "rssri_sigma_wait")
        return e.value, se.value, st.as_dict()

    def cv_train(self, opts: rssri_options, init_params: np.ndarray, steps: int, batch: int,
                 lr: float):
        """rssri_cv_train; returns (loss_before, loss_after)."""
        p = np.ascontiguousarray(init_params, dtype=np.float32)
        if p.size != RSSRI_CV_NPARAM:
            raise ValueError("init_params must hold RSSRI_CV_NPARAM floats")
        a, b = C.c_double(), C.c_double()
        check(lib().rssri_cv_train(self._h, C.byref(opts), p.ctypes.data, steps, batch, lr,
                                   C.byref(a), C.byref(b)), "rssri_cv_train")
        return a.value, b.value

    def cv_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != RSSRI_CV_NPARAM:
            raise ValueError("params must hold RSSRI_CV_NPARAM floats")
        check(lib().rssri_cv_set_params(self._h, p.ctypes.data), "rssri_cv_set_params")

    def cv_loss_grad(self, x, target, weight, params):
        """rssri_cv_loss_grad on host float32 arrays; returns (loss, grad)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(target, dtype=np.float32)
        w = np.ascontiguousarray(weight, dtype=np.float32)
        p = np.ascontiguousarray(params, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        grad = np.zeros(RSSRI_CV_NPARAM, dtype=np.float32)
        check(lib().rssri_cv_loss_grad(self._h, x.ctypes.data, t.ctypes.data, w.ctypes.data,
                                       x.shape[0], p.ctypes.data, loss.ctypes.data,
                                       grad.ctypes.data), "rssri_cv_loss_grad")
        return float(loss[0]), grad

    def export(self, name: str) -> np.ndarray:
        """Copy an intermediate (rssri_export) to a host array (float32 for
        CV_PARAMS, float64 otherwise)."""
        which = BUF[name]
        nb = C.c_size_t()
        check(lib().rssri_buffer_bytes(self._h, which, C.byref(nb)), "rssri_buffer_bytes")
        if name == "CV_PARAMS":
            out = np.empty(nb.value // 4, dtype=np.float32)
            check(lib().rssri_export(self._h, which, out.ctypes.data, nb.value, RSSRI_PTR_HOST),
                  "rssri_export")
            return out
        out = np.empty(nb.value // 8, dtype=np.float64)
        check(lib().rssri_export(self._h, which, out.ctypes.data, nb.value, RSSRI_PTR_HOST),
              "rssri_export")
        return out


def peak_measure(which: int, device: int = 0):
    """rssri_peak_measure: (TFLOP/s, ms per launch) of an arithmetic pipe."""
    tf, ms = C.c_double(), C.c_double()
    check(lib().rssri_peak_measure(which, device, C.byref(tf), C.byref(ms)), "rssri_peak_measure")
    return tf.value, ms.value


def sigma_batch(handles, opts: rssri_options, sigmas, e_pairs=None):
    """rssri_sigma_batch over handles (each set up, each on its own stream);
    returns ([e_corr], [e_stderr])."""
    k = len(handles)
    hs = (C.c_void_p * k)(*[h._h.value for h in handles])
    sg = (C.c_void_p * k)(*[_ptr(x) for x in sigmas])
    ep = (C.c_void_p * k)(*[_ptr(x) for x in e_pairs]) if e_pairs is not None else None
    e = (C.c_double * k)()
    se = (C.c_double * k)()
    check(lib().rssri_sigma_batch(hs, k, C.byref(opts), sg, ep, e, se), "rssri_sigma_batch")
    return list(e), list(se)
