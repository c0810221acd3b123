"""Benchmark of the RS-SRI-GF2 self-energy path on GB300.

Workload: N = 200 basis functions, 100 occupied, N_aux = 600, 64 tau points,
N_s = 300 sample pairs, eps = 1e-3, eps' = 0.02 (synthetic hydrogen-chain-like
integrals).  One step is one pass of the whole path for a new seed:
rssri_setup (V^{-1/2}, screening, [K]^L and its cut, the pair-space product,
G(tau) and the deterministic block for every tau) and rssri_sigma (the
Rademacher draws, R and R^L, the chain products for every (sample pair, tau)
unit, the energy and the symmetrised output).  The metric is Sigma(tau) units
per second, a unit being one (sample pair, tau point); inputs are resident in
HBM when the timed region starts.

The benchmark line times the plain form: every product in IEEE fp64.  Beside
it (extra): the chosen form (the deterministic block's products as
fp64-accurate sliced products on the bf16 tensor cores, the stochastic chain
in bf16 on the tensor cores), its error against the plain form on the same
draws, and the time of each form to reach a 1 mEh standard error of E_corr;
the double-float form; the range-separated estimator against plain stochastic
RI at the same N_s.

Multi-GPU: one process per GPU (torchrun); every rank runs independent
replicas with its own seeds, no collective on the data path (weak scaling).

--impl reference times the fp64 CPU oracle on the host cores on a bounded
sample of the same workload, extrapolated to the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2005_12338_gb300 import replicas, synth  # noqa: E402

WORKLOAD = "c2_n200"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# (chain precision, deterministic-block arithmetic) of the forms
FORMS = {"plain": ("fp64", "fp64"), "chosen": ("bf16", "oz"), "df64": ("df64", "df64")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.CONFIGS))
    ap.add_argument("--form", default="plain", choices=sorted(FORMS),
                    help="the form on the benchmark line: plain (IEEE fp64 products), chosen "
                         "(sliced fp64-accurate block on the tensor cores + bf16 chain) or df64 "
                         "(double-float products)")
    ap.add_argument("--no-compare", action="store_true",
                    help="time only the form on the benchmark line")
    ap.add_argument("--eps", type=float, default=None,
                    help="override the K^L cut eps of the workload (e.g. the paper's 0.1)")
    ap.add_argument("--n-tau", type=int, default=None,
                    help="override the number of tau points of the workload (for one-off "
                         "measurements on the largest workload; not the benchmark line)")
    ap.add_argument("--no-cv", action="store_true",
                    help="skip the learned control variate report (training on an independent "
                         "run, then the chosen form with and without it on the same draws)")
    ap.add_argument("--literal", action="store_true",
                    help="also run the literal Eq. 25 estimator (fp64 chain, exact-D cross "
                         "terms) on the first timed seed and report its cost and stderr")
    ap.add_argument("--many", type=int, default=0,
                    help="also time K independent chains of uneven size (N from 64 to 256) "
                         "one by one and batched on K streams (rssri_sigma_batch)")
    ap.add_argument("--c4", type=int, default=0, metavar="K",
                    help="instead of the benchmark line, run the many-chain workload: the "
                         "first K of its 64 chains (N 100..800, N_aux 3N, 64 tau, 200 pairs), "
                         "each set up and sampled in turn in --form, and print its own line")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


# --------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": num(rows[0][2]), "reasons": reasons,
                "power_w_median": float(np.median(pw)) if pw else None, "samples": len(rows)}


# ---------------------------------------------------------- the oracle -----
def oracle_sample(s, cfg, seed, budget_s=12.0):
    """Time the fp64 oracle on a bounded sample of one step and extrapolate.

    The sample: the whole setup (V^{-1/2}, screen, [K]^L); R and R^L for two
    sample pairs; the chain products of those pairs at two tau points; the
    deterministic block at one tau point restricted to a few first-index
    auxiliary functions; G at one tau point.  Each part is scaled by how many
    times a full step repeats it."""
    import oracle as O
    n_s, nt = cfg["n_s"], s.n_tau
    t0 = time.perf_counter()
    w = O.metric_inv_sqrt(s.metric)
    el, _, _ = O.screen(s.eri3, cfg["eps_prime"])
    kl, _ = O.large_factor(el, w, cfg["eps"])
    t_setup = time.perf_counter() - t0
    n_pair = 2
    t0 = time.perf_counter()
    th0 = O.rademacher(seed, 0, n_pair, s.n_aux)
    th1 = O.rademacher(seed, 1, n_pair, s.n_aux)
    r0, rl0 = O.stochastic_factors(s.eri3, w, kl, th0)
    r1, rl1 = O.stochastic_factors(s.eri3, w, kl, th1)
    t_r = (time.perf_counter() - t0) / n_pair
    taus = [0, nt - 1]
    t_g = t_chain = 0.0
    units = 0
    for it in taus:
        t0 = time.perf_counter()
        g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[it])
        t_g += time.perf_counter() - t0
        t0 = time.perf_counter()
        for x in range(n_pair):
            O.factor_pair(r0[x], r1[x], g, gb)
            O.factor_pair(rl0[x], rl1[x], g, gb)
            units += 1
        t_chain += time.perf_counter() - t0
    t_g /= len(taus)
    t_unit = t_chain / units
    nq = int((np.abs(kl).reshape(-1, s.n_aux).max(axis=0) > 0).sum())
    n_outer = 1
    t0 = time.perf_counter()
    g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[nt // 2])
    while True:
        O.sigma_from_factor(kl, g, gb, outer=range(n_outer))
        el_t = time.perf_counter() - t0
        if el_t > budget_s / 3 or n_outer >= nq:
            break
        n_outer *= 2
        t0 = time.perf_counter()
    t_dd_tau = el_t / n_outer * nq
    t_step = t_setup + t_r * n_s + t_g * nt + t_unit * n_s * nt + t_dd_tau * nt
    units_step = n_s * nt
    try:
        import threadpoolctl
        threads = max(i.get("num_threads", 1) for i in threadpoolctl.threadpool_info())
    except Exception:
        threads = int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"oracle timed on: full setup; R/R^L for {n_pair} sample pairs; chain products "
              f"for {units} (pair, tau) units; G at {len(taus)} tau; deterministic block at 1 tau "
              f"over {n_outer} of {nq} first-index aux functions; extrapolated to one step "
              f"({n_s} pairs x {nt} tau)")
    return dict(value=units_step / t_step, unit="units/s", cores=threads, kind="oracle",
                sample=sample, t_step_extrapolated_s=t_step,
                parts_s=dict(setup=t_setup, r_per_pair=t_r, green_per_tau=t_g,
                             chain_per_unit=t_unit, dd_per_tau=t_dd_tau))


def time_to_target(results, ns, target):
    """Device time to reach a target E_corr standard error: the fixed part
    (setup, G, deterministic block) once, then sample pairs at the measured
    cost per pair until sd(e_pair)/sqrt(n) <= target (at least 2 pairs)."""
    fixed = float(np.mean([r[2] for r in results])) / 1e3
    per_pair = float(np.mean([r[3] for r in results])) / 1e3 / ns
    sigma_pair = float(np.mean([r[1] for r in results])) * np.sqrt(ns)
    pairs = max(2.0, (sigma_pair / target) ** 2)
    return {"seconds": fixed + per_pair * pairs, "sampling_only_s": per_pair * pairs,
            "fixed_s": fixed, "per_pair_s": per_pair,
            "pairs_needed": pairs, "sd_per_pair": sigma_pair, "target": target}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfg = synth.CONFIGS[args.workload]
    s = synth.make_system(cfg["n"], cfg["n_occ"], cfg["n_aux"], cfg["n_tau"], input_seed=0)
    for k in range(args.warmup):
        oracle_sample(s, cfg, 10_000 + k, budget_s=6.0)
    vals, times = [], []
    for k in range(args.steps):
        r = oracle_sample(s, cfg, k, budget_s=6.0)
        vals.append(r["value"])
        times.append(r["t_step_extrapolated_s"])
    value = float(np.mean(vals))
    line = {"metric": "Sigma(tau) units/s (unit = one sample pair x one tau point)",
            "value": value, "unit": "units/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(times)) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: N={cfg['n']} n_occ={cfg['n_occ']} "
                                   f"N_aux={cfg['n_aux']} N_tau={cfg['n_tau']} N_s={cfg['n_s']} "
                                   f"eps={cfg['eps']} eps'={cfg['eps_prime']}"},
            "cpu_baseline": {"value": value, "unit": "units/s", "cores": r["cores"],
                             "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": value, "unit": "units/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- our arm -----
def traffic_for(cls, form):
    """Per-launch DRAM bytes of the dominant kernel class of a form from the
    committed ncu summary (profiles/traffic.json, keyed "form/class"), or None
    if absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(f"{form}/{cls}")
    if not d:
        return None
    src = os.path.join(ROOT, "paper_2005_12338_gb300", "csrc", d["source"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return d["bytes_per_launch"] if sha == d.get("source_sha") else None


def many_systems(args, binding, torch, prec, dd):
    """K independent chains of uneven size, each with its own handle and
    stream: the sampling calls (S4-S10) timed one after another and then all
    enqueued at once through rssri_sigma_batch.  Setups are done beforehand."""
    m = dict(synth.MANY, k=args.many)
    sizes = synth.many_sizes(m["k"], m["n_min"], m["n_max"])
    hs, outs, units = [], [], 0
    opts = binding.Handle.options(m["eps_prime"], m["eps"], m["n_s"], 5, precision=prec,
                                  dd_arith=dd)
    for k, n in enumerate(sizes):
        s = synth.make_system(n, n // 2, 3 * n, m["n_tau"], input_seed=k)
        st = torch.cuda.Stream()
        h = binding.Handle(torch.cuda.current_device(), stream=st.cuda_stream)
        dev = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                     s.tau_w)]
        torch.cuda.synchronize()
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
        hs.append((h, dev, st))
        outs.append(torch.empty((m["n_tau"], n, n), dtype=torch.float64, device="cuda"))
        units += m["n_s"] * m["n_tau"]

    def one_by_one():
        for (h, _, _), o in zip(hs, outs):
            h.sigma(opts, o)

    def batched():
        binding.sigma_batch([x[0] for x in hs], opts, outs)

    res = {}
    for name, fn in (("one_by_one", one_by_one), ("batched", batched)):
        fn()  # warm-up: autotuning, graph capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        res[name] = {"s_per_pass": dt, "units_per_s": units / dt}
    for h, _, _ in hs:
        h.close()
    return {"chains": len(sizes), "n": sizes, "n_tau": m["n_tau"], "n_s": m["n_s"],
            "timed": "rssri_sigma (S4-S10) of every chain, host wall clock, setups excluded",
            **res, "speedup": res["one_by_one"]["s_per_pass"] / res["batched"]["s_per_pass"]}


def c4_run(args):
    """The many-chain workload (64 chains of uneven size N_k = 100 + round(700 k/63),
    n_occ = N/2, N_aux = 3N, 64 tau points, 200 sample pairs, eps = 1e-3), one
    chain after another: inputs drawn on the device, setup (S1-S3, S6, S7) and
    rssri_sigma (S4, S5, S8-S10) timed with a device synchronisation on both
    sides, the handle and inputs freed before the next chain (the chains'
    (ij|A) alone would be 225 GB).  A chain of N = 100 is run first, untimed,
    to take the one-time tile tuning and graph capture out of the numbers."""
    import torch
    from paper_2005_12338_gb300 import binding, build
    build.build()
    pr, dd = FORMS[args.form]
    prec = {"bf16": binding.RSSRI_PREC_BF16, "fp64": binding.RSSRI_PREC_FP64,
            "df64": binding.RSSRI_PREC_DF64}[pr]
    dd = {"fp64": binding.RSSRI_DD_FP64, "df64": binding.RSSRI_DD_DF64,
          "oz": binding.RSSRI_DD_OZ}[dd]
    m = dict(synth.C4)
    sizes = synth.many_sizes(m["k"], m["n_min"], m["n_max"])[:args.c4]
    opts = binding.Handle.options(m["eps_prime"], m["eps"], m["n_s"], 5, precision=prec,
                                  dd_arith=dd)

    def one(n, seed):
        s = synth.make_system_torch(n, n // 2, 3 * n, m["n_tau"], input_seed=seed)
        sig = torch.empty((m["n_tau"], n, n), dtype=torch.float64, device="cuda")
        h = binding.Handle(torch.cuda.current_device())
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.setup(s.eri3, s.metric, s.orb_e, s.orb_c, s.tau, s.tau_w, n_occ=s.n_occ,
                    mu=s.mu, beta=s.beta, opts=opts)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            e, se, st = h.sigma(opts, sig)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
        finally:
            h.close()
        del s, sig
        torch.cuda.empty_cache()
        return {"n": n, "setup_s": t1 - t0, "sample_s": t2 - t1, "e_corr": e, "stderr": se,
                "pairs_kept": st["n_pairs_large"]}

    one(100, 1000)
    chains = []
    for k, n in enumerate(sizes):
        chains.append(one(n, k))
        c = chains[-1]
        print(f"chain {k} N={n}: setup {c['setup_s']:.3f} s, sampling {c['sample_s']:.3f} s",
              file=sys.stderr, flush=True)
    units = len(chains) * m["n_s"] * m["n_tau"]
    t_setup = sum(c["setup_s"] for c in chains)
    t_samp = sum(c["sample_s"] for c in chains)
    out = {"metric": "Sigma(tau) units/s (unit = one sample pair x one tau point)",
           "value": units / (t_setup + t_samp), "unit": "units/s", "n_gpus": 1,
           "higher_is_better": True, "dtype": {"plain": "f64", "chosen": "bf16+f64", "df64": "df64"}[args.form],
           "data": "synthetic",
           "config": {"workload": f"c4_many_chains: {len(chains)} of 64 chains, N {sizes[0]}.."
                                  f"{sizes[-1]}, N_aux=3N, N_tau={m['n_tau']}, "
                                  f"N_s={m['n_s']}, eps={m['eps']}", "form": args.form,
                      "timed": "setup + rssri_sigma per chain, host clock around device "
                               "synchronisations; chains one after another"},
           "units": units, "setup_s_total": t_setup, "sampling_s_total": t_samp,
           "sampling_units_per_s": units / t_samp, "chains": chains}
    print(json.dumps(out), flush=True)


def pipe_peaks(binding, device):
    """Measured fp64 and fp32 pipe peaks of this GPU, TFLOP/s: the library's
    DFMA, DMMA and FFMA micro-benchmarks, and (fp64, for reference only: not
    on the path) the library DGEMM behind torch's float64 matmul, 4096^3."""
    import torch
    out = {}
    for name, which in (("dfma", binding.RSSRI_PEAK_DFMA), ("dmma", binding.RSSRI_PEAK_DMMA),
                        ("ffma", binding.RSSRI_PEAK_FFMA)):
        try:
            out[name] = binding.peak_measure(which, device)[0]
        except Exception:
            out[name] = None
    try:
        a = torch.randn(4096, 4096, dtype=torch.float64, device=f"cuda:{device}")
        b = torch.randn(4096, 4096, dtype=torch.float64, device=f"cuda:{device}")
        for _ in range(2):
            torch.matmul(a, b)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        reps = 5
        for _ in range(reps):
            torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        out["dgemm_library"] = 2.0 * 4096 ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
        del a, b
    except Exception:
        out["dgemm_library"] = None
    out["fp64"] = max(v for k, v in out.items() if k != "ffma" and v)
    return out


def our_arm(args):
    import torch
    import torch.distributed as dist

    from paper_2005_12338_gb300 import binding, build
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    cfg = dict(synth.CONFIGS[args.workload])
    if args.eps is not None:
        cfg["eps"] = args.eps
    if args.n_tau is not None:
        cfg["n_tau"] = args.n_tau
    s = synth.make_system(cfg["n"], cfg["n_occ"], cfg["n_aux"], cfg["n_tau"], input_seed=0)
    n, nt, ns = s.n, s.n_tau, cfg["n_s"]
    units_step = ns * nt
    host = [s.eri3, s.metric, s.orb_e, s.orb_c, s.tau, s.tau_w]
    dev = [torch.from_numpy(a).to(f"cuda:{local}") for a in host]
    sig = torch.empty((nt, n, n), dtype=torch.float64, device=f"cuda:{local}")
    ep = torch.empty(ns, dtype=torch.float64, device=f"cuda:{local}")
    h = binding.Handle(local)
    stream = torch.cuda.current_stream(local)
    prec_code = {"bf16": binding.RSSRI_PREC_BF16, "tf32": binding.RSSRI_PREC_TF32,
                 "fp64": binding.RSSRI_PREC_FP64, "df64": binding.RSSRI_PREC_DF64}
    dd_code = {"fp64": binding.RSSRI_DD_FP64, "df64": binding.RSSRI_DD_DF64,
               "oz": binding.RSSRI_DD_OZ}

    def opts(form, seed, profile=0, estimator=binding.RSSRI_EST_CV, **kw):
        prec, dd = FORMS[form]
        return binding.Handle.options(cfg["eps_prime"], cfg["eps"], ns, seed, profile=profile,
                                      precision=prec_code[prec], dd_arith=dd_code[dd],
                                      estimator=estimator, **kw)

    def step(form, seed, profile=0, **kw):
        o = opts(form, seed, profile, **kw)
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=o)
        return h.sigma(o, sig, ep)

    def timed(form, seeds, profile=1, clock=None):
        """Steps over the seeds between CUDA events on the stream; returns
        (ms, per-step (e, se, fixed ms, sampling ms), summed stats)."""
        prof = {"ms": np.zeros(8), "gf": np.zeros(8), "tgf": np.zeros(8),
                "l": np.zeros(8, dtype=np.int64), "launches": 0}
        res = []
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for sd in seeds:
            e, se, st = step(form, sd, profile=profile)
            res.append((e, se, st["t_setup_ms"] + st["t_green_dd_ms"], st["t_sample_ms"]))
            prof["ms"] += st["prof_ms"]
            prof["gf"] += st["prof_gflop"]
            prof["tgf"] += st["prof_tensor_gflop"]
            prof["l"] += np.array(st["prof_launches"], dtype=np.int64)
            prof["launches"] += st["kernel_launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), res, prof

    form = args.form
    # ---- the benchmark line
    for k in range(args.warmup):
        step(form, replicas.rank_seed(rank, 900_000 + k))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    seeds = [replicas.rank_seed(rank, k) for k in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms_line, results, prof = timed(form, seeds[:1])
        sig_first = sig.clone()
        if args.steps > 1:
            ms_rest, res_rest, prof_rest = timed(form, seeds[1:])
            ms_line += ms_rest
            results += res_rest
            for key in ("ms", "gf", "tgf", "l"):
                prof[key] = prof[key] + prof_rest[key]
            prof["launches"] += prof_rest["launches"]
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    clocks = clk.summary()
    ms_max = replicas.max_over_ranks(ms_line, device=f"cuda:{local}")
    value = replicas.job_throughput(units_step, args.steps, world, ms_max / 1e3)
    forms = {form: {"chain": FORMS[form][0], "block": FORMS[form][1],
                    "units_per_s": units_step * args.steps / (ms_line / 1e3),
                    "ms_per_step": ms_line / args.steps,
                    "fixed_ms_per_step": float(np.mean([r[2] for r in results])),
                    "sampling_ms_per_step": float(np.mean([r[3] for r in results])),
                    "time_to_1mEh": time_to_target(results, ns, 1e-3)}}
    profs = {form: prof}

    # ---- the other forms on the same first seed: throughput and error against this one
    if not args.no_compare:
        base = sig_first
        base_e = results[0][0]
        for other in [f for f in ("chosen", "plain", "df64") if f != form]:
            k_other = args.steps if other == "chosen" else 1
            for k in range(min(args.warmup, 2)):
                step(other, replicas.rank_seed(rank, 990_000 + k))
            ms_o, res_o, prof_o = timed(other, seeds[:k_other])
            if k_other > 1:
                step(other, seeds[0])  # the output of the first seed, for the comparison
            sig_o = sig.clone()
            forms[other] = {"chain": FORMS[other][0], "block": FORMS[other][1],
                            "units_per_s": units_step * k_other / (ms_o / 1e3),
                            "ms_per_step": ms_o / k_other,
                            "steps_timed": k_other,
                            "fixed_ms_per_step": float(np.mean([r[2] for r in res_o])),
                            "sampling_ms_per_step": float(np.mean([r[3] for r in res_o])),
                            "time_to_1mEh": time_to_target(res_o, ns, 1e-3)}
            profs[other] = prof_o
            if other == "plain" or form == "plain":
                ref_sig = sig_o if other == "plain" else base
                ref_e = res_o[0][0] if other == "plain" else base_e
                got_sig = base if other == "plain" else sig_o
                got_e = base_e if other == "plain" else res_o[0][0]
                # the stochastic remainder of the plain form's estimate on these draws
                h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts("plain", seeds[0]))
                sdd = torch.from_numpy(h.export("SIGMA_DD").reshape(nt, n, n)).to(sig.device)
                rem = ref_sig - 0.5 * (sdd + sdd.transpose(1, 2))
                d = got_sig - ref_sig
                entry = forms[form if other == "plain" else other]
                entry["vs_plain_same_draws"] = {
                    "sigma_rel_fro": float(torch.linalg.norm(d) / torch.linalg.norm(ref_sig)),
                    "sigma_stochastic_part_rel_fro": float(torch.linalg.norm(d) /
                                                           torch.linalg.norm(rem)),
                    "e_corr_abs": abs(got_e - ref_e), "e_corr_rel": abs(got_e - ref_e) / abs(ref_e),
                    "e_stderr": results[0][1]}
    t_plain = forms.get("plain", {}).get("time_to_1mEh")
    t_chosen = forms.get("chosen", {}).get("time_to_1mEh")
    chosen_vs_plain = None
    if t_plain and t_chosen:
        chosen_vs_plain = {"time_to_1mEh_plain_s": t_plain["seconds"],
                           "time_to_1mEh_chosen_s": t_chosen["seconds"],
                           "speedup": t_plain["seconds"] / t_chosen["seconds"],
                           "sampling_only_speedup": t_plain["sampling_only_s"] /
                           max(t_chosen["sampling_only_s"], 1e-12),
                           "throughput_ratio": forms["chosen"]["units_per_s"] /
                           forms["plain"]["units_per_s"]}

    # Sec. IV: the range-separated estimator against plain stochastic RI at the
    # same number of sample pairs and the same seed (chosen form)
    rs_vs_sri = None
    if not args.no_compare:
        e_rs, se_rs, _ = step("chosen", seeds[0])
        e_sri, se_sri, _ = step("chosen", seeds[0], estimator=binding.RSSRI_EST_SRI)
        rs_vs_sri = {"e_corr_rs": e_rs, "stderr_rs": se_rs, "e_corr_sri": e_sri,
                     "stderr_sri": se_sri, "stderr_ratio_sri_over_rs": se_sri / se_rs,
                     "agree_within_3_sigma": abs(e_sri - e_rs) < 3 * (se_sri ** 2 + se_rs ** 2) ** 0.5}

    # learned control variate (fp64 chain): train on an independent run, then
    # estimate with it on the first timed seed, next to the plain estimate
    def at_eps(eps, plain_ttt=None):
        """Time to a 1 mEh standard error at one eps: the plain form, the
        chosen form, and the chosen form with the learned control variate
        (trained on an independent run, seed 777; statistics need the
        fp64-accurate double-float chain), the latter two on the same draws."""
        def o_e(form, seed, cvf=0):
            prec, dd = FORMS[form]
            return binding.Handle.options(cfg["eps_prime"], eps, ns, seed, cv=cvf,
                                          precision=prec_code[prec], dd_arith=dd_code[dd])
        tr = binding.Handle.options(cfg["eps_prime"], eps, ns, replicas.rank_seed(rank, 777),
                                    dd_arith=binding.RSSRI_DD_OZ,
                                    precision=binding.RSSRI_PREC_DF64)
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=tr)
        c0 = time.perf_counter()
        lb, la = h.cv_train(tr, synth.mlp_init(0), 400, 4096, 1e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - c0
        rows = {}
        runs = [("chosen", "chosen", 0), ("chosen+cv", "chosen", 1)]
        if plain_ttt is None:
            runs.insert(0, ("plain", "plain", 0))
        for name, form_, cvf in runs:
            o = o_e(form_, seeds[0], cvf)
            for _ in range(2):  # a warm-up call (graph capture, tile tuning), then the timed one
                h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=o)
                torch.cuda.synchronize()
                e_, se_, st_ = h.sigma(o, sig, ep)
                torch.cuda.synchronize()
            # the coefficients c are computed once per setup: fixed cost, not per pair
            cvc = st_["t_cv_c_ms"]
            rows[name] = (e_, se_, st_["t_setup_ms"] + st_["t_green_dd_ms"] + cvc,
                          st_["t_sample_ms"] - cvc, ep.cpu().numpy().copy())
        ttt = {k: time_to_target([v[:4]], ns, 1e-3) for k, v in rows.items()}
        if plain_ttt is not None:
            ttt["plain"] = plain_ttt
        a, b = rows["chosen"][4], rows["chosen+cv"][4]
        return {"eps": eps, "time_to_1mEh": ttt,
                "speedup_vs_plain": {k: ttt["plain"]["seconds"] / v["seconds"]
                                     for k, v in ttt.items() if k != "plain"},
                "stderr": {k: v[1] for k, v in rows.items()},
                "e_corr": {k: v[0] for k, v in rows.items()},
                "sampling_ms": {k: v[3] for k, v in rows.items()},
                "learned_cv": {"fit_loss_before": lb, "fit_loss_after": la, "train_s": t_train,
                               "paired_sd_ratio_plain_over_learned": float(np.std(a) / np.std(b))},
                "note": "chosen = bf16 chain + sliced fp64-accurate block; chosen+cv adds the "
                        "learned control variate (its one-time training, train_s, excluded; "
                        "its coefficients, computed once per setup, in the fixed part); "
                        "setup once plus sample pairs at the measured cost per pair"}

    cv_report, by_eps = None, None
    if not args.no_cv:
        by_eps = {str(cfg["eps"]): at_eps(cfg["eps"], forms.get("plain", {}).get("time_to_1mEh")),
                  "0.1": at_eps(0.1) if cfg["eps"] != 0.1 else None}
        cv_report = dict(by_eps[str(cfg["eps"])]["learned_cv"], eps=cfg["eps"])

    many_report = None
    if args.many > 0:
        pr, dd = FORMS["chosen"]
        many_report = many_systems(args, binding, torch, prec_code[pr], dd_code[dd])

    # the literal reading of Eq. 25 on the same draws as the first timed step
    literal_report = None
    if args.literal:
        l0 = torch.cuda.Event(enable_timing=True)
        l1 = torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        e_lit, se_lit, st_lit = step("plain", seeds[0], estimator=binding.RSSRI_EST_LITERAL)
        l1.record(stream)
        torch.cuda.synchronize()
        literal_report = {"e_corr_literal": e_lit, "stderr_literal": se_lit,
                          "e_corr_cv": results[0][0], "stderr_cv": results[0][1],
                          "stderr_ratio_literal_over_cv": se_lit / results[0][1],
                          "ms_per_step": l0.elapsed_time(l1),
                          "sampling_ms": st_lit["t_sample_ms"]}

    # end to end through the C ABI with host buffers (pinned), copies included
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(a).pin_memory().numpy() for a in host]
        sig_h = torch.empty((nt, n, n), dtype=torch.float64).pin_memory().numpy()
        ep_h = torch.empty(ns, dtype=torch.float64).pin_memory().numpy()
        hh = binding.Handle(local)

        def step_host(seed):
            o = opts(form, seed)
            hh.setup(*pinned, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=o)
            return hh.sigma(o, sig_h, ep_h)
        step_host(replicas.rank_seed(rank, 990_000))
        k_e2e = min(args.steps, 3)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(k_e2e):
            step_host(seeds[k])
        el = replicas.max_over_ranks(time.perf_counter() - t0, device=f"cuda:{local}")
        e2e = {"value": units_step * k_e2e * world / el, "unit": "units/s",
               "h2d_bytes_per_step": int(sum(a.nbytes for a in host)),
               "d2h_bytes_per_step": int(sig_h.nbytes + ep_h.nbytes + 4 * 8),
               "steps": k_e2e}
        hh.close()

    if rank != 0:
        h.close()
        if world > 1:
            dist.destroy_process_group()
        return
    peaks, peak_src = measured_peaks()
    pipes = pipe_peaks(binding, local)
    bf16_peak = float(peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"]))

    def classes_of(pr, steps_):
        return {binding.PROF_CLASSES[c]: {
            "ms_per_step": pr["ms"][c] / steps_, "gflop_per_step": pr["gf"][c] / steps_,
            "tensor_gflop_per_step": pr["tgf"][c] / steps_,
            "launches_per_step": int(pr["l"][c]) // steps_,
            "tflops_fp64_equivalent": (pr["gf"][c] / (pr["ms"][c] / 1e3) / 1e3
                                       if pr["ms"][c] > 0 else None),
            "tensor_tflops": (pr["tgf"][c] / (pr["ms"][c] / 1e3) / 1e3
                              if pr["ms"][c] > 0 and pr["tgf"][c] > 0 else None)}
            for c in range(len(binding.PROF_CLASSES))}

    for f in forms:
        forms[f]["classes"] = classes_of(profs[f], forms[f].get("steps_timed", args.steps))

    def roofline_of(f, pr):
        dom = int(np.argmax(pr["ms"]))
        name = binding.PROF_CLASSES[dom]
        chain, block = FORMS[f]
        tensor = pr["tgf"][dom] > 0
        if tensor:
            achieved = pr["tgf"][dom] / (pr["ms"][dom] / 1e3) / 1e3
            peak, unit = (bf16_peak / 2 if chain == "tf32" and name == "chain_gemm"
                          else bf16_peak), "TFLOP/s"
            psrc = "bf16 dense tensor peak, " + peak_src
            bound = "tensor"
            work = "tensor flops issued (digit products over the padded tiles)"
        else:
            achieved = pr["gf"][dom] / (pr["ms"][dom] / 1e3) / 1e3
            df = (block == "df64" and name in ("dd_spmm", "dd_gemm")) or \
                 (chain == "df64" and name == "chain_gemm")
            peak = pipes["ffma"] if df else pipes["fp64"]
            psrc = ("measured fp32 FFMA pipe (double-float: each multiply-add is about a "
                    "dozen fp32 instructions; the fraction is fp64-equivalent flops over the "
                    "fp32 rate)" if df else
                    "measured fp64 pipe: best of the DFMA and DMMA micro-benchmarks "
                    "(rssri_peak_measure) and the library DGEMM (torch float64 matmul, "
                    "4096^3)")
            bound, unit = "alu", "TFLOP/s"
            work = "algorithmic fp64 flops (2 N_aux P^2 per exchange contraction, 2mnk per product)"
        launches = int(pr["l"][dom])
        return {"bound": bound, "kernel": name, "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak if peak else None,
                "traffic": traffic_for(name, f),
                "peak_source": psrc, "work": work,
                "gflop_per_launch": (pr["tgf"][dom] if tensor else pr["gf"][dom]) /
                max(launches, 1),
                "launches": launches,
                "share_of_step": float(pr["ms"][dom] / max(pr["ms"].sum(), 1e-9))}

    roofline = roofline_of(form, prof)
    other_rooflines = {f: roofline_of(f, profs[f]) for f in forms if f != form}
    line = {"metric": "Sigma(tau) units/s (unit = one sample pair x one tau point)",
            "value": value, "unit": "units/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"plain": "f64", "chosen": "bf16+f64", "df64": "df64"}[form],
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: N={n} n_occ={s.n_occ} N_aux={s.n_aux} "
                                   f"N_tau={nt} N_s={ns} eps={cfg['eps']} "
                                   f"eps'={cfg['eps_prime']}, whole path per step",
                       "form": form, "chain_precision": FORMS[form][0],
                       "block_arith": FORMS[form][1],
                       "l2": "inputs larger than L2 (3-index integrals 192 MB); steps of seconds",
                       "parallelism": f"replicas x{world} (independent seeds, no collective)"},
            "roofline": roofline, "clocks": clocks, "gpu_launches": int(prof["launches"]),
            "e2e": e2e,
            "extra": {"e_corr_per_step": [r[0] for r in results],
                      "e_stderr_per_step": [r[1] for r in results],
                      "forms": forms, "chosen_vs_plain_fp64": chosen_vs_plain,
                      "rooflines_other_forms": other_rooflines,
                      "measured_pipe_peaks_tflops": pipes,
                      "rs_vs_sri_same_n_s": rs_vs_sri,
                      "learned_control_variate": cv_report,
                      "time_to_1mEh_by_eps": by_eps,
                      "literal_estimator": literal_report,
                      "many_systems": many_report}}
    if not args.no_cpu_baseline and world == 1:
        cb = oracle_sample(s, cfg, 0)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        one = oracle_single_thread(args)
        if one is not None:
            line["cpu_baseline"]["single_thread"] = one
    print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


def oracle_single_thread(args):
    """The same bounded oracle sample in a fresh interpreter whose BLAS may use
    one thread (the environment is set before numpy loads): the baseline's
    single-core figure.  None if it fails."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--workload",
           args.workload]
    if args.eps is not None:
        cmd += ["--eps", str(args.eps)]
    if args.n_tau is not None:
        cmd += ["--n-tau", str(args.n_tau)]
    try:
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def main():
    args = parse()
    if args.oracle_sample:
        cfg = dict(synth.CONFIGS[args.workload])
        if args.eps is not None:
            cfg["eps"] = args.eps
        if args.n_tau is not None:
            cfg["n_tau"] = args.n_tau
        s = synth.make_system(cfg["n"], cfg["n_occ"], cfg["n_aux"], cfg["n_tau"], input_seed=0)
        r = oracle_sample(s, cfg, 0, budget_s=6.0)
        print(json.dumps({k: r[k] for k in ("value", "unit", "cores")}), flush=True)
    elif args.impl == "reference":
        reference_arm(args)
    elif args.c4 > 0:
        c4_run(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
