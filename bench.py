"""Benchmark of the RS-SRI-GF2 self-energy path on GB300.

Workload: N = 200 basis functions, 100 occupied, N_aux = 600, 64 tau points,
N_s = 300 sample pairs, eps = 1e-3, eps' = 0.02 (synthetic hydrogen-chain-like
integrals).  One step is one pass of the whole path: V^{-1/2}, screening,
[K]^L and its cut, the pair-space product, G(tau), the deterministic block,
the Rademacher draws, R and R^L, the chain products for every (sample pair,
tau) unit, the energy and the symmetrised output.  The metric is Sigma(tau)
units per second, a unit being one (sample pair, tau point); inputs are
resident in HBM when the timed region starts.  Every step draws a new seed.
The timed form computes every product in double-float arithmetic (fp64
accurate: within 1e-10 of the fp64 oracle); the IEEE-fp64 form and a
reduced-precision tensor-core form are timed beside it for comparison.

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
# fp64 ALU peak of the DFMA pipe: 152 SMs x 2 fp64 FMA/clock/SM x 2 flop x
# 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# Double-float multiply-add (--dd df64, --precision df64): 12 fp32
# instructions each (TwoProduct with 3 fma, TwoSum, error collection) on
# 152 SMs x 128 fp32 lanes x 2070 MHz, counted as 2 fp64-equivalent flop.
DF64_PEAK_TFLOPS = 152 * 128 * 2.070e9 / 12 * 2 / 1e12
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.CONFIGS))
    ap.add_argument("--precision", default="df64", choices=["df64", "bf16", "tf32", "fp64"],
                    help="chain products: double-float on the fp32 pipes (fp64-accurate, the "
                         "benchmark line), bf16 or tf32 tensor cores (reduced precision), or "
                         "IEEE fp64 (plain)")
    ap.add_argument("--reduced", default="bf16", choices=["bf16", "tf32", "none"],
                    help="also time this reduced-precision tensor-core form and report its "
                         "error against the IEEE fp64 form on the same draws")
    ap.add_argument("--dd", default="df64", choices=["df64", "fp64"],
                    help="exchange contraction of the deterministic block: double-float on "
                         "the fp32 pipes (chosen) or IEEE fp64")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--eps", type=float, default=None,
                    help="override the K^L cut eps of the workload (e.g. the paper's 0.1)")
    ap.add_argument("--n-tau", type=int, default=None,
                    help="override the number of tau points of the workload (for one-off "
                         "measurements on the largest workload; not the benchmark line)")
    ap.add_argument("--cv", action="store_true",
                    help="also train the learned control variate on an independent run and "
                         "report its estimate (fp64 chain)")
    ap.add_argument("--literal", action="store_true",
                    help="also run the literal Eq. 25 estimator (fp64 chain, exact-D cross "
                         "terms) on the first timed seed and report its cost and stderr")
    ap.add_argument("--many", type=int, default=0,
                    help="also time K independent chains of uneven size (N from 64 to 256) "
                         "one by one and batched on K streams (rssri_sigma_batch)")
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


def tensor_peak(peaks, precision):
    """Dense tensor peak of the chain's operand type: the measured bf16 figure,
    halved for tf32 (the nominal tf32 : bf16 ratio)."""
    bf16 = float(peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"]))
    return bf16 / 2.0 if precision == "tf32" else bf16


def tensor_peak_source(peak_src, precision):
    if precision == "tf32":
        return "bf16 dense tensor peak x 1/2 (nominal tf32 ratio), " + peak_src
    return "bf16 dense tensor peak, " + peak_src


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
def traffic_for(key):
    """Per-launch DRAM bytes of the dominant kernel (key: kernel class, with
    "/df64" for the double-float deterministic block) from the committed ncu
    summary, or None if absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(key)
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
    host = [s.eri3, s.metric, s.orb_e, s.orb_c, s.tau, s.tau_w]
    dev = [torch.from_numpy(a).to(f"cuda:{local}") for a in host]
    sig = torch.empty((nt, n, n), dtype=torch.float64, device=f"cuda:{local}")
    ep = torch.empty(ns, dtype=torch.float64, device=f"cuda:{local}")
    h = binding.Handle(local)
    stream = torch.cuda.current_stream(local)

    prec_code = {"bf16": binding.RSSRI_PREC_BF16, "tf32": binding.RSSRI_PREC_TF32,
                 "fp64": binding.RSSRI_PREC_FP64, "df64": binding.RSSRI_PREC_DF64}
    prec = prec_code[args.precision]
    tensor_chain = args.precision in ("bf16", "tf32")
    dd = binding.RSSRI_DD_DF64 if args.dd == "df64" else binding.RSSRI_DD_FP64

    def step(seed, profile=0, precision=prec, dd_arith=dd, estimator=binding.RSSRI_EST_CV,
             pair_batch=0):
        o = binding.Handle.options(cfg["eps_prime"], cfg["eps"], ns, seed, profile=profile,
                                   precision=precision, dd_arith=dd_arith, estimator=estimator,
                                   pair_batch=pair_batch)
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=o)
        return h.sigma(o, sig, ep)

    for k in range(args.warmup):
        step(replicas.rank_seed(rank, 900_000 + k))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    prof_ms = np.zeros(8)
    prof_gf = np.zeros(8)
    prof_l = np.zeros(8, dtype=np.int64)
    launches = 0
    results = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            e, se, st = step(replicas.rank_seed(rank, k), profile=1)
            results.append((e, se, st["t_setup_ms"] + st["t_green_dd_ms"], st["t_sample_ms"]))
            if k == 0:
                sig_first = sig.clone()
            prof_ms += st["prof_ms"]
            prof_gf += st["prof_gflop"]
            prof_l += np.array(st["prof_launches"], dtype=np.int64)
            launches += st["kernel_launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    clocks = clk.summary()
    ms_max = replicas.max_over_ranks(e0.elapsed_time(e1), device=f"cuda:{local}")
    units = ns * nt * args.steps * world
    value = replicas.job_throughput(ns * nt, args.steps, world, ms_max / 1e3)

    # the plain fp64 form on the same seed: throughput and the error of the chosen form
    compare = None
    # (on the largest workloads the fp64 chain takes its pairs 100 at a time to
    # bound its scratch; the sums are the same up to rounding order)
    plain = dict(precision=binding.RSSRI_PREC_FP64, dd_arith=binding.RSSRI_DD_FP64,
                 pair_batch=100 if n >= 500 else 0)
    sig64 = None
    if (tensor_chain or args.dd == "df64" or args.precision == "df64") and \
            not args.no_fp64_compare:
        step(replicas.rank_seed(rank, 990_001), **plain)  # tunes the fp64 chain shapes
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        e64, se64, st64 = step(replicas.rank_seed(rank, 0), profile=1, **plain)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        sdd = torch.from_numpy(h.export("SIGMA_DD").reshape(nt, n, n)).to(sig.device)
        st_ref = sig - 0.5 * (sdd + sdd.transpose(1, 2))
        err_sigma = float(torch.linalg.norm(sig_first - sig) / torch.linalg.norm(sig))
        err_st = float(torch.linalg.norm(sig_first - sig) / torch.linalg.norm(st_ref))
        sig64, st_ref64 = sig.clone(), st_ref.clone()
        res64 = [(e64, se64, st64["t_setup_ms"] + st64["t_green_dd_ms"], st64["t_sample_ms"])]
        compare = {"plain_fp64_units_per_s": ns * nt / (ms64 / 1e3),
                   "plain_fp64_ms_per_step": ms64,
                   "plain_fp64_sampling_ms_per_step": st64["t_sample_ms"],
                   "chosen_sampling_ms_per_step": float(np.mean([r[3] for r in results])),
                   "sampling_speedup": st64["t_sample_ms"] / float(np.mean([r[3] for r in results])),
                   "chosen_vs_fp64_same_seed": {
                       "sigma_rel_fro": err_sigma,
                       "sigma_stochastic_part_rel_fro": err_st,
                       "e_corr_abs": abs(results[0][0] - e64),
                       "e_corr_rel": abs(results[0][0] - e64) / abs(e64),
                       "e_stderr": se64},
                   "time_to_1mEh_plain_fp64_s": time_to_target(res64, ns, 1e-3)}

    # the reduced-precision tensor-core form: throughput, and its error against
    # the IEEE fp64 form on the same draws
    reduced = None
    if args.reduced != "none" and not tensor_chain and sig64 is not None:
        rp = prec_code[args.reduced]
        er, ser, _ = step(replicas.rank_seed(rank, 0), precision=rp)  # graph capture + error
        torch.cuda.synchronize()
        d = sig - sig64
        err = {"sigma_rel_fro": float(torch.linalg.norm(d) / torch.linalg.norm(sig64)),
               "sigma_stochastic_part_rel_fro": float(torch.linalg.norm(d) /
                                                      torch.linalg.norm(st_ref64)),
               "e_corr_abs": abs(er - e64), "e_corr_rel": abs(er - e64) / abs(e64),
               "e_stderr": se64}
        step(replicas.rank_seed(rank, 990_002), precision=rp)
        torch.cuda.synchronize()
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        rres = []
        r0.record(stream)
        for k in range(args.steps):
            e_, se_, st_ = step(replicas.rank_seed(rank, k), precision=rp)
            rres.append((e_, se_, st_["t_setup_ms"] + st_["t_green_dd_ms"], st_["t_sample_ms"]))
        r1.record(stream)
        torch.cuda.synchronize()
        rms = r0.elapsed_time(r1) / args.steps
        reduced = {"precision": args.reduced, "units_per_s": ns * nt / (rms / 1e3),
                   "ms_per_step": rms,
                   "sampling_ms_per_step": float(np.mean([r[3] for r in rres])),
                   "vs_fp64_same_seed": err,
                   "time_to_1mEh_s": time_to_target(rres, ns, 1e-3)}

    # Sec. IV: the range-separated estimator against plain stochastic RI at the
    # same number of sample pairs and the same seed
    e_sri, se_sri, _ = step(replicas.rank_seed(rank, 0), estimator=binding.RSSRI_EST_SRI)
    rs_vs_sri = {"e_corr_rs": results[0][0], "stderr_rs": results[0][1], "e_corr_sri": e_sri,
                 "stderr_sri": se_sri, "stderr_ratio_sri_over_rs": se_sri / results[0][1],
                 "agree_within_3_sigma": abs(e_sri - results[0][0]) <
                 3 * (se_sri ** 2 + results[0][1] ** 2) ** 0.5}

    # learned control variate (fp64 chain): train on an independent run, then
    # estimate with it on the first timed seed, next to the plain estimate
    cv_report = None
    if args.cv:
        # the control variate needs F and F^L separately: fp64 or double-float chain
        cvp = prec if args.precision in ("fp64", "df64") else binding.RSSRI_PREC_FP64
        tr = binding.Handle.options(cfg["eps_prime"], cfg["eps"], ns, replicas.rank_seed(rank, 777),
                                    dd_arith=dd, precision=cvp)
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=tr)
        c0 = time.perf_counter()
        lb, la = h.cv_train(tr, synth.mlp_init(0), 400, 4096, 1e-3)
        t_train = time.perf_counter() - c0
        ev = dict(precision=cvp, dd_arith=dd)
        e_cv, se_cv, st_cv = step(replicas.rank_seed(rank, 0), **ev,
                                  estimator=binding.RSSRI_EST_CV)
        o_cv = binding.Handle.options(cfg["eps_prime"], cfg["eps"], ns, replicas.rank_seed(rank, 0),
                                      dd_arith=dd, cv=1, precision=cvp)
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=o_cv)
        e_l, se_l, st_l = h.sigma(o_cv, sig, ep)
        cv_report = {"fit_loss_before": lb, "fit_loss_after": la, "train_s": t_train,
                     "e_corr_plain": e_cv, "stderr_plain": se_cv, "e_corr_learned": e_l,
                     "stderr_learned": se_l, "stderr_ratio_plain_over_learned": se_cv / se_l}

    many_report = many_systems(args, binding, torch, prec, dd) if args.many > 0 else None

    # the literal reading of Eq. 25 on the same draws as the first timed step
    literal_report = None
    if args.literal:
        l0 = torch.cuda.Event(enable_timing=True)
        l1 = torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        e_lit, se_lit, st_lit = step(replicas.rank_seed(rank, 0),
                                     precision=binding.RSSRI_PREC_FP64,
                                     estimator=binding.RSSRI_EST_LITERAL)
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
            o = binding.Handle.options(cfg["eps_prime"], cfg["eps"], ns, seed, precision=prec,
                                       dd_arith=dd)
            hh.setup(*pinned, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=o)
            return hh.sigma(o, sig_h, ep_h)
        step_host(replicas.rank_seed(rank, 990_000))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            step_host(replicas.rank_seed(rank, k))
        el = replicas.max_over_ranks(time.perf_counter() - t0, device=f"cuda:{local}")
        e2e = {"value": units / el, "unit": "units/s",
               "h2d_bytes_per_step": int(sum(a.nbytes for a in host)),
               "d2h_bytes_per_step": int(sig_h.nbytes + ep_h.nbytes + 4 * 8)}
        hh.close()

    if rank != 0:
        h.close()
        if world > 1:
            dist.destroy_process_group()
        return
    peaks, peak_src = measured_peaks()
    dom = int(np.argmax(prof_ms))
    name = binding.PROF_CLASSES[dom]
    per_launch_gf = prof_gf[dom] / max(prof_l[dom], 1)
    achieved = prof_gf[dom] / (prof_ms[dom] / 1e3) / 1e3  # TFLOP/s
    df64_class = ((name in ("dd_spmm", "dd_gemm") and args.dd == "df64") or
                  (name in ("chain_gemm", "factor_gemm", "setup_gemm") and
                   args.precision == "df64"))
    if df64_class:
        peak = DF64_PEAK_TFLOPS
        psrc = ("derived: 152 SMs x 128 fp32 lanes x 2070 MHz / 12 fp32 instructions per "
                "double-float multiply-add x 2 flop (fp64-equivalent)")
    elif name == "chain_gemm" and tensor_chain:
        peak = tensor_peak(peaks, args.precision)
        psrc = tensor_peak_source(peak_src, args.precision)
    else:
        peak = FP64_PEAK_TFLOPS
        psrc = "derived: 152 SMs x 2 fp64 FMA/clk/SM x 2 flop x 2070 MHz (fp64 DFMA pipe)"
    roofline = {"bound": "tensor" if (name == "chain_gemm" and tensor_chain) else "alu",
                "kernel": name, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic_for(name + ("/df64" if name in ("dd_spmm", "dd_gemm") and
                                               args.dd == "df64" else "")),
                "peak_source": psrc + "; HBM/bf16 peaks " + peak_src,
                "gflop_per_launch": per_launch_gf, "launches": int(prof_l[dom]),
                "share_of_step": float(prof_ms[dom] / max(prof_ms.sum(), 1e-9))}
    tensor = None
    if tensor_chain:
        tpk = tensor_peak(peaks, args.precision)
        tf = prof_gf[0] / (prof_ms[0] / 1e3) / 1e3
        tensor = {"kernel": f"chain_gemm (tcgen05 {args.precision})", "bound": "tensor",
                  "achieved": tf, "peak": tpk, "unit": "TFLOP/s", "frac": tf / tpk,
                  "peak_source": tensor_peak_source(peak_src, args.precision)}
    classes = {binding.PROF_CLASSES[c]: {"ms_per_step": prof_ms[c] / args.steps,
                                         "gflop_per_step": prof_gf[c] / args.steps,
                                         "launches_per_step": int(prof_l[c]) // args.steps,
                                         "tflops": (prof_gf[c] / (prof_ms[c] / 1e3) / 1e3
                                                    if prof_ms[c] > 0 else None)}
               for c in range(len(binding.PROF_CLASSES))}
    line = {"metric": "Sigma(tau) units/s (unit = one sample pair x one tau point)",
            "value": value, "unit": "units/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "+".join(([args.precision] if tensor_chain else []) +
                              (["df64"] if "df64" in (args.precision, args.dd) else []) +
                              ["f64"]), "data": "synthetic",
            "config": {"workload": f"{args.workload}: N={n} n_occ={s.n_occ} N_aux={s.n_aux} "
                                   f"N_tau={nt} N_s={ns} eps={cfg['eps']} "
                                   f"eps'={cfg['eps_prime']}, whole path per step",
                       "chain_precision": args.precision,
                       "dd_exchange_arith": args.dd,
                       "l2": "inputs larger than L2 (3-index integrals 192 MB); steps of seconds",
                       "parallelism": f"replicas x{world} (independent seeds, no collective)"},
            "roofline": roofline, "clocks": clocks, "gpu_launches": launches,
            "e2e": e2e,
            "extra": {"e_corr_per_step": [r[0] for r in results],
                      "e_stderr_per_step": [r[1] for r in results],
                      "time_to_1mEh_s": time_to_target(results, ns, 1e-3),
                      "classes": classes, "tensor_roofline": tensor,
                      "chosen_vs_plain_fp64": compare, "rs_vs_sri_same_n_s": rs_vs_sri,
                      "reduced_precision_form": reduced,
                      "learned_control_variate": cv_report,
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
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
