#!/usr/bin/env python
"""Benchmark of the particle PHD filter step on GB300 (one JSON line on stdout).

Metric: particle x measurement pairs per second per PHD update (the update's
pairs, N_k x M_k summed over the timed steps, divided by the timed device
time of the whole steps), plus steps/s, at matched OSPA.  A step is one full
filter step: predict + birth, update, labelled extraction (+ CU fusion),
resampling (+ ring exchange), through libphd.so's phd_step (a CUDA graph of
the step's kernels, or the fused step kernel where a PE's slice fits one SM).

Default workload: the dense range-bearing configuration (100 targets, clutter
rate 500, ~600 measurements per scan, 2000 particles per target, 20000 births
per step, ~2.2e5 particles and ~1.3e8 pairs per update at steady state; FP32
bulk, FP64 normalisers and CDF), the largest single-GPU configuration.  A run
is 100 scans; the timed steps are scans 50.. of consecutive runs (all truth
targets exist from 40 % of a run on; the earlier scans are replayed untimed).
Measurement sets are resident in device memory before timing; L2 is flushed
(512 MiB write) between timed steps, outside the timed events.

OSPA (c = 100 m, p = 2) is computed on every timed scan and compared with the
FP64 oracle's on the same seeds and scans (a stored record written by
tests/golden/make_oracle_ospa.py, which calls only the oracle): once for the
timed run (in-kernel random numbers) and once for an untimed run that
injects the oracle's own random numbers; "matched" means within 5 %.

The line also carries compact sub-blocks for the 16-PE distributed workload,
the 256-run batch and the learned birth proposal (--no-subblocks drops them;
--workload NAME runs one workload alone).

--impl reference times the FP64 CPU oracle (the tests' reference
implementation) on the same workload on all host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

import scenario

METRIC = "particle×measurement pairs/s per PHD update and steps/s on 1 GB300 at matched OSPA"
UNIT = "pairs/s"
# nominal MUFU ex2 rate, context only: 152 SMs x 32 ex2/clk/SM x 2.07 GHz; the
# roofline divides by the rate phd_measure_ex2_rate measures on the device
EX2_NOMINAL_TEXP = 152 * 32 * 2.070e9 / 1e12
DEFAULT_WORKLOAD = "dense_rb_100t"
MATCH_TOL = 0.05


def cpu_info():
    """Host cores and CPU model (from /proc/cpuinfo, where the kernel reports one)."""
    model = None
    try:
        for ln in open("/proc/cpuinfo"):
            k, _, v = ln.partition(":")
            if k.strip().lower() in ("model name", "cpu model", "hardware") and v.strip():
                model = v.strip()
                break
            if k.strip() == "CPU part" and model is None:
                model = f"CPU part {v.strip()}"
    except OSError:
        pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def oracle_record(wname):
    """The stored oracle OSPA record of a workload, {seed: {scan: row}}, or None."""
    p = os.path.join(ROOT, "tests", "golden", f"oracle_ospa_{wname}.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    return {r["seed"]: {row["scan"]: row for row in r["scans"]} for r in d["runs"]}


def job_totals(amount, seconds, world, device="cpu"):
    """Whole-job aggregation over the ranks of a replicas run: the work units
    summed over ranks and the slowest rank's time (every rank returns the
    same pair).  One rank: the inputs unchanged."""
    if world <= 1:
        return float(amount), float(seconds)
    import torch
    t = torch.tensor([float(amount), float(seconds)], dtype=torch.float64, device=device)
    tp, tm = t.clone(), t.clone()
    torch.distributed.all_reduce(tp, op=torch.distributed.ReduceOp.SUM)
    torch.distributed.all_reduce(tm, op=torch.distributed.ReduceOp.MAX)
    return tp[0].item(), tm[1].item()


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def workload_config(w, runs, l2_note):
    return {"workload": w.name, "model": "particle PHD filter (DCPFPHD)" if w.num_pe > 1 else "particle PHD filter",
            "sensor": w.meas_model, "targets": w.n_targets, "clutter_rate": w.clutter_rate,
            "particles_per_target": w.particles_per_target, "births_per_step": w.birth_count,
            "num_pe": w.num_pe, "exchange_frac": w.exchange_frac, "ck_mode": w.ck_mode,
            "scans_per_run": w.steps, "runs": runs, "precision": w.precision, "l2": l2_note,
            "birth_mass": w.birth_mass, "global_batch": 1, "seq_len": w.steps, "parallelism": "replicas",
            **({"gate_sigma": w.gate_sigma, "likelihood": "truncated beyond gate_sigma std (a variant)"}
               if w.gate_sigma > 0 else {})}


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.02)
        self.mark = len(self.lines)

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.time(), ln.strip()))

    def begin(self):
        self.mark = len(self.lines)

    def end(self):
        time.sleep(0.12)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        for _, ln in self.lines[max(0, self.mark - 1):]:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                rows.append((float(p[0]), float(p[1]), p[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def ospa_metric(X, Y, c: float = 100.0, p: float = 2.0) -> float:
    """OSPA distance (Schuhmacher, Vo & Vo 2008) between two point sets with
    cut-off c and order p, by an optimal assignment (scipy)."""
    from scipy.optimize import linear_sum_assignment
    X = np.asarray(X, np.float64).reshape(-1, 2)
    Y = np.asarray(Y, np.float64).reshape(-1, 2)
    m, n = len(X), len(Y)
    if m == 0 and n == 0:
        return 0.0
    if m == 0 or n == 0:
        return float(c)
    if m > n:
        X, Y, m, n = Y, X, n, m
    D = np.minimum(np.linalg.norm(X[:, None, :] - Y[None, :, :], axis=2), c) ** p
    r, cidx = linear_sum_assignment(D)
    return float(((D[r, cidx].sum() + c ** p * (n - m)) / n) ** (1.0 / p))


def _bad_clocks(c):
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if any(r in bad for r in c.get("reasons", [])):
        return True
    if c.get("sm_mhz") and c.get("sm_max_mhz") and c["sm_mhz"] < 0.6 * c["sm_max_mhz"] and \
            "sw_power_cap" not in c.get("reasons", []):
        return True
    return False


# ----------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------

def oracle_run(w, seeds, max_steps, budget_s, skip=0, threads=1):
    """Run the FP64 oracle filter over whole runs of the scenarios of `seeds`
    with the scenario's injected random numbers (FP32-rounded, as the GPU
    path receives them); returns (pairs, seconds, steps, ospa_list) for the
    timed steps after `skip`, on `threads` host threads (the oracle's OpenMP
    build, bit-identical to the single-threaded one)."""
    import oracle
    used = oracle.set_threads(threads)
    oracle_run.threads_used = used
    pairs, secs, steps, ospas = 0, 0.0, 0, []
    done = 0
    try:
        for seed in seeds:
            sc = scenario.simulate(w, seed)
            f = oracle.OracleFilter(w)
            for k, Z in enumerate(sc.meas):
                noise = scenario.step_noise(seed, k, w.num_pe, w.pe_cap, np.float32)
                u = scenario.resample_u32(seed, k, w.num_pe)
                xu = scenario.exchange_u32(seed, k, w.num_pe, w.pe_cap) if w.num_pe > 1 else None
                n_before = sum(len(a) for a in f.x) + w.birth_count
                t0 = time.perf_counter()
                lab, zet = f.step(Z, noise, u, xu)
                dt = time.perf_counter() - t0
                done += 1
                if done <= skip:
                    continue
                pairs += n_before * len(Z)
                secs += dt
                steps += 1
                ospas.append(_ospa(zet, sc.truth[k]))
                if steps >= max_steps or secs >= budget_s:
                    return pairs, secs, steps, ospas
        return pairs, secs, steps, ospas
    finally:
        oracle.set_threads(1)


def _ospa(zet, truth):
    import oracle
    X = np.asarray(zet, np.float64)[:, [0, 2]] if len(zet) else np.zeros((0, 2))
    Y = truth[:, [0, 2]] if len(truth) else np.zeros((0, 2))
    return oracle.ospa(X, Y, 100.0, 2.0)


def cpu_baseline(w, seed, budget_s):
    """The oracle on whole filter steps of the workload, scans 0.. of run `seed`:
    single-threaded until ~budget_s, then the same steps on all host cores."""
    nproc = os.cpu_count() or 1
    p1, s1, n1, _ = oracle_run(w, [seed], 10 ** 9, budget_s, threads=1)
    pn, sn, nn, _ = oracle_run(w, [seed], n1, 10 ** 9, threads=nproc)
    import oracle
    info = cpu_info()
    return {"value": pn / sn if sn > 0 else None, "unit": UNIT, "cores": oracle_run.threads_used,
            "kind": "oracle",
            "sample": f"filter steps on scans 0..{n1 - 1} of {w.name} run {seed} ({p1:.3g} pairs; whole steps: "
                      f"predict, update, extraction, resampling), FP64 C oracle, OpenMP build on all host cores "
                      f"({sn:.1f} s)",
            **info,
            "single_thread": {"value": p1 / s1 if s1 > 0 else None, "unit": UNIT, "cores": 1, "seconds": round(s1, 2),
                              "sample": "the same steps, single-threaded build"},
            "openmp_seconds": round(sn, 2), "openmp_available": oracle.openmp_available()}


def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    budget = float(os.environ.get("PHD_REF_BUDGET_S", "150"))
    seeds = [args.seed + r for r in range(64)]
    nproc = os.cpu_count() or 1
    pairs, secs, steps, ospas = oracle_run(w, seeds, args.steps, budget, skip=args.warmup, threads=nproc)
    import oracle
    value = pairs / secs if secs > 0 else 0.0
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, None, "n/a (CPU)"),
        "steps_per_s": steps / secs if secs > 0 else 0.0,
        "ospa_mean": float(np.mean(ospas)) if ospas else None,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_run.threads_used,
                         "kind": "oracle", **cpu_info(),
                         "sample": f"{steps} whole filter steps of {w.name} (runs from seed {args.seed}, scans "
                                   f"from 0, after {args.warmup} untimed), FP64 C oracle on all host cores "
                                   f"(OpenMP build, bit-identical to the single-threaded one)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------

# Committed ncu summaries that carry per-update DRAM traffic: (summary file,
# the kernel sources the counters were taken on).  The traffic is reported
# only while those sources are unchanged.
_TRAFFIC_PROFILES = {
    ("grid", "dense_rb_100t"): ("k_step_grid_dense_rb_100t_ncu.md", ("k_persist.cuh", "phd_internal.cuh")),
    ("fused", "dist16_10t"): ("k_step_fused_dist16_ncu.md", ("k_fused.cu", "phd_internal.cuh")),
    ("staged", "dense_rb_100t"): ("update_dense_rb_100t_ncu.md",
                                  ("k_update.cu", "k_order.cu", "k_extract.cu", "phd_internal.cuh")),
}
UPDATE_KERNELS = "update stage (k_cell_hist, k_cell_scatter, k_colsum, k_finalize, k_rowsum, k_select)"


def kernel_sources_sha256(files):
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1503_03769_gb300", "csrc")
    for fn in files:
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()


def _traffic_from_profile(path, workload):
    """Per-update DRAM bytes of the timed kernels from the committed ncu
    summary, if it was taken on the current kernel sources (else None)."""
    entry = _TRAFFIC_PROFILES.get((path, workload))
    if entry is None:
        return None
    name, files = entry
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    want = traffic = None
    for ln in open(p).read().splitlines():
        if ln.startswith("source_sha256:"):
            want = ln.split(":", 1)[1].strip()
        if ln.startswith("traffic_bytes_per_update:"):
            try:
                traffic = float(ln.split(":", 1)[1].strip())
            except ValueError:
                traffic = None
    return traffic if want == kernel_sources_sha256(files) else None


def ex2_peak(local_rank):
    """The device's measured ex2 rate (phd_measure_ex2_rate: fastest of 20
    launches of ~6 ms), with the SM clock sampled while it ran."""
    import torch
    from paper_1503_03769_gb300 import phd
    clk = ClockSampler(_gpu_id(local_rank))
    clk.begin()
    rate, ms = phd.measure_ex2_rate(20)
    rate2, ms2 = phd.measure_ex2_rate(60)
    c = clk.end()
    best = max(rate, rate2)
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    out = {"ex2_per_s": best, "Texp_per_s": best / 1e12, "best_launch_ms": min(ms, ms2), "sms": sms,
           "sm_mhz_median": c.get("sm_mhz"), "clock_samples": c.get("samples"),
           "nominal_Texp_per_s": EX2_NOMINAL_TEXP,
           "how": "phd_measure_ex2_rate: 8 CTAs x 256 threads per SM, 8 independent chains of 4096 dependent "
                  "ex2.approx.ftz.f32 per thread; fastest launch (CUDA events)"}
    if c.get("sm_mhz"):
        out["ex2_per_clk_per_sm"] = best / (sms * c["sm_mhz"] * 1e6)
    return out


def _gpu_id(local_rank):
    import torch
    try:
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
        return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        return str(local_rank)


def _ospa_of(states, count, truth):
    n = int(count)
    est = states[:n].double().cpu().numpy() if n else np.zeros((0, 4))
    return ospa_metric(est[:, [0, 2]] if n else np.zeros((0, 2)),
                       truth[:, [0, 2]] if len(truth) else np.zeros((0, 2)), 100.0, 2.0)


def injected_ospa(f, w, seeds, scen, dev):
    """Untimed whole runs of `seeds` that inject the oracle's random numbers
    (the FP32-rounded draws tests/golden/make_oracle_ospa.py gives the oracle):
    OSPA (c = 100, p = 2) per (seed, scan)."""
    import torch
    out = {}
    K = w.num_pe
    for seed in seeds:
        sc = scen(seed)
        f.set_state([np.zeros((0, 4))] * K, [np.zeros(0)] * K)
        for k, Z in enumerate(sc.meas):
            noise = scenario.step_noise(seed, k, K, w.pe_cap, np.float32)
            u = scenario.resample_u32(seed, k, K)
            xu = scenario.exchange_u32(seed, k, K, w.pe_cap) if K > 1 else None
            st, lb = f.step_inject(Z, noise, u, xu)
            out[(seed, k)] = _ospa_of(st, len(lb), sc.truth[k])
    return out


def matched_ospa(w, timed_ospa, inj_ospa, rec, steady):
    """GPU OSPA against the oracle record on the same seeds and scans."""
    def mean_over(d, keys):
        v = [d[k] for k in keys if k in d]
        return float(np.mean(v)) if v else None

    keys_timed = [k for k in timed_ospa if k[0] in rec]
    orc = {(sd, sc): row["ospa2"] for sd, rows in rec.items() for sc, row in rows.items()}
    keys_steady = sorted({(sd, k) for sd, _ in keys_timed for k in range(steady, w.steps)})
    o_t, g_t, i_t = mean_over(orc, keys_timed), mean_over(timed_ospa, keys_timed), mean_over(inj_ospa, keys_timed)
    o_s, i_s = mean_over(orc, keys_steady), mean_over(inj_ospa, keys_steady)
    rel = lambda a, b: (a - b) / b if (a is not None and b) else None
    res = {"oracle_timed_scans": o_t, "gpu_timed": g_t, "gpu_injected_timed_scans": i_t,
           "rel_gpu_timed": rel(g_t, o_t), "rel_injected": rel(i_t, o_t),
           "oracle_scans_from_steady": o_s, "gpu_injected_scans_from_steady": i_s,
           "rel_injected_from_steady": rel(i_s, o_s),
           "scans_compared": len(keys_timed), "seeds": sorted({k[0] for k in keys_timed}),
           "tolerance": MATCH_TOL}
    ok = [abs(r) <= MATCH_TOL for r in (res["rel_injected"], res["rel_injected_from_steady"]) if r is not None]
    res["matched"] = bool(ok) and all(ok)
    res["note"] = ("matched: the GPU run injecting the oracle's random numbers has mean OSPA within 5 % of the "
                   "FP64 oracle's on the timed scans and on every scan from the steady window on; the timed run "
                   "(in-kernel Philox draws) is compared on the same scans for context")
    return res


def run_gpu(args, w, rank, world, local_rank, sub=False):
    """One-filter workloads through phd_step; returns the JSON line (rank 0) or None."""
    import torch
    from paper_1503_03769_gb300 import ParticlePHD

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    steps_per_run = w.steps
    # steady-state window: scans before `steady` of every run are replayed
    # untimed (all truth targets exist from 40 % of the run on)
    steady = args.steady_from if args.steady_from is not None else (50 if w.name.startswith("dense_rb_100t") else 0)
    per_run = steps_per_run - steady
    runs = max(1, math.ceil((args.warmup + args.steps) / per_run))
    base_seed = args.seed + 1000 * rank
    scen_cache = {}

    def scen_of(seed):
        if seed not in scen_cache:
            scen_cache[seed] = scenario.simulate(w, seed)
        return scen_cache[seed]

    scen = [scen_of(base_seed + r) for r in range(runs)]
    seq = [(r, k) for r in range(runs) for k in range(steady, steps_per_run)][: args.warmup + args.steps]
    dtype = torch.float64 if w.precision == "fp64" else torch.float32
    Zdev = {(r, k): torch.as_tensor(scen[r].meas[k], dtype=dtype, device=dev) for r, k in seq}

    f = ParticlePHD(w, seed=base_seed, device=f"cuda:{local_rank}")
    if args.path:
        f.set_path(args.path)
    empty_x = [np.zeros((0, 4))] * w.num_pe
    empty_w = [np.zeros(0)] * w.num_pe
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    cap = w.m_max

    # work of the untimed run heads, taken out of the counters (the stage
    # timer is off during them)
    head = {"pairs": 0, "pairs_evaluated": 0, "updates": 0, "launches": 0}
    head_phases = {}
    timer = {"on": False}

    def set_timer(on):
        timer["on"] = on
        f.set_stage_timer(on)

    def begin_run_if_needed(r, k):
        """Fresh filter at the run's first timed scan, the untimed head replayed."""
        if k == steady:
            f.set_state(empty_x, empty_w)
            if steady:
                s0 = f.stats()
                p0 = f.phase_times()
                f.set_stage_timer(False)
                f.run([scen[r].meas[q] for q in range(steady)], sync=False)
                s1 = f.stats()
                p1 = f.phase_times()
                f.set_stage_timer(timer["on"])
                for key in head:
                    head[key] += s1[key] - s0[key]
                for key in p1:
                    head_phases[key] = head_phases.get(key, 0.0) + p1[key] - p0[key]

    # set-up on the staged path: the pair passes' launch shape is autotuned
    # half-way through a run of the same workload, then the state is reset
    tuning = None
    if f.get_path() == "staged" and args.tuning:
        f.set_tuning(**args.tuning)
        tuning = {**{k: f.get_tuning()[k] for k in ("c_tile", "c_mb", "r_pb", "r_g", "grid1", "grid2", "gate", "order")},
                  "autotuned": False}
    elif f.get_path() == "staged" and not args.no_autotune:
        t_tune = time.perf_counter()
        tune_sc = scenario.simulate(w, base_seed + 7777, steps=steps_per_run // 2 + 1)
        for k in range(steps_per_run // 2):
            f.step(torch.as_tensor(tune_sc.meas[k], dtype=dtype, device=dev), cap=cap, sync=False)
        tuning = f.autotune(3)
        tuning = {**{k: tuning[k] for k in ("c_tile", "c_mb", "r_pb", "r_g", "grid1", "grid2", "gate", "order")},
                  "pass1_us": round(float(tuning["pass1_us"]), 2), "pass2_us": round(float(tuning["pass2_us"]), 2),
                  "setup_s": round(time.perf_counter() - t_tune, 3)}
        f.set_state(empty_x, empty_w)

    # warm-up (also captures the step graphs)
    set_timer(True)
    for r, k in seq[: args.warmup]:
        begin_run_if_needed(r, k)
        f.step(Zdev[(r, k)], cap=cap, sync=False)
    torch.cuda.synchronize()
    gpu_id = _gpu_id(local_rank)

    def timed_loop():
        f.reset_stats()
        for key in head:
            head[key] = 0
        head_phases.clear()
        evs = []
        est_log = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(gpu_id)
        clk.begin()
        nvtx_push("timed")
        for r, k in seq[args.warmup:]:
            begin_run_if_needed(r, k)
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            s, l, c = f.step(Zdev[(r, k)], cap=cap, sync=False)
            e1.record()
            evs.append((e0, e1))
            est_log.append((r, k, s.clone(), c.clone()))
        nvtx_pop()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = clk.end()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        st_ = f.stats()
        for key in head:
            st_[key] -= head[key]
        return ms, st_, clocks, est_log

    ms, st, clocks, est_log = timed_loop()
    if _bad_clocks(clocks):
        ms, st, clocks, est_log = timed_loop()
        clocks["remeasured"] = True

    pairs = st["pairs"]
    K = len(seq) - args.warmup
    # whole-job aggregation: sum of pairs over ranks, max time over ranks
    pairs_all, ms_max = job_totals(pairs, ms, world, dev)
    value = pairs_all / (ms_max * 1e-3)
    steps_per_s = world * K / (ms_max * 1e-3)

    # OSPA (c = 100, p = 2) of every timed scan against the truth
    timed_ospa = {}
    for r, k, s, c in est_log:
        timed_ospa[(base_seed + r, k)] = _ospa_of(s, c.item(), scen[r].truth[k])

    # roofline of the timed kernels: the fused step kernel (fused path) or the
    # update stage's kernels (staged path); one ex2 per pair, against the
    # device's measured ex2 rate
    path = f.get_path()
    peak = ex2_peak(local_rank)
    upd_ms = st["update_ms"]
    phases = None
    if path == "grid":
        # the step kernel's phase clock: the update is its spatial-order, pass-1,
        # normaliser and pass-2 phases (Eq. 7-8 with the order the passes walk)
        phases = {k: v - head_phases.get(k, 0.0) for k, v in f.phase_times().items()}
        step_ms = upd_ms
        upd_ms = sum(phases[k] for k in ("cell_starts", "scatter", "pass1", "normalisers", "pass2_ranks"))
    achieved = (pairs / (upd_ms * 1e-3)) / 1e12 if upd_ms > 0 else 0.0
    ev_frac = st["pairs_evaluated"] / pairs if pairs else None
    kname = {"fused": "k_step_fused (whole step, one CTA per PE)",
             "grid": "k_step_grid update phases (cell starts, scatter, pass 1, normalisers, pass 2 with the ranks)"
             }.get(path, UPDATE_KERNELS)
    roofline = {"bound": "alu", "kernel": kname,
                "achieved": achieved, "peak": peak["Texp_per_s"], "unit": "Texp/s",
                "frac": achieved / peak["Texp_per_s"], "traffic": _traffic_from_profile(path, w.name),
                "peak_source": "measured on this device: phd_measure_ex2_rate (burst; the kernel is timed alone)",
                "frac_evaluated": (achieved * ev_frac / peak["Texp_per_s"]) if ev_frac is not None else None,
                "frac_of_nominal": achieved / EX2_NOMINAL_TEXP,
                "kernel_ms_per_step": upd_ms / max(st["timed_updates"], 1),
                "pairs_per_update": pairs / max(st["updates"], 1),
                "pairs_evaluated_frac": ev_frac,
                "note": "achieved counts every particle x measurement pair (the metric's unit); pairs past "
                        "the exact likelihood gate contribute exactly 0 and are skipped (frac_evaluated counts "
                        "only the evaluated ones)"}
    if phases is not None:
        nt = max(st["timed_updates"], 1)
        roofline["traffic_scope"] = "DRAM bytes of one whole k_step_grid launch (one per step), from the ncu summary"
        roofline["step_kernel_ms_per_step"] = step_ms / nt
        roofline["phase_ms_per_step"] = {k: v / nt for k, v in phases.items()}
        _, pmax, _ = f.phase_times(detail=True)
        roofline["phase_longest_cta_ms"] = pmax

    # whole runs in one launch each (phd_run): S scans per call, L2 flushed
    # between runs (outside the events)
    run_ms, run_pairs, run_steps = 0.0, 0, 0
    by_run = {}
    for r, k in seq[args.warmup:]:
        by_run.setdefault(r, []).append(k)
    packed = {r: f.pack([Zdev[(r, k)] for k in ks]) for r, ks in by_run.items()}
    f.reset_stats()
    for r, ks in by_run.items():
        f.set_state(empty_x, empty_w)
        if ks[0] != 0:                   # a run the timed window entered mid-way: replay its head untimed
            f.run([scen[r].meas[k] for k in range(ks[0])], sync=False)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        before = f.stats()["pairs"]
        Zp, offt = packed[r]
        e0.record()
        f.run_packed(Zp, offt, len(ks), cap)
        e1.record()
        torch.cuda.synchronize()
        run_ms += e0.elapsed_time(e1)
        run_pairs += f.stats()["pairs"] - before
        run_steps += len(ks)

    # end to end through the public host-buffer call (pinned host memory)
    set_timer(False)
    Zhost = {key: torch.as_tensor(scen[key[0]].meas[key[1]], dtype=dtype).pin_memory().numpy()
             for key in seq}
    hs = torch.empty((cap, 4), dtype=dtype).pin_memory().numpy()
    hl = torch.empty(cap, dtype=torch.int32).pin_memory().numpy()
    f.reset_stats()
    e2e_s, h2d, d2h = 0.0, 0, 0
    for r, k in seq[: args.warmup]:
        begin_run_if_needed(r, k)
        f.step_host(Zhost[(r, k)], hs, hl)
    f.reset_stats()
    for key in head:
        head[key] = 0
    for r, k in seq[args.warmup:]:
        begin_run_if_needed(r, k)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = f.step_host(Zhost[(r, k)], hs, hl)
        e2e_s += time.perf_counter() - t0
        h2d += Zhost[(r, k)].nbytes
        d2h += min(n, cap) * (hs.itemsize * 4 + 4) + 4
    st2 = f.stats()
    e2e_pairs, e2e_max = job_totals(st2["pairs"] - head["pairs"], e2e_s, world, dev)
    e2e_val = e2e_pairs / e2e_max

    # matched OSPA: the oracle's stored record on the same seeds and scans,
    # and an untimed run with the oracle's own random numbers
    rec = oracle_record(w.name) if (w.gate_sigma == 0 and not args.no_matched) else None
    matched = None
    if rec is not None:
        seeds = sorted({sd for sd, _ in timed_ospa if sd in rec})
        if seeds:
            inj = injected_ospa(f, w, seeds, scen_of, dev)
            matched = matched_ospa(w, timed_ospa, inj, rec, steady)
    f.close()

    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_max / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {**workload_config(w, runs, "flushed between timed steps (512 MiB write, outside the events)"),
                   "timed_scans": f"{steady}..{w.steps - 1} of each run (earlier scans replayed untimed)"},
        "steps_per_s": steps_per_s,
        "path": path,
        "run_mode": {"api": "phd_run (one launch per run of scans)",
                     "value": run_pairs / (run_ms * 1e-3) if run_ms > 0 else None, "unit": UNIT,
                     "ms_per_step": run_ms / max(run_steps, 1), "steps": run_steps},
        "ospa_mean": float(np.mean(list(timed_ospa.values()))) if timed_ospa else None,
        "ospa_scans": len(timed_ospa),
        "matched_ospa": matched,
        "roofline": roofline,
        "ex2_peak": peak,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
                "d2h_bytes_per_step": d2h / K,
                "note": "phd_step_host: pinned host Z in, estimates + count out, synchronous per step"},
        "gpu_launches": int(st["launches"]),
        "clocks": clocks,
    }
    if tuning is not None:
        line["tuning"] = tuning
    if world == 1 and not args.no_cpu_baseline and not sub:
        budget = float(os.environ.get("PHD_CPU_BASELINE_S", "12"))
        line["cpu_baseline"] = cpu_baseline(w, args.seed, budget)
    return line


def run_gpu_batch(args, rank, world, local_rank):
    """The batched workload: 256 independent filters stepped together
    (phd_batch_step, one CUDA graph per batched step)."""
    import torch
    from paper_1503_03769_gb300 import ParticlePHDBatch

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ws = scenario.batch_workloads(seed=1000 + 7919 * rank, runs=args.runs)
    R = len(ws)
    steps_per_run = ws[0].steps
    total = args.warmup + args.steps
    scen = [scenario.simulate(w, 1000 + r + 7919 * rank, steps=steps_per_run) for r, w in enumerate(ws)]
    b = ParticlePHDBatch(ws, seed=1000 + rank, device=f"cuda:{local_rank}")
    if args.path:
        b.set_path(args.path)
    batch_path = b.get_path()
    packed = [b.pack([scen[r].meas[k] for r in range(R)]) for k in range(steps_per_run)]
    empty_x = [np.zeros((0, 4))] * R
    empty_w = [np.zeros(0)] * R
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    cap = 64
    states = torch.empty((R, cap, 4), dtype=torch.float32, device=dev)
    # set-up: the pair passes' launch shape is autotuned on the batch's own
    # slices half-way through a run (representative particle and measurement
    # counts), then the runs restart from empty
    t_tune = time.perf_counter()
    for k in range(steps_per_run // 2):
        b.batch_step(packed=packed[k % len(packed)], cap=cap, sync=False)
    if args.tuning:
        b.set_tuning(**args.tuning)
        tuning = b.get_tuning()
    else:
        tuning = b.autotune(5) if not args.no_autotune else b.get_tuning()
    t_tune = time.perf_counter() - t_tune
    b.set_state(empty_x, empty_w)
    b.set_stage_timer(True)
    for k in range(args.warmup):
        if k % steps_per_run == 0:
            b.set_state(empty_x, empty_w)
        b.batch_step(packed=packed[k % steps_per_run], cap=cap, sync=False)
    torch.cuda.synchronize()
    b.reset_stats()
    try:
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        gpu_id = str(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(gpu_id)
    clk.begin()
    evs = []
    logs = []   # (scan, states, counts) of every 4th scan of the runs begun in the warm-up
    nvtx_push("timed")
    for k in range(args.warmup, total):
        if k % steps_per_run == 0:
            b.set_state(empty_x, empty_w)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        s_, l_, c_ = b.batch_step(packed=packed[k % steps_per_run], cap=cap, sync=False)
        e1.record()
        evs.append((e0, e1))
        if k < steps_per_run and k % 4 == 0:
            logs.append((k, s_, c_))
    nvtx_pop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.end()
    per = [a.elapsed_time(c) for a, c in evs]
    ms = sum(per)
    st = b.stats()
    pairs = float(st["pairs"])
    pairs, ms = job_totals(pairs, ms, world, dev)
    upd_ms = st["update_ms"]
    b.close()
    # the same runs one at a time through the one-filter API (fused path where
    # a run fits, else staged): a sample of every 8th run over its whole 60
    # scans, L2 flushed between steps as above; OSPA of both on those runs
    from paper_1503_03769_gb300 import ParticlePHD
    sample = list(range(0, R, 8))
    one_ms, one_steps, one_ospa, paths = 0.0, 0, [], set()
    for r in sample:
        f = ParticlePHD(ws[r], seed=5000 + r + rank, device=f"cuda:{local_rank}")
        paths.add(f.get_path())
        Zr = [torch.as_tensor(z, dtype=torch.float32, device=dev) for z in scen[r].meas]
        evr, lg = [], []
        for k in range(steps_per_run):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            s1, l1, c1 = f.step(Zr[k], cap=cap, sync=False)
            e1.record()
            evr.append((e0, e1))
            if k >= args.warmup and k % 4 == 0:
                lg.append((k, s1.clone(), c1.clone()))
        torch.cuda.synchronize()
        one_ms += sum(a.elapsed_time(c) for a, c in evr)
        one_steps += len(evr)
        for k, s1, c1 in lg:
            n = int(c1.item())
            tr = scen[r].truth[k]
            one_ospa.append(ospa_metric(s1[:n].double().cpu().numpy()[:, [0, 2]] if n else np.zeros((0, 2)),
                                        tr[:, [0, 2]] if len(tr) else np.zeros((0, 2)), 100.0, 2.0))
        f.close()
    batch_ospa = []
    for k, s_, c_ in logs:
        if k < args.warmup:
            continue
        cn = c_.cpu().numpy()
        sn = s_.double().cpu().numpy()
        for r in sample:
            n = min(int(cn[r]), cap)
            tr = scen[r].truth[k]
            batch_ospa.append(ospa_metric(sn[r, :n][:, [0, 2]] if n else np.zeros((0, 2)),
                                          tr[:, [0, 2]] if len(tr) else np.zeros((0, 2)), 100.0, 2.0))
    one_rs = one_steps / (one_ms * 1e-3) if one_ms > 0 else None
    if rank != 0:
        return None
    achieved = (st["pairs"] / (upd_ms * 1e-3)) / 1e12 if upd_ms > 0 else 0.0
    peak = ex2_peak(local_rank)["Texp_per_s"]
    line = {
        "metric": METRIC, "value": pairs / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch256" if R == 256 else f"batch{R}", "runs": R, "scans_per_run": steps_per_run,
                   "targets": "U{1..50}", "clutter_rate": "U[5,200]", "particles_per_target": "U{256..4096}",
                   "births_per_step": "= particles per target", "pe_cap": ws[0].pe_cap,
                   "l2": "flushed between timed batched steps (512 MiB write, outside the events)",
                   "global_batch": R, "seq_len": steps_per_run, "parallelism": "replicas"},
        "run_steps_per_s": world * R * args.steps / (ms * 1e-3),
        "vs_one_filter_at_a_time": {
            "runs_sampled": len(sample), "paths": sorted(paths), "run_steps_per_s": one_rs,
            "speedup": (R * args.steps / (ms * 1e-3)) / one_rs if one_rs else None,
            "ospa_batch": float(np.mean(batch_ospa)) if batch_ospa else None,
            "ospa_one_at_a_time": float(np.mean(one_ospa)) if one_ospa else None,
            "note": "every 8th run of the batch stepped alone over its 60 scans; OSPA (c = 100 m, p = 2) "
                    "on every 4th scan of those runs, batch vs alone"},
        "per_run_latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
        "roofline": {"bound": "alu", "kernel": UPDATE_KERNELS,
                     "achieved": achieved, "peak": peak, "unit": "Texp/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": "measured on this device: phd_measure_ex2_rate",
                     "kernel_ms_per_step": upd_ms / max(st["timed_updates"], 1),
                     "pairs_per_update": st["pairs"] / max(st["updates"], 1),
                     "pairs_evaluated_frac": st["pairs_evaluated"] / st["pairs"] if st["pairs"] else None},
        "gpu_launches": int(st["launches"]), "clocks": clocks, "path": batch_path,
        "tuning": {**{k: tuning[k] for k in ("c_tile", "c_mb", "r_pb", "r_g", "grid1", "grid2", "gate", "order")},
                   "pass1_us": round(float(tuning["pass1_us"]), 2), "pass2_us": round(float(tuning["pass2_us"]), 2),
                   "autotuned": not (args.no_autotune or args.tuning), "setup_s": round(t_tune, 3)},
    }
    return line


def run_gpu_learned(args, rank, world, local_rank):
    """The learned-birth comparison (50 targets, range-bearing, clutter 100,
    1000 particles per target): plain birth with 5000 and 20000 birth
    particles and the trained measurement-driven proposal with 5000, each
    over the same scenarios; steps/s, pairs/s and OSPA (c = 100 m, p = 2)
    per variant.  Set-up (untimed): the birth network is trained by the
    library's kernels on two plain dense runs (100 targets, clutter 500)."""
    import torch
    from paper_1503_03769_gb300 import ParticlePHD, proposal

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    t0 = time.perf_counter()
    # birth intensity matched to the scenarios' truth birth rate (targets born
    # uniformly over the first 40 % of the scans); see the workload notes
    matched_nu = lambda w: w.n_targets / (0.4 * w.steps)
    wtrain = scenario.workload("dense_rb_100t")
    wtrain = wtrain.with_(birth_mass=matched_nu(wtrain))
    ft = ParticlePHD(wtrain, seed=2000 + rank, device=f"cuda:{local_rank}")
    Xs, Ts = [], []
    for s in (2000, 2001):
        X, T = proposal.collect_pairs(ft, scenario.simulate(wtrain, s + 7919 * rank).meas)
        Xs.append(X)
        Ts.append(T)
    ft.close()
    X, T = torch.cat(Xs), torch.cat(Ts)
    params, _ = proposal.train(X, T, steps=1500, batch=4096, lr=2e-3, seed=rank)
    loss = proposal.full_loss(params, X, T)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    w5 = scenario.workload("rb_50t")
    w5 = w5.with_(birth_mass=matched_nu(w5))
    variants = [("plain_J5000", w5, None)]
    variants += [(f"plain_J{J}", scenario.workload("rb_50t", birth_count=J, birth_mass=w5.birth_mass), None)
                 for J in (20000, 40000, 80000)]
    variants += [("learned_J5000", w5, params)]
    runs = max(1, -(-args.steps // w5.steps))   # OSPA is averaged over these runs: use several
    seeds = [3000 + r + 7919 * rank for r in range(runs)]
    scen = {s: scenario.simulate(w5, s) for s in seeds}
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    try:
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        gpu_id = str(local_rank)
    res, res_staged = {}, {}
    clocks = None
    # every variant on the library's default path for it, then all of them
    # again on the staged kernels (where the step's cost grows with the
    # particle count, so fewer birth particles buy speed)
    for (name, w, p), force in [(v, None) for v in variants] + [(v, "staged") for v in variants]:
        f = ParticlePHD(w, seed=11 + rank, device=f"cuda:{local_rank}")
        if p is not None:
            f.set_birth_proposal(p, 0.1)
        if force:
            f.set_path(force)
        path = f.get_path()
        Zd = {(s, k): torch.as_tensor(scen[s].meas[k], dtype=torch.float32, device=dev)
              for s in seeds for k in range(w.steps)}
        # warm-up run (graph capture), then the timed runs
        for k in range(min(args.warmup, w.steps)):
            f.step(Zd[(seeds[0], k)], sync=False)
        f.set_stage_timer(True)
        f.reset_stats()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(gpu_id)
        clk.begin()
        evs, logs = [], []
        for s in seeds:
            f.set_state([np.zeros((0, 4))] * f.K, [np.zeros(0)] * f.K)
            for k in range(w.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                st_, lb_, cnt = f.step(Zd[(s, k)], sync=False)
                e1.record()
                evs.append((e0, e1))
                logs.append((s, k, st_.clone(), cnt.clone()))
        torch.cuda.synchronize()
        c_ = clk.end()
        clocks = c_ if clocks is None or name == "learned_J5000" else clocks
        ms = sum(a.elapsed_time(b) for a, b in evs)
        st = f.stats()
        osp, card = [], []
        for s, k, st_, cnt in logs:
            n = int(cnt.item())
            est = st_[:n].double().cpu().numpy()[:, [0, 2]] if n else np.zeros((0, 2))
            tr = scen[s].truth[k]
            tr = tr[:, [0, 2]] if len(tr) else np.zeros((0, 2))
            osp.append(ospa_metric(est, tr, 100.0, 2.0))
            card.append(abs(len(est) - len(tr)))
        (res_staged if force else res)[name] = {"steps_per_s": len(evs) / (ms * 1e-3), "ms_per_step": ms / len(evs),
                     "pairs_per_s": st["pairs"] / (ms * 1e-3), "ospa_mean": float(np.mean(osp)),
                     "card_err_mean": float(np.mean(card)), "birth_count": w.birth_count,
                     "update_ms_per_step": st["update_ms"] / max(st["timed_updates"], 1),
                     "pairs": st["pairs"], "ms": ms, "launches": st["launches"], "steps": len(evs), "path": path}
        f.close()
    job_pairs, job_ms = job_totals(res["learned_J5000"]["pairs"], res["learned_J5000"]["ms"], world, dev)
    if rank != 0:
        return None
    L, P4 = res["learned_J5000"], res["plain_J20000"]
    matched = L["ospa_mean"] <= 1.05 * P4["ospa_mean"]

    def at_equal(rs):
        # the fastest plain-birth variant whose OSPA is within 5 % of the learned one's
        Ls = rs["learned_J5000"]
        eq = [k for k in rs if k.startswith("plain") and rs[k]["ospa_mean"] <= 1.05 * Ls["ospa_mean"]]
        best = max(eq, key=lambda k: rs[k]["steps_per_s"]) if eq else None
        return {"plain_variant": best,
                "steps_per_s_ratio": (Ls["steps_per_s"] / rs[best]["steps_per_s"]) if best else None,
                "note": "fastest plain-birth variant with OSPA within 5 % of the learned proposal's"}
    eq_default = at_equal(res)
    upd_s = L["update_ms_per_step"] * 1e-3
    achieved = (L["pairs"] / L["steps"]) / upd_s / 1e12 if upd_s > 0 else 0.0
    peak = ex2_peak(local_rank)["Texp_per_s"]
    line = {
        "metric": METRIC, "value": job_pairs / (job_ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": L["steps"],
        "warmup": args.warmup, "ms_per_step": L["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "rb_50t_learned", "targets": 50, "clutter_rate": 100.0, "sensor": "range-bearing",
                   "particles_per_target": 1000, "birth_count": 5000, "birth_mass": w5.birth_mass,
                   "runs": len(seeds), "scans_per_run": 100,
                   "l2": "flushed between timed steps (512 MiB write, outside the events)",
                   "global_batch": 1, "seq_len": 100, "parallelism": "replicas"},
        "steps_per_s": L["steps_per_s"],
        "variants": res,
        "learned_vs_plain_J20000": {"ospa_within_5pct": bool(matched),
                                    "steps_per_s_ratio": L["steps_per_s"] / P4["steps_per_s"]},
        "at_equal_ospa": eq_default,
        "staged_path": {"variants": res_staged, "at_equal_ospa": at_equal(res_staged),
                        "note": "the same variants on the staged kernels"},
        "training": {"pairs": int(X.shape[0]), "extracted_frac": float(T[:, 0].mean()), "adam_steps": 1500,
                     "loss": loss, "setup_s": round(t_train, 2)},
        "roofline": {"bound": "alu", "kernel": UPDATE_KERNELS if L["path"] == "staged" else
                     "k_step_grid (the whole step kernel)",
                     "achieved": achieved, "peak": peak, "unit": "Texp/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": "measured on this device: phd_measure_ex2_rate"},
        "gpu_launches": int(L["launches"]), "clocks": clocks,
    }
    return line


def _three_way(args, wd, seeds, dev, rank, local_rank, ospa_p, extra=()):
    """The paper's three filters on the same scenarios of workload wd: the
    global filter (PHD, all particles), the distributed scheme (DCPFPHD, wd's
    PEs, ring exchange, CU fusion) and the global filter on 1/K of the
    particles (partPHD), plus any `extra` (name, workload[, path]) variants;
    steps/s and OSPA (c = 100 m, order ospa_p) each."""
    import torch
    from paper_1503_03769_gb300 import ParticlePHD

    K = wd.num_pe
    # equal capacity: the global filter gets the K slices' slots, partPHD one slice's
    variants = [("PHD", wd.with_(num_pe=1, exchange_frac=0.0, pe_cap=K * wd.pe_cap)),
                ("DCPFPHD", wd),
                ("partPHD", wd.with_(num_pe=1, exchange_frac=0.0,
                                     particles_per_target=wd.particles_per_target // K,
                                     birth_count=wd.birth_count // K))] + list(extra)
    scen = {s_: scenario.simulate(wd, s_) for s_ in seeds}
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    res = {}
    for v in variants:
        name, w = v[0], v[1]
        f = ParticlePHD(w, seed=5 + rank, device=f"cuda:{local_rank}")
        if len(v) > 2:
            f.set_path(v[2])
        Zd = {(s_, k): torch.as_tensor(scen[s_].meas[k], dtype=torch.float32, device=dev)
              for s_ in seeds for k in range(w.steps)}
        for k in range(min(args.warmup, w.steps)):
            f.step(Zd[(seeds[0], k)], sync=False)
        f.reset_stats()
        torch.cuda.synchronize()
        evs, logs = [], []
        for s_ in seeds:
            f.set_state([np.zeros((0, 4))] * f.K, [np.zeros(0)] * f.K)
            for k in range(w.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                st_, lb_, cnt = f.step(Zd[(s_, k)], sync=False)
                e1.record()
                evs.append((e0, e1))
                logs.append((s_, k, st_.clone(), cnt.clone()))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        st = f.stats()
        osp = []
        for s_, k, st_, cnt in logs:
            n = int(cnt.item())
            est = st_[:n].double().cpu().numpy()[:, [0, 2]] if n else np.zeros((0, 2))
            tr = scen[s_].truth[k]
            osp.append(ospa_metric(est, tr[:, [0, 2]] if len(tr) else np.zeros((0, 2)), 100.0, ospa_p))
        res[name] = {"path": f.get_path(), "num_pe": w.num_pe, "particles_per_target": w.particles_per_target,
                     "birth_count": w.birth_count, "steps_per_s": len(evs) / (ms * 1e-3),
                     "ms_per_step": ms / len(evs), "pairs_per_s": st["pairs"] / (ms * 1e-3),
                     "ospa_mean": float(np.mean(osp)), "launches": st["launches"], "steps": len(evs),
                     "pairs": st["pairs"], "ms": ms}
        f.close()
    return res


def run_gpu_compare(args, rank, world, local_rank):
    """The paper's three-way comparison on the 16-PE workload (OSPA p = 2)."""
    import torch

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wd = scenario.workload("dist16_10t")
    K16 = wd.num_pe
    runs = max(1, -(-args.steps // wd.steps))
    seeds = [args.seed + r + 7919 * rank for r in range(runs)]
    # exchange variants (Step 6): all-to-all, and the ring only when a PE has
    # degenerated (its mass below half the PE mean)
    extra = [("DCPFPHD_grid", wd, "grid"),   # the PEs spread over the grid step kernel's CTAs
             ("DCPFPHD_all_to_all", wd.with_(exchange_mode="all")),
             ("DCPFPHD_adaptive_0.5", wd.with_(exchange_threshold=0.5)),
             # where the gap to the global filter comes from (Steps 2 and 6):
             # the normaliser (the PE mean of C^j instead of the local C^j),
             # the exchange, and the particles and births a PE holds
             ("DCPFPHD_ck_global", wd.with_(ck_mode="global")),
             ("DCPFPHD_no_exchange", wd.with_(exchange_frac=0.0)),
             ("DCPFPHD_4x_particles", wd.with_(particles_per_target=4 * wd.particles_per_target,
                                               birth_count=4 * wd.birth_count, pe_cap=4 * wd.pe_cap)),
             ("DCPFPHD_J_births_per_pe", wd.with_(birth_count=K16 * wd.birth_count))]
    res = _three_way(args, wd, seeds, dev, rank, local_rank, 2.0, extra)
    job_pairs, job_ms = job_totals(res["DCPFPHD"]["pairs"], res["DCPFPHD"]["ms"], world, dev)
    if rank != 0:
        return None
    D = res["DCPFPHD"]
    line = {
        "metric": METRIC, "value": job_pairs / (job_ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": D["steps"],
        "warmup": args.warmup, "ms_per_step": D["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "dist16_compare", "targets": wd.n_targets, "clutter_rate": wd.clutter_rate,
                   "runs": len(seeds), "scans_per_run": wd.steps, "birth_mass": wd.birth_mass,
                   "l2": "flushed between timed steps (512 MiB write, outside the events)",
                   "global_batch": 1, "seq_len": wd.steps, "parallelism": "replicas"},
        "steps_per_s": D["steps_per_s"], "variants": res,
        "speedup_vs_PHD": {k: res[k]["steps_per_s"] / res["PHD"]["steps_per_s"] for k in res},
        "gpu_launches": int(D["launches"]),
    }
    return line


def run_gpu_table1(args, rank, world, local_rank):
    """The paper's own scenario shape (Sec. 4: bearing-range sensor with a
    half-plane view over 200 m, Gaussian birth, p_S 0.9, p_D 1, 4 PEs of 200
    particles per target) at clutter rates 0, 10 and 20, PHD / DCPFPHD /
    partPHD each: steps/s and OSPA (c = 100 m, p = 1, the paper's order), the
    shape of Table 1 (context only: the paper's figures are MATLAB times)."""
    import torch

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    base = scenario.workload("paper_bot")
    runs = max(1, -(-args.steps // base.steps))
    seeds = [args.seed + r + 7919 * rank for r in range(runs)]
    table = {}
    for lam in (0.0, 10.0, 20.0):
        wd = base.with_(clutter_rate=lam)
        table[str(int(lam))] = _three_way(args, wd, seeds, dev, rank, local_rank, 1.0)
    job_pairs, job_ms = job_totals(table["10"]["DCPFPHD"]["pairs"], table["10"]["DCPFPHD"]["ms"], world, dev)
    if rank != 0:
        return None
    D = table["10"]["DCPFPHD"]
    line = {
        "metric": METRIC, "value": job_pairs / (job_ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": D["steps"],
        "warmup": args.warmup, "ms_per_step": D["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "paper_table1", "targets": base.n_targets, "clutter_rates": [0, 10, 20],
                   "num_pe": base.num_pe, "particles_per_target_per_pe": base.particles_per_target // base.num_pe,
                   "runs": len(seeds), "scans_per_run": base.steps, "birth_mass": base.birth_mass,
                   "ospa": {"c": 100.0, "p": 1.0},
                   "l2": "flushed between timed steps (512 MiB write, outside the events)",
                   "global_batch": 1, "seq_len": base.steps, "parallelism": "replicas"},
        "steps_per_s": D["steps_per_s"],
        "table": {lam: {k: {"steps_per_s": v["steps_per_s"], "ospa_mean": v["ospa_mean"], "path": v["path"]}
                        for k, v in arms.items()} for lam, arms in table.items()},
        "gpu_launches": int(D["launches"]),
    }
    return line


def _parse_tuning(text):
    keys = ("c_tile", "c_mb", "r_pb", "r_g", "grid1", "grid2", "gate", "order")
    out = {}
    for part in text.split(","):
        k, _, v = part.partition("=")
        if k.strip() not in keys:
            raise argparse.ArgumentTypeError(f"unknown tuning key {k!r}; known: {', '.join(keys)}")
        out[k.strip()] = int(v)
    return out


def nvtx_push(name):
    """NVTX range around a timed region (lets a profiler select its kernels)."""
    import torch
    try:
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    import torch
    try:
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def _compact(line, keys):
    return {k: line[k] for k in keys if k in line}


def compact_one(line):
    """Sub-block of a one-filter workload's line."""
    out = _compact(line, ("value", "unit", "steps", "ms_per_step", "steps_per_s", "path", "ospa_mean", "gpu_launches"))
    out["workload"] = line["config"]["workload"]
    out["roofline"] = _compact(line["roofline"], ("frac", "achieved", "peak", "unit", "frac_evaluated",
                                                  "kernel_ms_per_step", "pairs_per_update", "traffic"))
    out["e2e"] = _compact(line["e2e"], ("value", "unit"))
    out["run_mode"] = _compact(line["run_mode"], ("value", "ms_per_step"))
    if line.get("matched_ospa"):
        out["matched_ospa"] = _compact(line["matched_ospa"], ("matched", "oracle_timed_scans", "gpu_timed",
                                                              "gpu_injected_timed_scans", "rel_injected",
                                                              "rel_injected_from_steady", "rel_gpu_timed"))
    out["clocks"] = _compact(line["clocks"], ("sm_mhz", "reasons"))
    return out


def compact_batch(line):
    out = _compact(line, ("value", "unit", "steps", "ms_per_step", "run_steps_per_s", "per_run_latency_ms",
                          "vs_one_filter_at_a_time", "gpu_launches", "path"))
    out["workload"] = line["config"]["workload"]
    out["roofline"] = _compact(line["roofline"], ("frac", "achieved", "peak", "unit", "kernel_ms_per_step",
                                                  "pairs_evaluated_frac"))
    out["tuning"] = line.get("tuning")
    out["clocks"] = _compact(line["clocks"], ("sm_mhz", "reasons"))
    return out


def compact_learned(line):
    out = _compact(line, ("value", "unit", "steps", "ms_per_step", "steps_per_s", "learned_vs_plain_J20000",
                          "at_equal_ospa", "gpu_launches"))
    out["workload"] = line["config"]["workload"]
    out["variants"] = {k: _compact(v, ("steps_per_s", "ospa_mean", "card_err_mean", "birth_count", "path"))
                       for k, v in line["variants"].items()}
    sp = line.get("staged_path")
    if sp:
        out["staged_path"] = {"at_equal_ospa": sp["at_equal_ospa"],
                              "variants": {k: _compact(v, ("steps_per_s", "ospa_mean"))
                                           for k, v in sp["variants"].items()}}
    out["training"] = _compact(line["training"], ("pairs", "loss", "adam_steps", "setup_s"))
    out["roofline"] = _compact(line["roofline"], ("frac", "achieved", "peak", "unit"))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--runs", type=int, default=256, help="filters in the batched workload (batch256)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape of the pair passes")
    ap.add_argument("--path", default=None, choices=["staged", "fused", "grid"],
                    help="run the one-filter or batched workload on this path instead of the library's default")
    ap.add_argument("--steady-from", type=int, default=None,
                    help="time scans from this index of every run (earlier ones replayed untimed); "
                         "default 50 for dense_rb_100t, else 0")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-subblocks", action="store_true",
                    help="default workload only: leave out the 16-PE, batch and learned-birth sub-blocks")
    ap.add_argument("--no-matched", action="store_true", help="skip the matched-OSPA run against the oracle record")
    ap.add_argument("--gate-sigma", type=float, default=0.0,
                    help="likelihood truncation beyond this many standard deviations (a variant that "
                         "changes results; 0 = the exact likelihood)")
    ap.add_argument("--tuning", type=_parse_tuning, default=None,
                    help="fixed launch shape of the pair passes instead of autotuning, "
                         "e.g. c_tile=512,c_mb=4,r_pb=1,r_g=1,grid1=1216,grid2=608,gate=1,order=1")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    world = _env_int("WORLD_SIZE", 1)
    rank, local_rank = _env_int("RANK", 0), _env_int("LOCAL_RANK", 0)
    special = {"paper_table1": run_gpu_table1, "dist16_compare": run_gpu_compare,
               "rb_50t_learned": run_gpu_learned, "batch256": run_gpu_batch}
    if args.impl == "reference":
        w = scenario.workload({"batch256": "linear4_fp64", "rb_50t_learned": "rb_50t", "paper_table1": "paper_bot",
                               "dist16_compare": "dist16_10t"}.get(args.workload, args.workload))
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend="gloo")
        try:
            return run_reference(args, w, rank, world)
        finally:
            if world > 1:
                import torch.distributed as dist
                dist.destroy_process_group()
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group(backend="nccl")
    try:
        if args.workload in special:
            line = special[args.workload](args, rank, world, local_rank)
        else:
            w = scenario.workload(args.workload)
            if args.gate_sigma > 0:
                w = w.with_(gate_sigma=args.gate_sigma)
            line = run_gpu(args, w, rank, world, local_rank)
            if args.workload == DEFAULT_WORKLOAD and not args.no_subblocks:
                sub_args = argparse.Namespace(**{**vars(args), "steady_from": None, "tuning": None})
                subs = {}
                t0 = time.perf_counter()
                l2 = run_gpu(sub_args, scenario.workload("dist16_10t"), rank, world, local_rank, sub=True)
                lb = run_gpu_batch(sub_args, rank, world, local_rank)
                ll = run_gpu_learned(sub_args, rank, world, local_rank)
                if rank == 0:
                    subs["dist16_10t"] = compact_one(l2)
                    subs["batch256"] = compact_batch(lb)
                    subs["rb_50t_learned"] = compact_learned(ll)
                    line["subblocks"] = {**subs, "seconds": round(time.perf_counter() - t0, 1),
                                         "note": "the 16-PE distributed workload, the 256-run batch and the "
                                                 "learned birth proposal, each measured as its own --workload "
                                                 "run measures it; compact"}
        if rank == 0 and line is not None:
            print(json.dumps(line), flush=True)
        return 0
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
