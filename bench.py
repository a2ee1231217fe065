#!/usr/bin/env python3
"""Benchmark of the ECC hot path: line-pair samples per second on one GB300.

Workload (default): the 496-view, 200-degree short scan (620x480 detector, 0.6 mm
pixels, SID 750 / SDD 1200 mm, 40 seeded ellipsoids), 768x768 dRadon/ds grid,
512 plane angles per pair, all 122,760 view pairs.  One step is the whole path on
inputs resident in HBM: per-view set-up, the dRadon/ds precompute of every view,
the pair set-up and the pair x kappa gather-reduce down to the total.  One unit
is one (pair, kappa) sample with both look-ups.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun with N > 1 every rank runs its own
independent copy of the workload (weak scaling; no data-path collective).  Besides
the contract's keys the line carries the per-kernel shares, the evaluation alone
(FP32 storage), the same evaluation on FP16 and BF16 sinograms against the FP32
total ("storage_forms"), the motion and calibration gradients on the same
sinograms ("adjoint_forms"), and the served form with p50/p99 latency ("serving").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "ECC line-pair samples/s"
UNIT = "line-pair samples/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
L1_PEAK_TBS = 128.0 * 152 * 2.07e9 / 1e12  # L1 data bytes per second (unit counts x max SM clock)
# FP32 work of one Joseph tap written directly: position x0 + k dx (an FMA, 2 FLOP), floor
# and fraction (2), the lerp v0 + f (v1 - v0) (a subtraction and an FMA, 3), accumulate (1)
FLOPS_PER_TAP = 8


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2", choices=["c2"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving (continuous batching) leg")
    ap.add_argument("--no-adjoint-forms", action="store_true",
                    help="skip the gradient legs (motion gradient and calibration gradient on the same sinograms)")
    ap.add_argument("--no-storage-forms", action="store_true",
                    help="skip the FP16/BF16 sinogram storage leg (evaluation against the FP32 form)")
    ap.add_argument("--no-c4", dest="c4_leg", action="store_false",
                    help="skip the precision leg (1240-view 976x976 scan, FP16/BF16 sinograms, 1024 kappa)")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: one job over all ranks (view slices + all-gather of the sinograms, pair tiles + "
                         "FP64 all-reduce; strong scaling) instead of one independent job per rank (weak scaling)")
    ap.add_argument("--ref-stride", type=int, default=3,
                    help="reference arm: the pairs timed per step are those among every ref-stride-th view")
    ap.add_argument("--serve-jobs", type=int, default=24, help="jobs of the serving leg")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="mean Poisson arrival rate [jobs/s]")
    ap.add_argument("--views", type=int, default=0,
                    help="use the first N views of the workload (smaller case for profiling); 0 = all")
    return ap.parse_args(argv)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def workload_config(cfg):
    return {
        "workload": (f"{cfg.name}: {cfg.n_views}-view {cfg.arc_deg:g}-degree short scan, {cfg.W}x{cfg.H} detector "
                     f"({cfg.pixel_mm} mm), {cfg.n_prim} seeded ellipsoids, {cfg.n_alpha}x{cfg.n_s} dRadon/ds, "
                     f"{cfg.K} kappa, all {cfg.n_pairs} pairs; step = dRadon/ds precompute + ECC evaluation"),
        "n_views": cfg.n_views, "n_pairs": cfg.n_pairs, "n_kappa": cfg.K, "n_alpha": cfg.n_alpha, "n_s": cfg.n_s,
        "detector": [cfg.W, cfg.H],
        "l2": "inputs larger than L2 (projections 590 MB, sinograms 1.17 GB > 135 MB L2); no flush",
        "parallelism": "independent replicas per GPU",
    }


def joseph_taps(cfg) -> int:
    """Taps of the Joseph line sums that fall inside the image (algorithmic work of
    the dRadon/ds precompute): per line, the integer steps where the interpolation
    coordinate lies in (-1, limit)."""
    W, H, n_alpha, n_s = cfg.W, cfg.H, cfg.n_alpha, cfg.n_s
    ds = np.hypot(W, H) / (n_s - 1)
    cx, cy = 0.5 * (W - 1), 0.5 * (H - 1)
    m = np.arange(n_alpha)
    a = m * np.pi / n_alpha
    ca, sa = np.cos(a), np.sin(a)
    rows = (4 * m <= n_alpha) | (4 * m >= 3 * n_alpha)
    sig = (np.arange(n_s + 1) - 0.5 * n_s) * ds
    total = 0
    for i in range(n_alpha):
        if rows[i]:
            x0 = cx + (sig + cy * sa[i]) / ca[i]
            d, n_steps, limit = -sa[i] / ca[i], H, W
        else:
            x0 = cy + (sig + cx * ca[i]) / sa[i]
            d, n_steps, limit = -ca[i] / sa[i], W, H
        if abs(d) < 1e-12:
            cnt = np.where((x0 > -1) & (x0 < limit), n_steps, 0)
        else:
            t1, t2 = (-1 - x0) / d, (limit - x0) / d
            lo, hi = np.minimum(t1, t2), np.maximum(t1, t2)
            first = np.maximum(np.floor(lo) + 1, 0)
            last = np.minimum(np.ceil(hi) - 1, n_steps - 1)
            cnt = np.maximum(last - first + 1, 0)
        total += int(cnt.sum())
    return total * cfg.n_views


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", self.gpu_id],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(pg, x: float, device) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ serving leg
SERVE_DETECTORS = {  # detector -> (W, H, pixel mm, n_alpha, n_s, ellipsoids of the pool phantom)
    "256x256": (256, 256, 1.0, 256, 363, 12),
    "620x480": (620, 480, 0.6, 768, 768, 40),
    "976x976": (976, 976, 0.3, 1024, 1382, 16),
}


def serving_leg(args, c2_scan):
    """Poisson stream of motion-compensation jobs through ecc_submit / ecc_poll.

    Jobs (seeded): detector uniform over the three sizes, views U{50..500}, kappa
    U{256..1024}, FP16 sinogram storage, 20 gradient iterations, initial motion
    rotations N(0, 1 deg) and translations N(0, 2 mm).  Each detector size has one
    seeded ellipsoid phantom scanned over 500 views (the 620x480 one is the timed
    short scan); a job takes a contiguous run of its views (a sub-arc), so job inputs
    are slices of pinned host pools.  Wall time runs from the first submission to
    the last result on the host; throughput counts every job's line-pair samples
    (pairs x kappa x 21 evaluations)."""
    import torch
    import synth
    import paper_1806_02637_gb300 as ecc
    rng = np.random.default_rng(20)
    pools = {}
    for name, (W, H, px, na, ns, nprim) in SERVE_DETECTORS.items():
        if name == "620x480":
            sc = c2_scan
        else:
            cfg = synth.ScanConfig(f"serve{W}", n_views=500, arc_deg=200.0, full_scan=False, W=W, H=H, pixel_mm=px,
                                   n_prim=nprim, n_alpha=na, n_s=ns, seed=7000 + W)
            sc = synth.make_scan(cfg)
        pools[name] = (torch.from_numpy(np.ascontiguousarray(sc["P"])).pin_memory(),
                       torch.from_numpy(np.ascontiguousarray(sc["images"])).pin_memory())
    names = list(SERVE_DETECTORS)
    jobs = []
    t_arr = np.cumsum(rng.exponential(1.0 / args.serve_rate, args.serve_jobs))
    for i in range(args.serve_jobs):
        det = names[int(rng.integers(0, 3))]
        P_pool, I_pool = pools[det]
        n = int(rng.integers(50, 501))
        n = min(n, P_pool.shape[0])
        s0 = int(rng.integers(0, P_pool.shape[0] - n + 1))
        K = int(rng.integers(256, 1025))
        th = np.zeros((n, 6))
        th[:, :3] = np.deg2rad(rng.normal(0.0, 1.0, (n, 3)))
        th[:, 3:] = rng.normal(0.0, 2.0, (n, 3))
        jobs.append((t_arr[i], det, P_pool[s0:s0 + n], I_pool[s0:s0 + n], K, th))
    ctx = ecc.Context(0)
    iters, step = 20, 1e-6
    pending, results = {}, {}
    t0 = time.perf_counter()
    k = 0
    while k < len(jobs) or pending:
        now = time.perf_counter() - t0
        while k < len(jobs) and jobs[k][0] <= now:
            _, det, P, I, K, th = jobs[k]
            W, H, _, na, ns, _ = SERVE_DETECTORS[det]
            pending[k] = ecc.ecc_submit(ctx, P, I, W, H, na, ns, K, n_iters=iters, step=step, dtype="float16",
                                        motion0=th)
            k += 1
        for j, t in list(pending.items()):
            r = ecc.ecc_poll(ctx, t)
            if r is not None:
                r["t_done"] = time.perf_counter() - t0
                results[j] = r
                del pending[j]
        time.sleep(0.0005)
    wall = max(r["t_done"] for r in results.values()) - t_arr[0]
    st = ecc.ecc_serve_stats(ctx)
    dev_t = ecc.ecc_serve_times(ctx)
    lat = np.array([results[j]["latency_ms"] for j in sorted(results)])
    que = np.array([results[j]["queue_ms"] for j in sorted(results)])
    lp = sum(r["line_pairs"] for r in results.values())
    # accuracy of the served FP16 form: the two smallest jobs' first totals against the
    # plain FP32 form (precompute + ecc_evaluate at the same motion) on the same GPU
    small = sorted(range(len(jobs)), key=lambda j: jobs[j][2].shape[0] * jobs[j][4])[:2]
    acc = []
    for j in small:
        _, det, P, I, K, th = jobs[j]
        W, H, _, na, ns, _ = SERVE_DETECTORS[det]
        Pd = P.cuda()
        S, _ = ecc.ecc_precompute_radon_derivative(ctx, Pd, I.cuda(), na, ns)
        ref = float(ecc.ecc_evaluate(ctx, Pd, S, W, H, K, motion=torch.from_numpy(th).cuda(),
                                     want_per_pair=False)["total"].cpu()[0])
        acc.append(abs(results[j]["total_first"] - ref) / abs(ref))
    # two jobs' first totals against the FP64 oracle (its own dRadon/ds of the job's views): the two
    # with the least dRadon/ds work for the oracle (views x detector pixels)
    from oracle import oracle as orc
    acc_or = []
    small_or = sorted(range(len(jobs)), key=lambda j: jobs[j][3].shape[0] * jobs[j][3].shape[1] * jobs[j][3].shape[2])[:2]
    for j in small_or:
        _, det, P, I, K, th = jobs[j]
        W, H, _, na, ns, _ = SERVE_DETECTORS[det]
        Pn = P.numpy().astype(np.float64)
        S_or = orc.radon_derivative(Pn, I.numpy(), na, ns)
        ref = orc.ecc(Pn, S_or, W, H, K, motion=th)["total"]
        acc_or.append(abs(results[j]["total_first"] - ref) / abs(ref))
    # the same jobs, one after the other, through plain calls on one stream: upload,
    # precompute, n_iters x (ecc_evaluate_grad, step), final ecc_evaluate.  Two passes:
    # the first also pays one-time costs (first allocations of each job shape, first
    # launches; about a second after the served run); the second is reported.
    plain_passes = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _, det, P, I, K, th in jobs:
            W, H, _, na, ns, _ = SERVE_DETECTORS[det]
            Pd, Id = P.cuda(non_blocking=True), I.cuda(non_blocking=True)
            S, scales = ecc.ecc_precompute_radon_derivative(ctx, Pd, Id, na, ns, dtype=torch.float16)
            del Id
            theta = torch.from_numpy(th).cuda()
            for _ in range(iters):
                g = ecc.ecc_evaluate_grad(ctx, Pd, S, W, H, K, motion=theta, scales=scales, want_per_pair=False)["grad"]
                theta -= step * g
            ecc.ecc_evaluate(ctx, Pd, S, W, H, K, motion=theta, scales=scales, want_per_pair=False)
            del S, scales
        torch.cuda.synchronize()
        plain_passes.append(time.perf_counter() - t0)
    plain_s = plain_passes[-1]
    ctx.close()
    return {"metric": "ECC line-pair samples/s, served (FP16 storage, with gradients)", "value": lp / wall,
            "unit": UNIT, "jobs": len(results), "wall_s": wall, "arrival_rate_per_s": args.serve_rate,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "queue_ms": {"p50": float(np.percentile(que, 50)), "p99": float(np.percentile(que, 99))},
            "rounds": st["rounds"], "mean_jobs_per_round": st["job_rounds"] / max(1, st["rounds"]),
            "device_time_ms": dev_t,
            "shares_of_wall": {"upload": dev_t["upload_ms"] / 1e3 / wall, "precompute": dev_t["precompute_ms"] / 1e3 / wall,
                               "rounds": dev_t["round_ms"] / 1e3 / wall,
                               "note": "device time of each part over the wall time; admissions overlap rounds, so "
                                       "the parts may sum above 1"},
            "plain_calls_same_jobs": {"value": lp / plain_s, "unit": UNIT, "wall_s": plain_s,
                                      "first_pass_wall_s": plain_passes[0],
                                      "how": "the same jobs back to back, no arrival process: upload, precompute, "
                                             f"{iters} x (ecc_evaluate_grad + step), ecc_evaluate, one stream; "
                                             "second of two passes (the first also pays one-time allocations and "
                                             "launches)"},
            "max_jobs_per_round": st["max_batch"], "iterations_per_job": iters, "step": step,
            "fp16_vs_fp32_total_rel_err": {"jobs": len(acc), "max": float(max(acc)) if acc else None},
            "fp16_vs_oracle_total_rel_err": {"jobs": len(acc_or), "max": float(max(acc_or)) if acc_or else None,
                                             "how": "first totals (at the initial motion) of the two jobs with the "
                                                    "fewest view pixels, against the FP64 oracle on its own dRadon/ds "
                                                    "of the job's views"},
            "jobs_mix": "detector uniform {256^2, 620x480, 976^2}, views U{50..500}, kappa U{256..1024}, "
                        "FP16 storage, 20 gradient iterations + final evaluation, Poisson arrivals",
            "wall_includes": "admission (H2D of projections from pinned host pools, dRadon/ds precompute) and "
                             "all iterations; arrivals exceed the device's capacity, so latency includes queueing"}


# ------------------------------------------------------------------ CPU baseline
def oracle_energies(orc, P, S, W, H, K, pairs):
    """E_ab of each pair (reading R10): the mean of (S_a^2 + S_b^2) / 2 over the pair's
    valid planes, from the oracle with zero-sinogram copies of the views."""
    n = S.shape[0]
    P2 = np.concatenate([P, P])
    S2 = np.concatenate([S, np.zeros_like(S)])
    pairs = np.asarray(pairs)
    ea = orc.ecc(P2, S2, W, H, K, pairs=np.stack([pairs[:, 0], pairs[:, 1] + n], axis=1))["d"]
    eb = orc.ecc(P2, S2, W, H, K, pairs=np.stack([pairs[:, 0] + n, pairs[:, 1]], axis=1))["d"]
    return 0.5 * (ea + eb)


def error_stats(d, d_ref, E, total, total_ref):
    """Errors of one result against the FP64 oracle: per pair plain |dd| / d and with
    reading R10's floor |dd| / max(d, 1e-2 E); the total plain."""
    d, d_ref = np.asarray(d, dtype=np.float64), np.asarray(d_ref, dtype=np.float64)
    plain = np.abs(d - d_ref) / np.maximum(d_ref, 1e-300)
    floored = np.abs(d - d_ref) / np.maximum(d_ref, 1e-2 * np.asarray(E))
    q = lambda x: {"max": float(x.max()), "p99": float(np.percentile(x, 99)), "median": float(np.median(x))}
    return {"pairs": int(d.size), "pair_plain": q(plain), "pair_floored": q(floored),
            "total_rel_err": float((total - total_ref) / total_ref)}


def oracle_job(cfg, scan, n_threads: int):
    """The oracle on the whole job: dRadon/ds of every view and the ECC of every pair,
    each timed (FP64, n_threads host threads)."""
    from oracle import oracle as orc
    t0 = time.perf_counter()
    S = orc.radon_derivative(scan["P"], scan["images"], cfg.n_alpha, cfg.n_s, n_threads=n_threads)
    t1 = time.perf_counter()
    r = orc.ecc(scan["P"], S, cfg.W, cfg.H, cfg.K, n_threads=n_threads)
    t2 = time.perf_counter()
    return S, r, t1 - t0, t2 - t1


def reference_sample(cfg, stride=3):
    """The views and pairs one step of the reference arm times: the dRadon/ds of 8 views
    (a different 8 each step, over the whole scan) and the ECC of all pairs among every
    stride-th view (stride 3: 166 views, 13,695 pairs), whose sinograms the oracle
    computes once before the steps."""
    pv = np.arange(0, cfg.n_views, stride)
    return pv, synth.upper_pairs(len(pv))


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores, on the same
    workload.  A step times a bounded sample (reference_sample) and the rate is
    extrapolated per view and per pair to the whole job; ms_per_step is the measured
    time of one step's sample, so steps x ms_per_step is the time actually measured."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as orc
    cfg = synth.CONFIGS[args.workload]
    scan = synth.make_scan(cfg)
    cores = os.cpu_count() or 1
    pv, pairs = reference_sample(cfg, args.ref_stride)
    S_pv = orc.radon_derivative(scan["P"][pv], scan["images"][pv], cfg.n_alpha, cfg.n_s, n_threads=cores)
    nv_step = 8
    t_radon = t_ecc = 0.0
    sample_s = []
    for it in range(args.warmup + args.steps):
        views = (it * nv_step + np.arange(nv_step) * (cfg.n_views // nv_step)) % cfg.n_views
        t0 = time.perf_counter()
        orc.radon_derivative(scan["P"][views], scan["images"][views], cfg.n_alpha, cfg.n_s, n_threads=cores)
        t1 = time.perf_counter()
        orc.ecc(scan["P"][pv], S_pv, cfg.W, cfg.H, cfg.K, pairs=pairs, n_threads=cores)
        t2 = time.perf_counter()
        if it >= args.warmup:
            t_radon += t1 - t0
            t_ecc += t2 - t1
            sample_s.append(t2 - t0)
    per_view = t_radon / (args.steps * nv_step)
    per_pair = t_ecc / (args.steps * len(pairs))
    job_s = per_view * cfg.n_views + per_pair * cfg.n_pairs
    value = cfg.n_pairs * cfg.K / job_s
    sample = (f"per step: dRadon/ds of {nv_step} of the {cfg.n_views} views (a different {nv_step} each step) and the "
              f"ECC of the {len(pairs)} pairs among one view in {args.ref_stride}, on {cores} host threads; measured "
              f"{per_view:.3f} s per view and {per_pair * 1e3:.4f} ms per pair over {args.steps} steps "
              f"({t_radon:.2f} s + {t_ecc:.2f} s), extrapolated to the whole job ({job_s:.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(sample_s),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "extrapolated": True,
            "sample_per_step": {"views_radon": nv_step, "pairs_ecc": int(len(pairs)), "n_kappa": cfg.K},
            "config": workload_config(cfg),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def wall_ms(fn, reps):
    """Mean time of fn() over reps calls, CUDA events on the current stream around the
    calls (the pair set-up of later pair chunks overlaps earlier chunks' pair kernels on
    a second stream, so summed kernel times overstate a call)."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        fn()
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / reps


# ------------------------------------------------------------------ storage forms
def storage_forms(ctx, P, images, cfg, total_f32, reps=10, oracle=None, l2_gbs=None):
    """The reduced-precision form: the same scan's sinograms stored in FP16 (per-view
    scale) and BF16, then the evaluation of all pairs timed as in the FP32 form (the
    library's CUDA events, inputs resident).  Reports line-pair samples/s of the
    evaluation, the pair kernel against HBM and L2 at 16 B per line pair, the total's
    relative difference from the plain FP32 form on the same GPU, and (with the
    oracle's result of the job) every pair's and the total's error against the FP64
    oracle."""
    import torch
    import paper_1806_02637_gb300 as ecc
    units = cfg.n_pairs * cfg.K
    peaks = measured_peaks()
    out = {}
    for name, dt in (("float16", torch.float16), ("bfloat16", torch.bfloat16)):
        S, scales = ecc.ecc_precompute_radon_derivative(ctx, P, images, cfg.n_alpha, cfg.n_s, dtype=dt)
        tot = torch.empty((1,), dtype=torch.float64, device=S.device)
        for _ in range(3):
            ecc.ecc_evaluate(ctx, P, S, cfg.W, cfg.H, cfg.K, scales=scales, total=tot, want_per_pair=False)
        torch.cuda.synchronize()
        ecc.ecc_profile_read(ctx)
        ecc.ecc_profile_enable(ctx, True)
        for _ in range(reps):
            ecc.ecc_evaluate(ctx, P, S, cfg.W, cfg.H, cfg.K, scales=scales, total=tot, want_per_pair=False)
        torch.cuda.synchronize()
        prof = ecc.ecc_profile_read(ctx)
        ecc.ecc_profile_enable(ctx, False)
        eval_ms = wall_ms(lambda: ecc.ecc_evaluate(ctx, P, S, cfg.W, cfg.H, cfg.K, scales=scales, total=tot,
                                                   want_per_pair=False), reps)
        pk_ms = prof["ecc_pair_kernel"][1] / reps   # all chunks of one evaluation
        gbs = 16.0 * units / (pk_ms / 1e3) / 1e9
        t = float(tot.cpu()[0])
        out[name] = {"ms_per_eval": eval_ms, "line_pairs_per_s": units / (eval_ms / 1e3), "pair_kernel_ms": pk_ms,
                     "pair_kernel_gather_gbs": gbs, "pair_kernel_frac_of_hbm": gbs / peaks.get("hbm_gbs", 6800.0),
                     "pair_kernel_frac_of_l2": gbs / l2_gbs if l2_gbs else None,
                     "total": t, "total_rel_diff_vs_f32": abs(t - total_f32) / abs(total_f32)}
        if oracle is not None:
            r = ecc.ecc_evaluate(ctx, P, S, cfg.W, cfg.H, cfg.K, scales=scales)
            out[name]["vs_oracle"] = error_stats(r["per_pair"][:, 0].cpu().numpy(), oracle["d"], oracle["E"],
                                                 float(r["total"].cpu()[0]), oracle["total"])
        del S, scales
    out["note"] = ("evaluation only (view/pair set-up, pair kernel, reduction), 16 B per line pair for the gather; "
                   "the sinograms come from the same precompute in the stated storage type; vs_oracle: every pair "
                   "against the FP64 oracle's result of the job (pair_floored uses reading R10's 1e-2 E_ab floor)")
    return out


def l2_read_rate(dev, sizes_mb=(32, 64, 96), reps=20):
    """Read rate of a buffer resident in L2 (129 MB), the denominator of the L2
    fractions: the library's diagnostic read kernel (16-byte loads that skip L1, 8
    blocks per SM), CUDA events around `reps` launches; the best of three sizes."""
    import ctypes
    import paper_1806_02637_gb300 as ecc
    lib = ecc.load()
    lib.ecc_internal_l2_read_rate.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.ecc_internal_l2_read_rate.restype = ctypes.c_int
    rates = {}
    for mb in sizes_mb:
        g = ctypes.c_double(0.0)
        if lib.ecc_internal_l2_read_rate(ctypes.c_size_t(mb << 20), reps, ctypes.byref(g)) == 0:
            rates[f"{mb}MB"] = g.value
    best = max(rates.values()) if rates else float("nan")
    return {"gbs": best, "by_size_gbs": rates,
            "how": f"L2-resident buffers read with ld.global.cg float4 (about 1 GB per launch), 8 blocks per SM, "
                   f"{reps} launches, CUDA events"}


# ------------------------------------------------------------------ precision leg (1240-view scan)
def c4_leg(ctx, l2_gbs, reps=5):
    """The precision workload: 1240 views over 360 degrees, 976x976 detector (0.3 mm),
    60 seeded ellipsoids, 1024 x 1382 dRadon/ds stored in FP16 and BF16 (and FP32 for
    comparison), 1024 kappa, all 768,180 pairs.  Times the precompute and the evaluation
    (the library's CUDA events, inputs resident), the pair kernel's algorithmic bytes (16 B
    per line pair in FP16/BF16, 32 B in FP32) against HBM and L2, and the oracle: the
    dRadon/ds of 16 seeded views and the 120 pairs among them (each form's per-pair errors
    against the FP64 oracle, storage included, and the stored sinograms' errors), and the
    ECC of 4,096 seeded pairs among 92 seeded views on the stored FP16 values (the pair
    kernel's own error, and the oracle's per-pair cost).  The oracle's rate is its measured
    cost per view (dRadon/ds) and per pair (the 4,096 pairs) extrapolated to the whole job."""
    import torch
    import paper_1806_02637_gb300 as ecc
    from oracle import oracle as orc
    cfg = synth.CONFIGS["c4"]
    peaks = measured_peaks()
    t0 = time.perf_counter()
    scan = synth.make_scan(cfg)
    gen_s = time.perf_counter() - t0
    dev = torch.device("cuda", torch.cuda.current_device())
    P = torch.from_numpy(scan["P"]).to(dev)
    images = torch.from_numpy(scan["images"]).to(dev)
    units = cfg.n_pairs * cfg.K
    views = np.sort(np.random.default_rng(1240).choice(cfg.n_views, 16, replace=False))
    sub = synth.upper_pairs(16)
    ga, gb = views[sub[:, 0]], views[sub[:, 1]]
    flat = ga * (2 * cfg.n_views - ga - 1) // 2 + (gb - ga - 1)
    cores = os.cpu_count() or 1
    ta = time.perf_counter()
    S_or = orc.radon_derivative(scan["P"][views], scan["images"][views], cfg.n_alpha, cfg.n_s, n_threads=cores)
    tb = time.perf_counter()
    r_or = orc.ecc(scan["P"][views], S_or, cfg.W, cfg.H, cfg.K, pairs=sub, n_threads=cores)
    E_or = oracle_energies(orc, scan["P"][views], S_or, cfg.W, cfg.H, cfg.K, sub)
    # 4,096 seeded pairs among 92 seeded views, evaluated by the oracle on the stored FP16 values
    rng = np.random.default_rng(1241)
    v92 = np.sort(rng.choice(cfg.n_views, 92, replace=False))
    sub92 = synth.upper_pairs(92)
    sub92 = sub92[np.sort(rng.choice(len(sub92), 4096, replace=False))]
    g92a, g92b = v92[sub92[:, 0]], v92[sub92[:, 1]]
    flat92 = g92a * (2 * cfg.n_views - g92a - 1) // 2 + (g92b - g92a - 1)
    out = {"workload": (f"c4: {cfg.n_views}-view 360-degree scan, {cfg.W}x{cfg.H} detector ({cfg.pixel_mm} mm), "
                        f"{cfg.n_prim} seeded ellipsoids, {cfg.n_alpha}x{cfg.n_s} dRadon/ds, {cfg.K} kappa, all "
                        f"{cfg.n_pairs} pairs"),
           "line_pairs": units, "scan_generation_s": gen_s}
    for name, dt in (("float16", torch.float16), ("bfloat16", torch.bfloat16), ("float32", torch.float32)):
        esize = 4 if dt == torch.float32 else 2
        S, scales = ecc.ecc_precompute_radon_derivative(ctx, P, images, cfg.n_alpha, cfg.n_s, dtype=dt)
        torch.cuda.synchronize()
        ecc.ecc_profile_read(ctx)
        ecc.ecc_profile_enable(ctx, True)
        ecc.ecc_precompute_radon_derivative(ctx, P, images, cfg.n_alpha, cfg.n_s, dtype=dt, out=S, scales=scales)
        torch.cuda.synchronize()
        pre = ecc.ecc_profile_read(ctx)
        tot = torch.empty((1,), dtype=torch.float64, device=dev)
        for _ in range(2):
            ecc.ecc_evaluate(ctx, P, S, cfg.W, cfg.H, cfg.K, scales=scales, total=tot, want_per_pair=False)
        torch.cuda.synchronize()
        ecc.ecc_profile_read(ctx)
        for _ in range(reps):
            ecc.ecc_evaluate(ctx, P, S, cfg.W, cfg.H, cfg.K, scales=scales, total=tot, want_per_pair=False)
        torch.cuda.synchronize()
        prof = ecc.ecc_profile_read(ctx)
        ecc.ecc_profile_enable(ctx, False)
        eval_ms = wall_ms(lambda: ecc.ecc_evaluate(ctx, P, S, cfg.W, cfg.H, cfg.K, scales=scales, total=tot,
                                                   want_per_pair=False), reps)
        pk_ms = prof["ecc_pair_kernel"][1] / reps
        gbs = 8.0 * esize * units / (pk_ms / 1e3) / 1e9
        r = ecc.ecc_evaluate(ctx, P, S, cfg.W, cfg.H, cfg.K, scales=scales)
        d = r["per_pair"][:, 0].cpu().numpy()
        stored = S[torch.as_tensor(views, device=dev)].float()
        if scales is not None:
            stored = stored * scales[torch.as_tensor(views, device=dev)][:, None, None]
        stored = stored.cpu().numpy().astype(np.float64)
        sino_err = (np.abs(stored - S_or).reshape(16, -1).max(axis=1) / np.abs(S_or).reshape(16, -1).max(axis=1))
        if name == "float16":  # the oracle on the stored values of 92 views: 4,096 pairs
            s92 = S[torch.as_tensor(v92, device=dev)].float() * scales[torch.as_tensor(v92, device=dev)][:, None, None]
            s92 = s92.cpu().numpy().astype(np.float64)
            td = time.perf_counter()
            r92 = orc.ecc(scan["P"][v92], s92, cfg.W, cfg.H, cfg.K, pairs=sub92, n_threads=cores)
            te = time.perf_counter()
            E92 = oracle_energies(orc, scan["P"][v92], s92, cfg.W, cfg.H, cfg.K, sub92)
            del s92
            job_s = (tb - ta) / 16 * cfg.n_views + (te - td) / len(sub92) * cfg.n_pairs
            out["cpu_baseline"] = {
                "value": units / job_s, "unit": UNIT, "cores": cores, "kind": "oracle", "extrapolated": True,
                "sample": (f"dRadon/ds of 16 seeded views ({tb - ta:.2f} s) and the ECC of 4096 seeded pairs among 92 "
                           f"seeded views ({te - td:.3f} s, on the stored FP16 values), extrapolated per view and "
                           f"per pair to the whole job ({job_s:.0f} s)")}
            out["pair_kernel_vs_oracle_4096_pairs_on_stored_fp16"] = error_stats(
                d[flat92], r92["d"], E92, float(d[flat92].sum()), float(r92["d"].sum()))
        out[name] = {"precompute_ms": sum(ms for _, ms in pre.values()), "ms_per_eval": eval_ms,
                     "line_pairs_per_s": units / (eval_ms / 1e3), "pair_kernel_ms": pk_ms,
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs", 6800.0),
                                  "unit": "GB/s", "frac": gbs / peaks.get("hbm_gbs", 6800.0),
                                  "frac_of_l2": gbs / l2_gbs,
                                  "work": f"{8 * esize} B (2 views x 4 taps x {esize} B) per line pair"},
                     "total": float(r["total"].cpu()[0]),
                     "vs_oracle_120_pairs": error_stats(d[flat], r_or["d"], E_or, float(d[flat].sum()),
                                                        float(r_or["d"].sum())),
                     "stored_sinogram_err_max_over_16_views": float(sino_err.max())}
        del S, scales, r
        torch.cuda.empty_cache()
    del images, P
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ adjoint forms
def adjoint_forms(ctx, P, sino, cfg, reps=5):
    """The differentiated forms on the same FP32 sinograms, with a seeded rigid motion
    (rotations N(0, 1 deg), translations N(0, 2 mm)): ecc_evaluate_grad (d total / d theta,
    6 per view) and ecc_evaluate_grad_projection (d total / d P, 12 per view).  Timed
    with the library's CUDA events, inputs resident; reports line-pair samples/s of the
    whole call and the per-kernel times."""
    import torch
    import paper_1806_02637_gb300 as ecc
    rng = np.random.default_rng(2024)
    th = np.concatenate([rng.normal(0.0, np.deg2rad(1.0), (cfg.n_views, 3)),
                         rng.normal(0.0, 2.0, (cfg.n_views, 3))], axis=1)
    motion = torch.from_numpy(th).to(sino.device)
    units = cfg.n_pairs * cfg.K
    out = {}
    for name, fn in (("motion_gradient", ecc.ecc_evaluate_grad),
                     ("calibration_gradient", ecc.ecc_evaluate_grad_projection)):
        for _ in range(2):
            fn(ctx, P, sino, cfg.W, cfg.H, cfg.K, motion=motion, want_per_pair=False)
        torch.cuda.synchronize()
        ecc.ecc_profile_read(ctx)
        ecc.ecc_profile_enable(ctx, True)
        for _ in range(reps):
            fn(ctx, P, sino, cfg.W, cfg.H, cfg.K, motion=motion, want_per_pair=False)
        torch.cuda.synchronize()
        prof = ecc.ecc_profile_read(ctx)
        ecc.ecc_profile_enable(ctx, False)
        ms = wall_ms(lambda: fn(ctx, P, sino, cfg.W, cfg.H, cfg.K, motion=motion, want_per_pair=False), reps)
        out[name] = {"ms_per_call": ms, "line_pairs_per_s": units / (ms / 1e3),
                     "kernels_ms": {k: t / reps for k, (c, t) in sorted(prof.items(), key=lambda kv: -kv[1][1])}}
    out["note"] = ("ecc_evaluate_grad / ecc_evaluate_grad_projection on the FP32 sinograms of this scan, seeded "
                   "motion, all pairs; the per-sample adjoint runs in the pair kernel (ecc_pair_grad_kernel)")
    return out


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import paper_1806_02637_gb300 as ecc

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = synth.CONFIGS[args.workload]
    if args.views:
        import dataclasses
        full = cfg
        cfg = dataclasses.replace(cfg, n_views=args.views)
        scan = synth.make_scan(full, views=np.arange(args.views))
    else:
        scan = synth.make_scan(cfg)
    ctx = ecc.Context(local)
    stream = torch.cuda.current_stream(dev)
    P = torch.from_numpy(scan["P"]).to(dev)
    images = torch.from_numpy(scan["images"]).to(dev)
    sino = torch.empty((cfg.n_views, cfg.n_alpha, cfg.n_s), dtype=torch.float32, device=dev)
    total = torch.empty((1,), dtype=torch.float64, device=dev)

    shard = args.shard and world > 1

    def step():
        if shard:   # one job over all ranks: view slices, all-gather, pair tiles, FP64 all-reduce
            from paper_1806_02637_gb300 import distributed as D
            t, _ = D.sharded_consistency(ctx, P, images, cfg.W, cfg.H, cfg.n_alpha, cfg.n_s, cfg.K, rank, world)
            total.copy_(t)
            return
        ecc.ecc_precompute_radon_derivative(ctx, P, images, cfg.n_alpha, cfg.n_s, out=sino)
        ecc.ecc_evaluate(ctx, P, sino, cfg.W, cfg.H, cfg.K, total=total, want_per_pair=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    ecc.ecc_profile_read(ctx)               # drop anything recorded so far
    ecc.ecc_profile_enable(ctx, True)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)
    sampler = ClockSampler(gpu_id) if rank == 0 else None
    if sampler:
        sampler.start()
    launches0 = ecc.ecc_kernel_launches(ctx)
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if pg is not None:
        pg.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = ecc.ecc_kernel_launches(ctx) - launches0
    prof = ecc.ecc_profile_read(ctx)
    ecc.ecc_profile_enable(ctx, False)
    clocks = sampler.stop() if sampler else None
    result_total = float(total.cpu()[0])
    elapsed_ms = max_over_ranks(pg, elapsed_ms, dev)
    ms_per_step = elapsed_ms / args.steps
    units = cfg.n_pairs * cfg.K
    value = units * (1 if shard else world) / (ms_per_step / 1e3)

    e2e = None
    if not args.no_e2e:
        # ---------------- end to end through the host-buffer entry point
        P_host = torch.from_numpy(scan["P"]).pin_memory()
        img_host = torch.from_numpy(scan["images"]).pin_memory()
        for _ in range(2):
            ecc.ecc_scan_consistency_host(ctx, P_host, img_host, cfg.n_alpha, cfg.n_s, cfg.K)
        if pg is not None:
            pg.barrier()
        e_steps = max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        e_total = None
        for _ in range(e_steps):
            e_total = ecc.ecc_scan_consistency_host(ctx, P_host, img_host, cfg.n_alpha, cfg.n_s, cfg.K)
        e_s = time.perf_counter() - t0
        e_s = max_over_ranks(pg, e_s, dev)
        e2e = {"value": units * world / (e_s / e_steps), "unit": UNIT, "steps": e_steps,
               "ms_per_step": e_s / e_steps * 1e3,
               "h2d_bytes_per_step": int(scan["images"].nbytes + scan["P"].nbytes), "d2h_bytes_per_step": 8,
               "api": "ecc_scan_consistency_host (pinned host buffers, synchronous)",
               "total_matches_device_path": bool(e_total == result_total)}


    if rank != 0:
        return 0

    # ---------------- per-kernel shares and the dominant kernel's roofline
    kern = {}
    tot_prof = sum(ms for _, ms in prof.values()) or 1.0
    for name, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        kern[name] = {"launches_per_step": n / args.steps, "ms_per_step": ms / args.steps, "share": ms / tot_prof}
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    peaks = measured_peaks()
    n_dom, ms_dom = prof[dom]
    if dom == "joseph_kernel":
        taps = joseph_taps(cfg)
        flops = FLOPS_PER_TAP * taps * args.steps / n_dom
        achieved = flops / (ms_dom / n_dom / 1e3) / 1e12
        # DRAM bytes (read + write) of one launch, from an ncu capture of a 32-view launch of this
        # kernel (183.3 MB + 58.3 MB), scaled to the views of an average launch of this step
        views_per_launch = cfg.n_views * args.steps / n_dom
        traffic = (183.299840e6 + 58.299392e6) / 32 * views_per_launch
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a 32-view launch, "
                                  f"scaled to {views_per_launch:.1f} views per launch",
                "peak_source": "FP32 lanes x FMA x max SM clock (152 x 128 x 2 x 2.07 GHz)",
                "work": f"{FLOPS_PER_TAP} FLOP per in-image Joseph tap, {taps} taps per step",
                # the kernel's actual limiter (ncu: L1 data-pipe wavefronts): the 8-byte
                # interpolation pair each tap reads, against the L1 data rate
                "l1_gather": {"achieved_tbs": 8.0 * taps * args.steps / n_dom / (ms_dom / n_dom / 1e3) / 1e12,
                              "peak_tbs": L1_PEAK_TBS,
                              "frac": 8.0 * taps * args.steps / n_dom / (ms_dom / n_dom / 1e3) / 1e12 / L1_PEAK_TBS,
                              "peak_source": "128 B per clock per SM x 152 SMs x 2.07 GHz",
                              "work": "8 B (one interpolation pair) per in-image tap"}}
    else:
        bytes_per_launch = 32.0 * units * args.steps / n_dom
        achieved = bytes_per_launch / (ms_dom / n_dom / 1e3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback",
                "work": "32 B (2 views x 4 taps x FP32) per line-pair sample"}
    ev_names = ("view_setup_kernel", "alpha_dir_kernel", "pair_setup_kernel", "ecc_pair_kernel", "reduce_kernel")
    eval_ms = wall_ms(lambda: ecc.ecc_evaluate(ctx, P, sino, cfg.W, cfg.H, cfg.K, total=total, want_per_pair=False),
                      10)
    pk = kern.get("ecc_pair_kernel")
    eval_only = None
    if pk:
        gbs = 32.0 * units / (pk["ms_per_step"] / 1e3) / 1e9
        eval_only = {"ms_per_eval": eval_ms, "line_pairs_per_s": units / (eval_ms / 1e3),
                     "how": "ecc_evaluate alone on resident sinograms, 10 calls between CUDA events",
                     "pair_kernel_ms": pk["ms_per_step"],
                     "pair_kernel_gather_gbs": gbs,
                     "pair_kernel_frac_of_hbm": gbs / peaks.get("hbm_gbs", 6800.0),
                     # one ncu capture of this launch (one-pass metrics, same kernel build):
                     # DRAM read + write and L2 sector bytes per launch
                     "pair_kernel_dram_bytes_ncu": 441123328 + 33391104,
                     "pair_kernel_l2_bytes_ncu": 86831338 * 32}
    l2 = l2_read_rate(dev)
    if eval_only:
        eval_only["pair_kernel_frac_of_l2"] = eval_only["pair_kernel_gather_gbs"] / l2["gbs"]
        eval_only["l2_read_probe"] = l2
    adjoint = None
    if not args.no_adjoint_forms:
        adjoint = adjoint_forms(ctx, P, sino, cfg)
    # the oracle on the whole job (FP64, host cores): the CPU baseline, and the reference
    # every result of this line is compared with
    cpu = oracle = None
    if not args.no_cpu_baseline and world == 1:
        from oracle import oracle as orc
        cores = os.cpu_count() or 1
        S_or, r_or, t_radon, t_ecc = oracle_job(cfg, scan, cores)
        cpu = {"value": units / (t_radon + t_ecc), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"the whole job, not extrapolated: dRadon/ds of all {cfg.n_views} views ({t_radon:.2f} s) "
                          f"and the ECC of all {cfg.n_pairs} pairs ({t_ecc:.2f} s), FP64 on {cores} host threads")}
        E_or = oracle_energies(orc, scan["P"], S_or, cfg.W, cfg.H, cfg.K, r_or["pairs"])
        del S_or
        oracle = {"d": r_or["d"], "total": r_or["total"], "E": E_or, "nk": r_or["nk"]}
    accuracy = None
    if oracle is not None:
        r32 = ecc.ecc_evaluate(ctx, P, sino, cfg.W, cfg.H, cfg.K)
        accuracy = error_stats(r32["per_pair"][:, 0].cpu().numpy(), oracle["d"], oracle["E"],
                               float(r32["total"].cpu()[0]), oracle["total"])
        accuracy["oracle_total"] = oracle["total"]
        # N_kappa of every pair (integer sample ranges of the set-up) against the oracle's
        accuracy["nkappa_mismatches"] = int(np.count_nonzero(r32["nkappa"].cpu().numpy() != np.asarray(oracle["nk"])))
    forms = None
    if not args.no_storage_forms:
        forms = storage_forms(ctx, P, images, cfg, result_total, oracle=oracle, l2_gbs=l2["gbs"])
    serving = None
    if not args.no_serving and world == 1:
        serving = serving_leg(args, scan)
    precision_c4 = None
    if args.c4_leg and world == 1:
        del images, sino
        torch.cuda.empty_cache()
        precision_c4 = c4_leg(ctx, l2["gbs"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong" if shard else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": dict(workload_config(cfg), **({"parallelism": f"one job over {world} ranks: view slices + all-gather of the sinograms, pair tiles + FP64 all-reduce"} if shard else {})),
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "kernels": kern, "ecc_eval_only": eval_only, "accuracy_vs_oracle": accuracy, "storage_forms": forms,
            "adjoint_forms": adjoint, "serving": serving, "precision_c4": precision_c4,
            "total": result_total,
            "geometry_precision": "f64 per-view/per-pair set-up, double-float (~48-bit) tile anchors, f32 per-sample"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
