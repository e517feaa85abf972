#!/usr/bin/env python
"""Benchmark: validated space-time edges/s of the batched Extend planner on GB300.

Workload (default, one GPU): UR5e (standard DH) with 32 link spheres among 16
sphere obstacles (r = 0.06 m) on 4-waypoint paths in a 1.2 m cube, joint
v_max pi/2, horizon 15 s, root recycling with N = 8 slots, W = 1024 Extend
workers per iteration, FP32. A step is one stp_plan call from a fresh state
running --iters iterations (every iteration: Philox sampling, NN scan, steering,
edge validation, ordered insertion, bridge scan and validation, publish, root
recycling). The metric counts validated edges (extension + bridge edges sent to
the collision kernel) per second of device time.

End to end (`e2e`): per step stp_create_problem from host arrays, stp_plan with
the library's default graph size, the path read back, stp_free, timed on the
host.

Beside the headline line: the batched form on 512 mixed problems (autotuned;
also a 48-problem sample planned as one batch against the same problems planned
one after another, first-solution times from a common start),
the learned-proposal study on the 7-DoF distribution (training data from
plain plans, the proposal network trained on the tensor cores, held-out
problems planned plain and learned at the same budget), and the allocation
ablation (root recycling against a fixed forest over broad arrival ranges).

Timing: CUDA events on the library's stream around each step's GPU work
(stats step_ms; the events around the whole call, which also hold the host's
synchronisation, are reported as ms_per_step_call); an L2 flush (512 MB
write) runs between steps outside the events; a second pass of the same
steps records CUDA events between the kernels inside the captured graphs to give
per-kernel times and the collision kernel's roofline. The 2^20-edge collision
microbenchmark and the FP64 oracle (CPU baseline) are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): independent problem replicas per rank (seed = rank), no
collective on the data path; value = all ranks' edges / max rank time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as WL  # noqa: E402

WORKLOAD = "ur5e-6dof-32sph-16obs-recycling-N8-W1024"
# DRAM bytes per profiled collision interval of the planner on this workload,
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum; summary
# in profiles/k_validate_ur5e_plan_ncu.md): the extension launch (237.1 KB) and
# the two bridge passes together (141.6 + 80.6 KB), averaged over the two
# intervals. The figure belongs to the kernel source it was taken from: when
# the source's hash differs, the bench reports no traffic.
TRAFFIC_CAPTURE = {"kernel": "k_validate", "bytes_per_launch": 234.9e3,
                   "sources": [os.path.join("paper_2609_30533_gb300", "csrc", f)
                               for f in ("stp_validate.cu", "stp_validate_body.cuh", "stp_internal.cuh")],
                   "sha256_16": "1680dd7e7fdf08ea", "profile": "profiles/k_validate_ur5e_plan_ncu.md"}
METRIC = "validated space-time edges/s"
UNIT = "edges/s"
FLUSH_BYTES = 512 << 20


def kernel_source_hash(sources):
    """First 16 hex digits of the SHA-256 of the kernel's source files, in order."""
    import hashlib
    d = hashlib.sha256()
    try:
        for src in sources:
            with open(os.path.join(ROOT, src), "rb") as f:
                d.update(f.read())
    except OSError:
        return None
    return d.hexdigest()[:16]


def _capture_traffic():
    """(bytes per launch or None, note) of the ncu traffic capture, None when
    the kernel source changed since it was taken."""
    h = kernel_source_hash(TRAFFIC_CAPTURE["sources"])
    if h is None:
        return None, "kernel source not found"
    if h != TRAFFIC_CAPTURE["sha256_16"]:
        return None, "kernel source changed since the ncu capture (%s)" % TRAFFIC_CAPTURE["profile"]
    return TRAFFIC_CAPTURE["bytes_per_launch"], "from the ncu capture in %s (same kernel source)" % (
        TRAFFIC_CAPTURE["profile"])


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def fp32_peak_tflops(n_sm, mhz):
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return n_sm * 128 * 2 * mhz * 1e6 / 1e12


def point_flops(prob):
    """Per check point, excluding pair tests: sphere transforms (18 flops per
    sphere), forward kinematics (about 60 flops per joint) and obstacle
    interpolation (9 flops per obstacle); each pair test adds 8 flops."""
    S = len(prob.spheres)
    M = len(prob.obs_r)
    return 18 * S + 60 * prob.dof + 9 * M


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # Raw samples go to $STP_CLOCKS_DIR (default: the system temp directory).
        import tempfile
        out_dir = os.environ.get("STP_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, "clocks_rank%d.csv" % gpu_index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # Let the sampler take its first reading before the timed region.
            t0 = time.time()
            while time.time() - t0 < 2.0:
                self.f.flush()
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_reference(args):
    """The oracle (single-threaded FP64 CPU) on the same workload and metric; each
    step is a bounded sample: --ref-iters iterations of the same W = 1024 plan."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    prob, prm = WL.ur5e(0)
    import dataclasses
    prm = dataclasses.replace(prm, max_iters=args.ref_iters)
    for _ in range(args.warmup):
        O.plan(prob, dataclasses.replace(prm, max_iters=1))
    edges = 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        r = O.plan(prob, dataclasses.replace(prm, seed=k))
        edges += r.ext_checked + r.bridge_checked
    secs = time.perf_counter() - t0
    value = edges / secs
    sample = "%d steps x %d iterations x W=1024 of the %s plan" % (args.steps, args.ref_iters, WORKLOAD)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "iters_per_step": args.ref_iters, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_baseline(args):
    import dataclasses

    import oracle as O
    prob, prm = WL.ur5e(0)
    prm = dataclasses.replace(prm, max_iters=args.cpu_iters)
    t0 = time.perf_counter()
    r = O.plan(prob, prm)
    secs = time.perf_counter() - t0
    edges = r.ext_checked + r.bridge_checked
    return {"value": edges / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d iterations x W=1024 of the %s plan (%d edges, %.1f s)" % (
                args.cpu_iters, WORKLOAD, edges, secs)}


def _oracle_mixed(job):
    """One mixed-batch problem planned by the FP64 oracle in a worker process;
    returns (edges validated, seconds of planning, construction excluded)."""
    import dataclasses

    import oracle as O
    index, workers, iters = job
    prob, prm = WL.mixed(index)
    prm = dataclasses.replace(prm, workers=workers, max_iters=iters, problem_id=index)
    t0 = time.perf_counter()
    r = O.plan(prob, prm)
    return r.ext_checked + r.bridge_checked, time.perf_counter() - t0


def cpu_batched_baseline(problems, workers, iters, cores=None):
    """The FP64 oracle on a bounded sample of the mixed batched workload, one
    problem per process over the host's cores (spawn pool, started and warmed
    before the timed map). Reports the pool's edges/s over all cores (wall
    clock of the timed map) and the single-core rate (edges over the summed
    planning seconds)."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    # Heaviest first (spheres x obstacles), so the pool's tail stays short.
    cost = {}
    for i in range(problems):
        pr, _ = WL.mixed(i)
        cost[i] = len(pr.spheres) * max(len(pr.obs_r), 1)
    jobs = [(i, workers, iters) for i in sorted(range(problems), key=lambda i: -cost[i])]
    with mp.get_context("spawn").Pool(min(cores, problems)) as pool:
        # Bounded waits: a worker that died would otherwise leave map() waiting.
        pool.map_async(_oracle_mixed, [(i, workers, 1) for i in range(min(cores, problems))]).get(timeout=300)
        t0 = time.perf_counter()
        res = pool.map_async(_oracle_mixed, jobs, chunksize=1).get(timeout=600)
        wall = time.perf_counter() - t0
    edges = sum(e for e, _ in res)
    cpu_s = sum(t for _, t in res)
    return {"value": edges / wall, "unit": UNIT, "cores": min(cores, problems), "kind": "oracle",
            "single_core_value": edges / cpu_s if cpu_s > 0 else None,
            "sample": "%d mixed problems x %d iterations x W=%d, one problem per process (%d edges, %.1f s wall, "
                      "%.1f s of planning summed over processes)" % (problems, iters, workers, edges, wall, cpu_s)}


def microbench(args, P, prob, prm, stream, flush, rank, local, n=None):
    """Collision kernel alone on random edges of the problem's robot and
    obstacles (2^20 UR5e edges by default) resident on the device, with and
    without early exit; kernel time from CUDA events around the launch."""
    import torch
    n = n or args.micro_edges
    qa, ta, qb, tb = WL.microbench_edges(prob, n, prm.eta, prm.H, seed=rank)
    dev = torch.device("cuda", local)
    tq = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev) for a in (qa, ta, qb, tb)]
    ver = torch.zeros(n, dtype=torch.uint8, device=dev)
    micro = {}
    for label, early in (("early_exit", True), ("no_early_exit", False)):
        for _ in range(3):
            P.check_edges_device(tq[0].data_ptr(), tq[1].data_ptr(), tq[2].data_ptr(), tq[3].data_ptr(), n,
                                 ver.data_ptr(), early_exit=early)
        kms, kpts, kpairs, call_ms = [], 0, 0, []
        for _ in range(5):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.check_edges_device(tq[0].data_ptr(), tq[1].data_ptr(), tq[2].data_ptr(), tq[3].data_ptr(), n,
                                 ver.data_ptr(), early_exit=early)
            e1.record(stream)
            e1.synchronize()
            call_ms.append(e0.elapsed_time(e1))
            ms, pts, prs = P.last_validate()
            kms.append(ms)
            kpts, kpairs = pts, prs
        k_ms = statistics.median(kms)
        flops = kpairs * 8 + kpts * point_flops(prob)
        micro[label] = {"edges_per_s": n / (statistics.median(call_ms) * 1e-3),
                        "kernel_ms": k_ms, "check_points": kpts, "pair_tests": kpairs,
                        "achieved_tflops": flops / (k_ms * 1e-3) / 1e12,
                        "free_fraction": float(ver.float().mean().item())}
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = float(_peaks().get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(n_sm, max_mhz)
    for m in micro.values():
        m["frac"] = m["achieved_tflops"] / peak
    return micro, peak


def microbench_arm7(args, stream, flush, rank, local):
    """The collision kernel on the 7-DoF workload (48 link spheres, 64 sphere
    obstacles with radii U[0.04, 0.1] m on 8-waypoint paths, H 60 s): random
    edges of length eta = 0.5 rad, 3,072 sphere-obstacle pairs per check point."""
    from paper_2609_30533_gb300 import stp
    prob7, prm7 = WL.arm7(rank)
    P7 = stp.problem_from(prob7, prm7, precision=0, max_iters=1)
    P7.set_stream(stream.cuda_stream)
    micro7, peak7 = microbench(args, P7, prob7, prm7, stream, flush, rank, local, n=args.micro7_edges)
    P7.close()
    return dict(micro7, n_edges=args.micro7_edges, peak_tflops=peak7,
                workload="arm7, 48 spheres, 64 obstacles, 8 waypoints")


def batched(args, rank):
    """Batched form: mixed problems (2/6/7-DoF, 4..128 obstacles, 10..60 s
    horizons) planned together in one graph-captured launch sequence; W and the
    launch shape are chosen by the autotuner on a sample. Reports throughput and
    first-solution latency percentiles, beside the same problems planned one by
    one (plain) on a sample."""
    import dataclasses

    from paper_2609_30533_gb300 import autotune, stp

    def make(indices, W, iters):
        out = []
        for i in indices:
            prob, prm = WL.mixed(i)
            prm = dataclasses.replace(prm, workers=W, max_iters=iters, problem_id=i, seed=rank)
            out.append(stp.problem_from(prob, prm, precision=0, iters_per_graph=16))
        return out

    sample = list(range(48))
    choice = autotune.autotune(lambda W: make(sample, W, args.tune_iters), workers=(128, 256, 512),
                               team_ctas=(1, 2, 4, 8, 16), nn_ctas=(2, 4, 8, 16), validate_ctas=(2, 4, 8, 16))
    idx = list(range(args.batch_problems))
    probs = make(idx, choice.workers, args.batch_iters)

    def run_full(t):
        B = stp.Batch(probs, nn_ctas=t.nn_ctas, validate_ctas=t.validate_ctas, iters_per_graph=16,
                      launch_mode=t.launch_mode, team_ctas=t.team_ctas)
        B.plan()
        runs = [B.plan() for _ in range(args.batch_reps)]
        B.close()
        return statistics.median(r[0] for r in runs), runs[0][1]

    # The sample ranks the shapes of each launch form; the whole batch then
    # decides between the two forms' best shapes (a 48-problem sample fills
    # the persistent queue's teams about once, the whole batch many times).
    # The queue's best team size also depends on how many problems each team
    # plans, so every team size of the sample's best W is timed on the whole
    # batch (each a few hundred ms).
    forms = {}
    for mode, name in ((stp.STP_LAUNCH_DEFAULT, "persistent_queue"), (1, "per_step")):
        cand = [t for t in choice.trials if t.launch_mode == mode and t.workers == choice.workers]
        if not cand:
            continue
        t = min(cand, key=autotune._rank)
        f_ms, f_stats = run_full(t)
        if mode == stp.STP_LAUNCH_DEFAULT:
            team_ms = {t.team_ctas: f_ms}
            for alt in cand:
                if alt.team_ctas not in team_ms:
                    a_ms, a_stats = run_full(alt)
                    team_ms[alt.team_ctas] = a_ms
                    if a_ms < f_ms:
                        t, f_ms, f_stats = alt, a_ms, a_stats
        f_fs = [st["first_solution_ms"] for st in f_stats if st["first_solution_iter"] >= 0]
        forms[name] = {"launch_mode": t.launch_mode, "team_ctas": t.team_ctas, "nn_ctas": t.nn_ctas,
                       "validate_ctas": t.validate_ctas, "batch_ms": f_ms, "problems_per_s": len(idx) / (f_ms * 1e-3),
                       "batch_ms_per_team_size": team_ms if mode == stp.STP_LAUNCH_DEFAULT else None,
                       "solved": len(f_fs), "first_solution_ms_p50": float(np.percentile(f_fs, 50)) if f_fs else None,
                       "first_solution_ms_p99": float(np.percentile(f_fs, 99)) if f_fs else None,
                       "_trial": t, "_stats": f_stats}
    best_name = min(forms, key=lambda k: (-forms[k]["solved"], forms[k]["batch_ms"]))
    best = forms[best_name]
    choice = dataclasses.replace(choice, launch_mode=best["_trial"].launch_mode, team_ctas=best["_trial"].team_ctas,
                                 nn_ctas=best["_trial"].nn_ctas, validate_ctas=best["_trial"].validate_ctas)
    ms, stats = best["batch_ms"], best["_stats"]
    for f in forms.values():
        del f["_trial"], f["_stats"]
    fs = sorted(st["first_solution_ms"] for st in stats if st["first_solution_iter"] >= 0)
    edges = sum(st["edges_validated"] + st["bridges_validated"] for st in stats)

    # Plain: the same problems one at a time (sample), same W and budget.
    # As a queue (one after another from a common start), a problem's first
    # solution waits for every earlier problem's whole plan.
    plain_fs, plain_ms, plain_solved, queue_fs = [], [], 0, []
    plain_each = []   # per problem: first-solution ms from its own start, or None
    elapsed = 0.0
    for i in idx[:args.plain_sample]:
        out = probs[i].plan()
        plain_ms.append(out.stats["plan_ms"])
        if out.stats["first_solution_iter"] >= 0:
            plain_solved += 1
            plain_fs.append(out.stats["first_solution_ms"])
            queue_fs.append(elapsed + out.stats["first_solution_ms"])
            plain_each.append(out.stats["first_solution_ms"])
        else:
            plain_each.append(None)
        elapsed += out.stats["plan_ms"]
    # The same sample planned as one batch (chosen launch shape, same budget):
    # every problem starts at once.
    nq = len(plain_ms)
    Bq = stp.Batch(probs[:nq], nn_ctas=choice.nn_ctas, validate_ctas=choice.validate_ctas, iters_per_graph=16,
                   launch_mode=choice.launch_mode, team_ctas=choice.team_ctas)
    Bq.plan()
    qruns = sorted((Bq.plan() for _ in range(args.batch_reps)), key=lambda r: r[0])
    Bq.close()
    q_ms, q_stats = qruns[len(qruns) // 2]
    batch_fs = [st["first_solution_ms"] for st in q_stats if st["first_solution_iter"] >= 0]
    # Per problem at equal success: the problems solved both alone and in the
    # batch; alone a problem's first solution counts from its own start, in the
    # batch from the batch's start (all problems share the GPU).
    common = [(pe, st["first_solution_ms"]) for pe, st in zip(plain_each, q_stats)
              if pe is not None and st["first_solution_iter"] >= 0]
    for P in probs:
        P.close()

    def pct(v, q):
        return float(np.percentile(v, q)) if v else None

    cpu_all = None
    if not args.no_cpu and rank == 0 and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        n_cpu = args.cpu_batch_problems or min(32, 2 * (os.cpu_count() or 1))
        try:
            cpu_all = cpu_batched_baseline(n_cpu, choice.workers, args.cpu_batch_iters)
        except Exception as exc:  # a host-side baseline must not cost the GPU measurement
            cpu_all = {"error": str(exc)}

    return {
        "workload": "mixed 2/6/7-DoF, 4-128 obstacles, 10-60 s horizons",
        "cpu_oracle_all_cores": cpu_all,
        "problems": len(idx), "iters_budget": args.batch_iters,
        "autotuned": {"workers": choice.workers, "launch_mode": choice.launch_mode, "team_ctas": choice.team_ctas,
                      "nn_ctas": choice.nn_ctas, "validate_ctas": choice.validate_ctas, "form": best_name,
                      "trials": [dataclasses.asdict(t) for t in choice.trials]},
        "forms_whole_batch": forms,
        "batch_ms": ms, "problems_per_s": len(idx) / (ms * 1e-3), "edges_per_s": edges / (ms * 1e-3),
        "solved": len(fs), "success_rate": len(fs) / len(idx),
        "first_solution_ms_p50": pct(fs, 50), "first_solution_ms_p99": pct(fs, 99),
        "queue_vs_batch": {"problems": nq, "iters_budget": args.batch_iters,
                           "note": "first-solution ms counted from a common start: the sample planned as one "
                                   "batch against the same problems planned one after another",
                           "batch_solved": len(batch_fs), "batch_first_ms_p50": pct(batch_fs, 50),
                           "batch_total_ms": q_ms,
                           "queue_solved": len(queue_fs), "queue_first_ms_p50": pct(queue_fs, 50),
                           "queue_total_ms": elapsed},
        "per_problem_vs_plain": {
            "problems": nq, "solved_alone": plain_solved, "solved_batched": len(batch_fs), "common": len(common),
            "note": "first-solution ms on the commonly solved problems: alone from each problem's own start, "
                    "batched from the start of the batch of the same problems",
            "alone_first_ms_p50": pct([c[0] for c in common], 50),
            "alone_first_ms_p99": pct([c[0] for c in common], 99),
            "batched_first_ms_p50": pct([c[1] for c in common], 50),
            "batched_first_ms_p99": pct([c[1] for c in common], 99)},
        "plain_sample": {"problems": len(plain_ms), "solved": plain_solved,
                         "first_solution_ms_p50": pct(plain_fs, 50), "first_solution_ms_p99": pct(plain_fs, 99),
                         "ms_per_problem_p50": pct(plain_ms, 50), "sequential_ms_per_problem": float(np.mean(plain_ms)),
                         "batched_ms_per_problem": ms / len(idx)},
    }


def aggregate_over_ranks(edges, total_ms, e2e_edges, e2e_secs, dist=None, device="cpu"):
    """Whole-job figures over the ranks of an initialised process group (or
    this process alone): edge counts summed, times the maximum over ranks.
    Returns (edges, ms, e2e edges, e2e seconds)."""
    import torch
    vals = torch.tensor([float(edges), float(total_ms), float(e2e_edges), float(e2e_secs)], dtype=torch.float64,
                        device=device)
    if dist is not None:
        tot = vals.clone()
        dist.all_reduce(tot[0:1], op=dist.ReduceOp.SUM)
        dist.all_reduce(tot[2:3], op=dist.ReduceOp.SUM)
        mx = vals.clone()
        dist.all_reduce(mx[1:2], op=dist.ReduceOp.MAX)
        dist.all_reduce(mx[3:4], op=dist.ReduceOp.MAX)
        vals = torch.stack([tot[0], mx[1], tot[2], mx[3]])
    return tuple(float(x) for x in vals.cpu())


def _paired(a, b):
    """Plain arm a against learned arm b on the problems both solved (equal
    success by construction): counts, first-solution ms p50/p99, first
    iteration p50 and mean arrival U over the common set, and each arm's
    own solved count."""
    both = a.solved & b.solved

    def q(v, p):
        return float(np.percentile(v, p)) if len(v) else None

    return {"plain_solved": int(a.solved.sum()), "learned_solved": int(b.solved.sum()),
            "common_solved": int(both.sum()),
            "plain_first_ms_p50": q(a.first_ms[both], 50), "learned_first_ms_p50": q(b.first_ms[both], 50),
            "plain_first_ms_p99": q(a.first_ms[both], 99), "learned_first_ms_p99": q(b.first_ms[both], 99),
            "plain_first_iter_p50": q(a.first_iter[both], 50), "learned_first_iter_p50": q(b.first_iter[both], 50),
            "plain_mean_arrival": float(np.mean(a.U[both])) if both.any() else None,
            "learned_mean_arrival": float(np.mean(b.U[both])) if both.any() else None}


def sweep(args, rank):
    """Allocation ablation and broad-range sweep on the UR5e workload with 8
    obstacles (the scene keeps its 15 s obstacle motion; only the arrival-time
    range H changes): root recycling against no recycling (fixed forest) over
    H = 25 / 50 / 100 s (16 roots, W 512), root counts 8..128 (W 512, H 100 s)
    and W 128..2048 (16 roots, H 100 s). Each condition plans the same problems
    in one batch for a fixed iteration budget; reported: solved count, mean
    arrival over the problems both variants solved, median first-solution time."""
    import dataclasses

    from paper_2609_30533_gb300 import proposal as PR
    from paper_2609_30533_gb300 import stp

    n, iters = args.sweep_problems, args.sweep_iters

    def run(variant, H, N, W):
        probs = []
        for i in range(n):
            prob, prm = WL.ur5e(seed=i, n_obs=8)
            prm = dataclasses.replace(prm, variant=variant, H=H, n_roots=N, workers=W, max_iters=iters,
                                      problem_id=i, seed=rank)
            probs.append(stp.problem_from(prob, prm, precision=0, iters_per_graph=16))
        o = PR.plan_batch(probs)
        for P in probs:
            P.close()
        return o

    def pair(H, N, W):
        r, f = run(1, H, N, W), run(2, H, N, W)
        both = r.solved & f.solved
        return {"H": H, "roots": N, "W": W,
                "solved_recycling": int(r.solved.sum()), "solved_fixed": int(f.solved.sum()),
                "mean_arrival_recycling": float(np.mean(r.U[both])) if both.any() else None,
                "mean_arrival_fixed": float(np.mean(f.U[both])) if both.any() else None,
                "p50_first_ms_recycling": float(np.median(r.first_ms[r.solved])) if r.solved.any() else None,
                "p50_first_ms_fixed": float(np.median(f.first_ms[f.solved])) if f.solved.any() else None}

    return {"workload": "ur5e, 8 obstacles, %d problems, %d iterations, batched" % (n, iters),
            "range": [pair(H, 16, 512) for H in (25.0, 50.0, 100.0)],
            "roots": [pair(100.0, N, 512) for N in (8, 16, 32, 64, 128)],
            "batch": [pair(100.0, 16, W) for W in (128, 256, 512, 1024, 2048)]}


def scan_bytes_per_node(dof):
    """Algorithmic bytes of one tree vertex read by an NN or bridge scan:
    coordinates and time padded to 16-byte vectors, plus a flag / root-time word."""
    return 16 * ((dof + 1 + 3) // 4) + 4


def run_config(name, make, n_problems, peak_tflops, hbm_gbs):
    """Plans n_problems of one configuration one at a time (FP32, one graph per
    8 iterations, CUDA events around each plan) and then profiles one of them:
    validated edges/s, first-solution ms p50/p99 and mean arrival over the
    solved problems, per-kernel shares, and the NN and bridge scans against
    their FP32 and HBM rooflines (algorithmic flops: (3d + 5) per (query,
    vertex) evaluation; bytes: every vertex of a scanned set once per iteration)."""
    from paper_2609_30533_gb300 import stp
    edges, ms_total, fs, U, solved = 0, 0.0, [], [], 0
    for i in range(n_problems):
        prob, prm = make(i)
        P = stp.problem_from(prob, prm, precision=0)
        P.plan()
        out = P.plan()
        st = out.stats
        edges += st["edges_validated"] + st["bridges_validated"]
        ms_total += st["plan_ms"]
        if st["first_solution_iter"] >= 0:
            solved += 1
            fs.append(st["first_solution_ms"])
            U.append(out.U)
        P.close()
    prob, prm = make(0)
    P = stp.problem_from(prob, prm, precision=0)
    P.set_profiling(True)
    out = P.plan()
    prof = P.profile()
    P.close()
    st = out.stats
    d = prob.dof
    total = sum(v[0] for v in prof.values()) or 1e-12
    scans = {}
    for key, ev, nd in (("k_nn", "nn_evals", "nn_nodes"), ("k_bridge", "bridge_evals", "bridge_nodes")):
        ms = prof.get(key, (0.0, 0))[0]
        fl = st[ev] * (3 * d + 5)
        by = st[nd] * scan_bytes_per_node(d)
        tf = fl / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
        gb = by / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        scans[key] = {"ms": ms, "evals": st[ev], "nodes": st[nd], "tflops": tf, "fp32_frac": tf / peak_tflops,
                      "gbs": gb, "hbm_frac": gb / hbm_gbs}

    def pct(v, q):
        return float(np.percentile(v, q)) if v else None

    return {"workload": name, "problems": n_problems, "solved": solved,
            "edges_per_s": edges / (ms_total * 1e-3) if ms_total > 0 else None,
            "plan_ms_mean": ms_total / n_problems,
            "first_solution_ms_p50": pct(fs, 50), "first_solution_ms_p99": pct(fs, 99),
            "mean_arrival": float(np.mean(U)) if U else None,
            "profiled": {"iterations": st["iterations"], "nodes": st["nodes"],
                         "kernel_share": {k: round(v[0] / total, 4) for k, v in prof.items()},
                         "scans": scans}}


def stated_configs(args, peak_tflops):
    """The point-robot and 7-DoF configurations at their stated sizes: disc2d
    (8 discs, interval root with 4 groups, W 64, 2000 iterations) and the
    7-DoF arm (48 link spheres, 64 obstacles on 8-waypoint paths, H 60 s,
    W 4096; root recycling with 16 trees and interval root)."""
    import dataclasses
    hbm = float(_peaks().get("hbm_gbs", 6685.8))

    def c0(i):
        prob, prm = WL.disc2d(i)
        return prob, dataclasses.replace(prm, max_iters=args.c0_iters, problem_id=i)

    def c2(variant):
        def mk(i):
            prob, prm = WL.arm7(i, variant=variant)
            return prob, dataclasses.replace(prm, workers=4096, max_iters=args.c2_iters, problem_id=i)
        return mk

    return {
        "c0_disc2d": run_config("disc2d, 8 discs, interval root N 4, W 64, %d iterations" % args.c0_iters, c0,
                                args.c0_problems, peak_tflops, hbm),
        "c2_arm7_recycling": run_config("arm7, 48 spheres, 64 obstacles, root recycling N 16, W 4096, %d iterations"
                                        % args.c2_iters, c2(1), args.c2_problems, peak_tflops, hbm),
        "c2_arm7_interval": run_config("arm7, 48 spheres, 64 obstacles, interval root N 16, W 4096, %d iterations"
                                       % args.c2_iters, c2(0), args.c2_problems, peak_tflops, hbm),
    }


def mlp_throughput(rank, B=65536, reps=3):
    """Tensor-core GEMMs of proposal-network training steps at batch B on
    synthetic inputs and targets (CUDA events around the forward chain and
    the backward pass, which hold GEMM launches only)."""
    from paper_2609_30533_gb300 import proposal as PR
    from paper_2609_30533_gb300 import stp
    rng = np.random.default_rng(rank)
    X = np.zeros((B, stp.MLP_IN), dtype=np.float32)
    X[:, :26] = rng.uniform(-1, 1, size=(B, 26))
    T = np.zeros((B, stp.MLP_NTGT), dtype=np.float32)
    T[:, 0] = rng.uniform(0.05, 0.5, size=B)
    T[:, 1:-1] = rng.normal(scale=0.1, size=(B, 128))
    T[:, -1] = 7
    net = stp.Mlp(B)
    net.set_params(PR.init_params(1))
    net.train_step(X, T, 0.0)
    net.set_profiling(True)
    for _ in range(reps):
        net.train_step(X, T, 0.0)
    gms, gfl, gby = net.profile()
    sms, nst = net.profile_step()
    net.close()
    peak = float(_peaks().get("bf16_tflops", 1917.3))
    hbm = float(_peaks().get("hbm_gbs", 6801.7))
    tf = gfl / (gms * 1e-3) / 1e12 if gms > 0 else 0.0
    gbs = gby / (gms * 1e-3) / 1e9 if gms > 0 else 0.0
    return {"batch": B, "gemm_ms_per_step": gms / reps, "gemm_flops_per_step": gfl / reps,
            "gemm_bytes_per_step": gby / reps, "tflops": tf, "peak_tflops": peak, "frac": tf / peak,
            "gbs": gbs, "peak_gbs": hbm, "hbm_frac": gbs / hbm,
            "train_ms_per_step": sms / nst if nst else None,
            "train_note": "device time of the whole training step (input packing, forward chain, loss, backward "
                          "pass, gradient sums, Adam), CUDA events on the network's stream, inputs staged",
            "note": "BF16 tcgen05 GEMMs of forward + backward training steps; CUDA events around the forward "
                    "chain (four products) and around the backward pass (input gradients on the main stream, "
                    "weight gradients beside them), GEMM launches only; algorithmic bytes over the logical layer "
                    "shapes; K = 256 products at about 100 flop/byte sit below the BF16 ridge (about 290), "
                    "so HBM bounds them"}


def learned(args, rank):
    """Learned proposal study on the 7-DoF distribution (seeded DH, 48 link
    spheres, 64 obstacles on 8-waypoint paths, 60 s horizon): training data
    from plain batched plans of the training problems (both allocation
    variants, two planner seeds), the proposal network trained on the tensor
    cores with validation early stopping, then the held-out problems planned
    plain and learned (batched, same W and iteration budget), a sample of them
    planned one at a time, and the network's GEMM throughput at a large
    training batch."""
    import dataclasses

    from paper_2609_30533_gb300 import proposal as PR
    from paper_2609_30533_gb300 import stp

    W, iters = args.learned_workers, args.learned_iters

    def make(split, idxs, learned_flag=0, variant=1, seed=None):
        out = []
        for i in idxs:
            prob, prm = WL.arm7_c4(split, i)
            prm = dataclasses.replace(prm, variant=variant, workers=W, max_iters=iters,
                                      seed=(prm.seed if seed is None else seed))
            out.append(stp.problem_from(prob, prm, precision=0, iters_per_graph=16, learned=learned_flag))
        return out

    def run_chunks(split, n, learned_flag, variant, net=None, seed=None):
        outs, X, T = [], [], []
        for c in range(0, n, 512):
            probs = make(split, range(c, min(n, c + 512)), learned_flag, variant, seed)
            if net is not None:
                PR.install(net, probs)
            o = PR.plan_batch(probs)
            if split == "train":
                x, t = PR.collect(probs, o)
                X.append(x)
                T.append(t)
            outs.append(o)
            for P in probs:
                P.close()
        o = PR.Outcome(np.concatenate([x.solved for x in outs]), np.concatenate([x.first_ms for x in outs]),
                       np.concatenate([x.first_iter for x in outs]), np.concatenate([x.U for x in outs]),
                       float(sum(x.batch_ms for x in outs)))
        return o, X, T

    t0 = time.time()
    Xs, Ts = [], []
    for variant in (1, 0):
        for sd in (0, 1):
            _, X, T = run_chunks("train", args.learned_train, 0, variant, seed=sd)
            Xs += X
            Ts += T
    X, T = np.concatenate(Xs), np.concatenate(Ts)
    gen_s = time.time() - t0
    net = stp.Mlp(4096)
    net.set_params(PR.init_params(rank))
    t1 = time.time()
    log = PR.train(net, X, T, args.learned_steps, 128, 3e-4, seed=rank)
    train_s = time.time() - t1

    def arm(o):
        return {"solved": int(o.solved.sum()), "success_rate": float(o.solved.mean()), "batch_ms": o.batch_ms}

    res = {}
    solvable = {}
    for variant, name in ((1, "recycling"), (0, "interval")):
        op, _, _ = run_chunks("test", args.learned_test, 0, variant)
        ol, _, _ = run_chunks("test", args.learned_test, 1, variant, net=net)
        solvable[variant] = np.nonzero(op.solved | ol.solved)[0][:args.learned_single]
        res[name] = {"plain_batched": arm(op), "learned_batched": arm(ol), "paired": _paired(op, ol)}
    # One problem at a time on held-out problems that either batched arm
    # solved (the first --learned-single of them), plain and learned.
    single = {}
    for variant, name in ((1, "recycling"), (0, "interval")):
        for flag, arm_name in ((0, "plain"), (1, "learned")):
            probs = make("test", [int(i) for i in solvable[variant]], flag, variant)
            if flag:
                PR.install(net, probs)
            fs = []
            for P in probs:
                out = P.plan()
                if out.stats["first_solution_iter"] >= 0:
                    fs.append(out.stats["first_solution_ms"])
                P.close()
            single["%s_%s" % (name, arm_name)] = {
                "problems": len(probs), "solved": len(fs),
                "p50_first_ms": float(np.median(fs)) if fs else None}
    net.close()
    return {
        "workload": "7-DoF seeded DH, 48 spheres, 64 obstacles, H 60 s; W %d, %d iterations" % (W, iters),
        "train": {"problems": args.learned_train, "runs_per_problem": 4, "samples": int(len(X)),
                  "gen_s": gen_s, "steps": args.learned_steps, "best_step": log.best_step,
                  "val_loss_first": log.val[0][1], "val_loss_best": log.best_val, "train_s": train_s},
        "heldout_problems": args.learned_test,
        "batched": res,
        "single_sample": single,
        "mlp_gemm": mlp_throughput(rank),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters", type=int, default=32, help="planner iterations per step")
    ap.add_argument("--ref-iters", type=int, default=1)
    ap.add_argument("--cpu-iters", type=int, default=8)
    ap.add_argument("--cpu-batch-problems", type=int, default=0, help="0 = one per host core (at most 32)")
    ap.add_argument("--cpu-batch-iters", type=int, default=2)
    ap.add_argument("--micro-edges", type=int, default=1 << 20)
    ap.add_argument("--micro7-edges", type=int, default=1 << 16)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batch-problems", type=int, default=512)
    ap.add_argument("--batch-iters", type=int, default=64)
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--tune-iters", type=int, default=24)
    ap.add_argument("--plain-sample", type=int, default=48)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--learned-train", type=int, default=2048)
    ap.add_argument("--learned-test", type=int, default=1000)
    ap.add_argument("--learned-steps", type=int, default=1500)
    ap.add_argument("--learned-workers", type=int, default=256)
    ap.add_argument("--learned-iters", type=int, default=96)
    ap.add_argument("--learned-single", type=int, default=32)
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-micro", action="store_true", help="skip the collision microbenchmarks")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--c0-iters", type=int, default=2000)
    ap.add_argument("--c0-problems", type=int, default=16)
    ap.add_argument("--c2-iters", type=int, default=48)
    ap.add_argument("--c2-problems", type=int, default=8)
    ap.add_argument("--sweep-problems", type=int, default=64)
    ap.add_argument("--sweep-iters", type=int, default=64)
    ap.add_argument("--only", default="", choices=["", "micro", "batch", "learned", "mlp", "sweep", "configs"],
                    help="micro: run only the collision microbenchmark (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2609_30533_gb300 import build as B
    B.build()
    from paper_2609_30533_gb300 import stp

    prob, prm = WL.ur5e(rank)
    P = stp.problem_from(prob, prm, precision=0, max_iters=args.iters, iters_per_graph=args.iters)
    stream = torch.cuda.Stream()
    P.set_stream(stream.cuda_stream)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    if args.only == "micro":
        micro, peak = microbench(args, P, prob, prm, stream, flush, rank, local)
        m7 = microbench_arm7(args, stream, flush, rank, local)
        print(json.dumps({"microbench": dict(micro, n_edges=args.micro_edges, peak_tflops=peak),
                          "microbench_arm7": m7}))
        return
    if args.only == "batch":
        print(json.dumps({"batched": batched(args, rank)}))
        return
    if args.only == "learned":
        print(json.dumps({"learned": learned(args, rank)}))
        return
    if args.only == "mlp":
        print(json.dumps({"mlp_gemm": mlp_throughput(rank)}))
        return
    if args.only == "sweep":
        print(json.dumps({"sweep": sweep(args, rank)}))
        return
    if args.only == "configs":
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        pk = fp32_peak_tflops(n_sm, float(_peaks().get("sm_max_mhz", 2070.0)))
        print(json.dumps({"configs": stated_configs(args, pk)}))
        return

    def step_timed():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = P.plan()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    # Clock samples cover the warm-up, the timed steps, the kernel-timing pass
    # and the end-to-end pass.
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        step_timed()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # Step time: the library's CUDA events on its stream around every GPU
    # operation of the stp_plan call (memsets, reset, iterations, path
    # extraction, statistics copy). The bench's own events around the call
    # (host_ms) also hold the GPU idle while the host synchronises and
    # returns; they are reported beside it.
    total_ms = 0.0
    host_ms = 0.0
    edges = 0
    launches = 0
    plan_ms = []
    fs_ms = []
    for k in range(args.steps):
        ms, out = step_timed()
        host_ms += ms
        total_ms += out.stats["step_ms"]
        st = out.stats
        edges += st["edges_validated"] + st["bridges_validated"]
        plan_ms.append(st["plan_ms"])
        if st["first_solution_ms"] >= 0:
            fs_ms.append(st["first_solution_ms"])
        launches += 2 + 8 * args.iters  # reset, 8 kernels per iteration, path extraction
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    # Kernel-timing pass: the same steps with CUDA events between the kernels
    # inside the captured graphs.
    prof_tot = {}
    pairs = points = 0
    nn_evals = br_evals = 0
    prof_step_ms = 0.0
    prof_error = None
    try:
        P.set_profiling(True)
        for k in range(args.steps):
            ms, out = step_timed()
            prof_step_ms += ms
            for name, (kms, n) in P.profile().items():
                a = prof_tot.setdefault(name, [0.0, 0])
                a[0] += kms
                a[1] += n
            pairs += out.stats["pair_tests"]
            points += out.stats["check_points"]
            nn_evals += out.stats["nn_evals"]
            br_evals += out.stats["bridge_evals"]
    except Exception as exc:  # report, keep the measured value
        prof_error = str(exc)
        prof_tot = {}
    finally:
        P.set_profiling(False)

    # End to end through the C ABI with host buffers: create (H2D of the
    # problem), plan, read the path back (D2H), free.
    h2d = sum(np.asarray(a, dtype=np.float64).nbytes for a in
              (prob.dh, prob.qlo, prob.qhi, prob.spheres, prob.obs_r, prob.way, prob.qs, prob.qg))
    e2e_edges = 0
    d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        Q = stp.problem_from(prob, prm, precision=0, max_iters=args.iters)   # library default graph size
        out = Q.plan(cap=4096)
        e2e_edges += out.stats["edges_validated"] + out.stats["bridges_validated"]
        d2h = out.path.size * 8 + 8 * 16
        Q.close()
    torch.cuda.synchronize()
    e2e_secs = time.perf_counter() - t0
    clk = clocks.stop()

    # The same plan as one persistent launch (STP_LAUNCH_PERSISTENT), for comparison.
    Pp = stp.problem_from(prob, prm, precision=0, max_iters=args.iters, launch_mode=stp.STP_LAUNCH_PERSISTENT)
    Pp.set_stream(stream.cuda_stream)
    pers_ms = []
    for k in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Pp.plan()
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            pers_ms.append(e0.elapsed_time(e1))
    pers_prof = Pp.profile()
    Pp.close()
    persistent_single = {"ms_per_step": statistics.median(pers_ms),
                         "step_us_per_iteration": {k: v[0] * 1e3 / max(v[1], 1) for k, v in pers_prof.items()},
                         "note": "the timed plan as one persistent cooperative launch (steps separated by "
                                 "device-wide barriers); step times barrier to barrier on the device timer"}

    if args.no_micro:
        micro, micro7 = None, None
        peak = fp32_peak_tflops(torch.cuda.get_device_properties(local).multi_processor_count,
                                float(_peaks().get("sm_max_mhz", 2070.0)))
    else:
        micro, peak = microbench(args, P, prob, prm, stream, flush, rank, local)
        micro7 = microbench_arm7(args, stream, flush, rank, local)
    batch_result = None if args.no_batch else batched(args, rank)
    learned_result = None if args.no_learned else learned(args, rank)
    sweep_result = None if args.no_sweep else sweep(args, rank)
    configs_result = None if args.no_configs else stated_configs(args, peak)
    n = args.micro_edges
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = float(_peaks().get("sm_max_mhz", 2070.0))

    edges_all, ms_max, e2e_edges_all, e2e_max = aggregate_over_ranks(edges, total_ms, e2e_edges, e2e_secs,
                                                                     dist, "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    value = edges_all / (ms_max * 1e-3)
    traffic, traffic_note = _capture_traffic()
    kv = prof_tot.get("k_validate(ext)", [0.0, 0])
    kb = prof_tot.get("k_validate(bridge)", [0.0, 0])
    val_ms = kv[0] + kb[0]
    val_launches = kv[1] + kb[1]
    flops = pairs * 8 + points * point_flops(prob)
    step_flops = (flops + (nn_evals + br_evals) * (3 * prob.dof + 5)) / max(args.steps, 1)
    achieved = flops / (val_ms * 1e-3) / 1e12 if val_ms > 0 else 0.0
    kernels = {k: {"ms_total": round(v[0], 4), "launches": v[1],
                   "share": round(v[0] / max(sum(x[0] for x in prof_tot.values()), 1e-12), 4)}
               for k, v in prof_tot.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "ms_per_step_call": host_ms / args.steps,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "iters_per_step": args.iters, "workers": prm.workers,
                   "n_roots": prm.n_roots, "l2": "flushed between steps (512 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": e2e_edges_all / e2e_max, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "note": "per step: stp_create_problem from host arrays, stp_plan, path read back, stp_free"},
        "gpu_launches": launches * world,
        "roofline": {"bound": "alu", "kernel": "k_validate", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                     "traffic": traffic, "traffic_note": traffic_note,
                     "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz (max SM clock)" % (
                         n_sm, max_mhz),
                     "launches": val_launches, "avg_launch_ms": val_ms / max(val_launches, 1),
                     "flops_per_launch": flops / max(val_launches, 1)},
        # The whole planner step against the FP32 peak: algorithmic flops of
        # the collision checks (pair tests x 8 + per-point FK, transforms and
        # interpolation) and of the NN and bridge scans ((3d + 5) per
        # (query, vertex) evaluation), over the timed step time.
        "roofline_step": {
            "bound": "alu", "unit": "TFLOP/s", "peak": peak,
            "flops_per_step": step_flops,
            "achieved": step_flops / (ms_max / args.steps * 1e-3) / 1e12,
            "frac": step_flops / (ms_max / args.steps * 1e-3) / 1e12 / peak if peak else None},
        "kernels": kernels,
        "profiled_ms_per_step": prof_step_ms / args.steps,
        "profiling_error": prof_error,
        "plan_ms_p50": statistics.median(plan_ms),
        "first_solution_ms_p50": statistics.median(fs_ms) if fs_ms else None,
        "microbench": dict(micro, n_edges=n, peak_tflops=peak) if micro is not None else None,
        "persistent_single": persistent_single,
        "microbench_arm7": micro7,
    }
    if clk:
        line["clocks"] = clk
    if not args.no_batch:
        line["batched"] = batch_result
    if not args.no_learned:
        line["learned"] = learned_result
    if not args.no_sweep:
        line["sweep"] = sweep_result
    if not args.no_configs:
        line["configs"] = configs_result
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
