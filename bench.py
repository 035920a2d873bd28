#!/usr/bin/env python3
"""Benchmark of the batched growth step (robot-link-steps per second).

Workload: 4096 robots x 100 links of 1.5 cm, radius U[2, 4] cm, pressure
U[2, 10] kPa, 0-6 sPAM actuators, 20 circles + 20 boxes each in a 1.5 m box
(seeded synthetic scenes), every robot grown from one link to 100 links with
every step solved to the equilibrium tolerance 1e-6.  One bench step = one
vine_simulate call over the whole batch (a robot-link-step is one link
present during one growth step: 100*101/2 per robot).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the
host cores (a bounded sample of the same workload per step).  Under torchrun
each rank grows its own replica of the workload (weak scaling, no
collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "robot-link-steps/s at equilibrium tol 1e-6 on 1 GB300 (batched/served vs plain); p50/p99 latency"
UNIT = "robot-link-steps/s"
WORKLOAD = "design-optimisation batch: 4096 robots x 100 links (1.5 cm), 20 circles + 20 boxes, 0-6 sPAM actuators"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) of one growth launch per robot, from an ncu
# capture of one launch over 1024 robots x 100 links of this workload:
# designs and obstacles are read once per robot, so traffic scales with robots.
GROW_DRAM_BYTES_PER_ROBOT = (1.431296e6 + 9.216e3) / 1024


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.samples, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        rows = [r for r in self.samples if len(r) >= 8]
        if rows:
            sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
            mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
            out["sm_mhz"] = float(np.median(sm)) if sm else None
            out["sm_max_mhz"] = max(mx) if mx else None
            names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
            out["reasons"] = sorted({n for r in rows for n, v in zip(names, r[4:8]) if v.lower() == "active"})
            out["samples"] = len(rows)
        return out


def _hbm_fraction(traffic_bytes, launch_s):
    """DRAM bytes per launch over the launch time, against the measured copy
    bandwidth (MEASURED_PEAKS.json; the fallback 6.8 TB/s if it is absent)."""
    peak, src = 6800.0, "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, src = float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        pass
    if traffic_bytes is None:
        return None
    gbs = traffic_bytes / launch_s / 1e9
    return {"achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak, "peak_source": src}


def reduce_over_ranks(seconds: float, units: float, device: str):
    """Whole-job figures under torchrun: the slowest rank's time and the sum
    of the units all ranks processed (weak scaling, one replica per rank)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def run_gpu(args):
    import torch

    from paper_2509_15180_gb300 import scenes, vine

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if ws > 1 and args.shard == "lpt":
        # one batch split over the ranks (strong scaling): LPT shards by cost
        from paper_2509_15180_gb300 import shard
        full = scenes.design_batch(args.robots)
        sc = scenes.subset(full, shard.lpt_partition(shard.robot_cost(full), ws)[rank])
    else:
        sc = scenes.design_batch(args.robots, replicate=rank)  # a replica per rank (weak scaling)
    rls_per_step = scenes.robot_link_steps(sc["n_links"])
    stream = torch.cuda.current_stream()
    dsc = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in sc.items()}
    prm = vine.vine_params_default()
    prm.threads_per_robot = args.threads_per_robot
    b = vine.Batch(dsc, prm, stream=stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step():
        b.reset(stream)
        b.simulate(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    stats = b.stats(stream)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    conv_rls = 0
    for k in range(args.steps):
        flush.zero_()  # L2 flush outside the timed interval
        b.reset(stream)
        starts[k].record(stream)
        b.simulate(stream)
        ends[k].record(stream)
        torch.cuda.synchronize()
        conv_rls += b.stats(stream)["robot_link_steps"]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    step_ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    total_s = float(step_ms.sum()) / 1e3
    if ws > 1:
        total_s, conv_all = reduce_over_ranks(total_s, conv_rls, "cuda")
    else:
        conv_all = float(conv_rls)
    value = conv_all / total_s
    st_last = b.stats(stream)
    rc = b.robot_counters(stream)
    cyc_ms = rc["cycles"] / 2.07e6  # at the maximum SM clock
    robots = {"mean_ms": float(cyc_ms.mean()), "p99_ms": float(np.percentile(cyc_ms, 99)),
              "max_ms": float(cyc_ms.max()), "evals_mean": float(rc["evals"].mean()),
              "evals_max": int(rc["evals"].max()),
              "what": "per-robot time its warp spent (clock64 at 2.07 GHz) in the last timed step"}

    # --- adjoint (vine_grad) at the final equilibria of the last timed step
    goals = torch.from_numpy(scenes.goal_points(len(sc["n_links"]), 1.5, replicate=rank)).cuda()
    b.grad(goals, stream)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    gout = b.grad(goals, stream)
    a1.record(stream)
    torch.cuda.synchronize()
    gstat = gout["status"].cpu().numpy()
    adjoint = {"ms": a0.elapsed_time(a1), "robots": int(gstat.size), "ok": int((gstat == 0).sum()),
               "not_pd": int((gstat == 1).sum()), "no_state": int((gstat == 2).sum()),
               "what": "one vine_grad launch: tip-distance cost and its derivatives w.r.t. every actuator's "
                       "pressure and span at every robot's final equilibrium"}

    # --- end to end through the C ABI with host buffers (create/copy in, grow, read back)
    e2e_steps = 0 if args.no_e2e else max(2, min(args.steps, 5))
    host = {k: np.ascontiguousarray(v) for k, v in sc.items()}
    h2d = int(sum(v.nbytes for v in host.values()))
    T = int(sc["n_links"].sum())
    n = len(sc["n_links"])
    d2h = T * 4 + T * 12 + n * (8 + 4 + 4 + 4 + 8 + 4)
    if e2e_steps:
        bw = vine.Batch(host, prm, stream=stream)  # warm (tables, graph) once
        bw.simulate(stream)
        bw.state(stream)
        bw.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_rls = 0
    for _ in range(e2e_steps):
        be = vine.Batch(host, prm, stream=stream)
        be.simulate(stream)
        out = be.state(stream)
        e2e_rls += int(be.stats(stream)["robot_link_steps"])
        be.close()
    e2e_s = time.perf_counter() - t0
    e2e = None if not e2e_steps else {
        "value": e2e_rls / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
        "ms_per_step": 1e3 * e2e_s / e2e_steps}

    # --- plain form: one launch per robot, same kernel (subset of the batch)
    n_plain = args.plain_robots
    plain = None
    if n_plain > 0:
        plain = _plain(scenes, vine, torch, sc, stream, n_plain, prm)

    # --- roofline of the growth kernel: algorithmic FP32 flops per launch
    # flops of the work the launch ran: 40 per link-evaluation, 10 per
    # disc-circle and 14 per disc-box test actually executed (the broad phase
    # skips obstacles out of reach; the circle share is the batch's)
    fc = st_last["circle_pair_tests"] / max(st_last["pair_tests"], 1)
    flops = (40.0 * st_last["link_evaluations"] +
             st_last["pair_tests_executed"] * (10.0 * fc + 14.0 * (1.0 - fc)))
    flops_all_pairs = (40.0 * st_last["link_evaluations"] + 10.0 * st_last["circle_pair_tests"] +
                       14.0 * (st_last["pair_tests"] - st_last["circle_pair_tests"]))
    launch_s = float(np.mean(step_ms)) / 1e3
    achieved = flops / launch_s / 1e12
    # the algorithmic work of the method: I W per robot-link-step, I the Newton
    # iterations per growth step, W = 40 + K_s (10 N_circ + 14 N_box) flops
    # per link and iteration (1000 for 20 circles and 20 boxes, K_s = 2)
    n_obs = np.diff(sc["obs_ptr"]).astype(np.int64)
    n_c = np.bincount(np.repeat(np.arange(n_obs.size), n_obs), weights=(sc["obs_kind"] == 0), minlength=n_obs.size)
    W = float(np.mean(40.0 + 2.0 * (10.0 * n_c + 14.0 * (n_obs - n_c))))
    iters_per_step = st_last["iterations"] / max(st_last["steps_total"], 1)
    flops_s8d = st_last["robot_link_steps"] * iters_per_step * W
    traffic = args.traffic if args.traffic is not None else GROW_DRAM_BYTES_PER_ROBOT * n
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                "frac_s8d": flops_s8d / launch_s / 1e12 / FP32_PEAK_TFLOPS,
                "flops_s8d_per_launch": flops_s8d,
                "s8d_what": "robot-link-steps x Newton iterations per step (%.2f) x W = %.0f flops per link and "
                            "iteration (40 + K_s (10 N_circ + 14 N_box))" % (iters_per_step, W),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a 1024-robot launch, "
                                  "scaled by robots",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (derived; MEASURED_PEAKS has no FP32 figure)",
                "flops_per_launch": flops,
                "hbm": _hbm_fraction(traffic, launch_s),
                "all_pairs_flops_per_launch": flops_all_pairs,
                "pair_tests_executed_fraction": st_last["pair_tests_executed"] / max(st_last["pair_tests"], 1)}

    result = None
    # the serving and uneven-batch legs describe one GPU: they run at N = 1
    serve = None
    if ws == 1 and not args.no_serve:
        serve = serve_leg(args, vine, scenes)
    uneven = None
    if ws == 1 and args.uneven_robots > 0:
        uneven = uneven_leg(args, vine, scenes, torch, stream, flush)
    overlapped = None
    if ws == 1 and not args.no_overlap:
        overlapped = overlapped_leg(args, vine, scenes, torch, sc)
    robust = None
    if ws == 1 and args.robust_perturb > 0:
        robust = robust_leg(args, vine, scenes, torch, stream, flush)
    stud = studies_leg(args) if ws == 1 and args.robust_trials > 0 else None
    plan = None
    if ws == 1 and args.plan_seconds > 0:
        plan = planner_leg(args, scenes)
    synth_r = synthesis_leg(args) if ws == 1 and args.synth_targets > 0 else None
    surr = surrogate_leg(args) if ws == 1 and args.surrogate_steps > 0 else None
    if rank == 0:
        cpu = cpu_baseline(args, sc) if ws == 1 and not args.no_cpu else None
        if cpu is not None and args.cpu_other_robots > 0:
            cpu["other_configs"] = cpu_other_configs(args)
        lat = {"p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
               "what": "latency of one whole-batch simulate call"}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
            "scaling": "strong" if (ws > 1 and args.shard == "lpt") else "weak", "vs_baseline": None,
            "dtype": "f32 (f64 residual test)", "data": "synthetic",
            "config": {"workload": WORKLOAD if n == 4096 else WORKLOAD.replace("4096", str(n)),
                       "robots_per_gpu": n, "links": 100, "threads_per_robot": b.launch()["threads_per_robot"],
                       "robot_link_steps_per_step": rls_per_step, "l2": "flushed between timed steps (512 MiB write)",
                       "tol": 1e-6},
            "e2e": e2e, "plain": plain, "latency": lat, "roofline": roofline, "cpu_baseline": cpu,
            "adjoint": adjoint, "serving": serve, "uneven": uneven, "robustness": robust,
            "overlapped": overlapped, "planner": plan, "synthesis": synth_r, "surrogate": surr, "studies": stud,
            "clocks": ck, "gpu_launches": args.steps, "robots": robots,
            "solver": {"iters_per_step": st_last["iterations"] / max(st_last["steps_total"], 1),
                       "evals_per_step": st_last["evaluations"] / max(st_last["steps_total"], 1),
                       "steps_converged": st_last["steps_converged"], "steps_total": st_last["steps_total"],
                       "robots_maxiter": st_last["n_maxiter"], "robots_nonfinite": st_last["n_nonfinite"],
                       "gn_fallbacks_per_step": st_last["gn_fallbacks"] / max(st_last["steps_total"], 1)},
        }
    b.close()
    if ws > 1:
        dist.destroy_process_group()
    return result


def _plain(scenes, vine, torch, sc, stream, n_plain, prm=None):
    """Plain form: one launch per robot, same kernel, on the first robots."""
    sub = scenes.subset(sc, np.arange(n_plain))
    bp = vine.Batch(sub, prm, stream=stream)
    bp.simulate_plain(stream)
    torch.cuda.synchronize()
    bp.reset(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bp.simulate_plain(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_s = e0.elapsed_time(e1) / 1e3
    out = {"value": bp.stats(stream)["robot_link_steps"] / plain_s, "unit": UNIT, "robots": n_plain,
           "launches": n_plain, "note": "one launch per robot, sequential; the first %d robots" % n_plain}
    bp.close()
    return out


def serve_leg(args, vine, scenes):
    """Serving loop on request streams shaped like the serving workload
    (each request U{1..256} robots drawn as the uneven batch with U{20..300}
    links and 5-200 obstacles).  A pool of distinct requests is generated once
    and cycled.  (1) capacity: closed loop, the client keeps the server's
    slots full; robot-link-steps of the requests completed inside the window;
    (2) Poisson arrivals at 70 % of that capacity: p50/p99 latency from
    arrival to completion; (3) Poisson arrivals at 2000 requests/s (the
    workload's rate, far beyond capacity): achieved vs offered.  Each phase
    drains before the next."""
    import threading

    pool_t, pool = scenes.serve_requests(args.serve_pool, rate_hz=2000.0)
    sizes = [(int(len(r["n_links"])), scenes.robot_link_steps(r["n_links"])) for r in pool]
    srv = vine.Server(max_slots=args.serve_slots, max_links=320, max_obs=200, max_act=8, max_request=256,
                      steps_per_tick=args.serve_tick, lanes=args.serve_lanes, window=args.serve_window)

    def run(rate, duration):
        """Submissions for `duration` s: open loop at `rate` req/s (None:
        closed loop).  Returns [(arrival, done, rls)] relative to the start,
        the number submitted, and the drain end."""
        rng = np.random.default_rng(55)
        done, lock = [], threading.Lock()
        outstanding = {}
        stop = [False]
        t0 = vine.serve_clock()

        def poller():
            while not stop[0] or outstanding:
                with lock:
                    items = list(outstanding.items())
                for rid, t_arr in items:
                    r = srv.poll(rid, timeout_us=0)
                    if r is not None:
                        with lock:
                            outstanding.pop(rid, None)
                            done.append((t_arr - t0, r["t_done"] - t0, r["rls"]))
                time.sleep(0.0005)

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        k, t_next = 0, t0
        while vine.serve_clock() - t0 < duration:
            now = vine.serve_clock()
            if rate is None:
                t_arr = now
            else:
                if now < t_next:
                    time.sleep(min(t_next - now, 0.001))
                    continue
                t_arr = t_next
                t_next += rng.exponential(1.0 / rate)
            rid = srv.submit(pool[k % len(pool)])
            while rid is None and vine.serve_clock() - t0 < duration:  # slots full: retry
                time.sleep(0.0005)
                rid = srv.submit(pool[k % len(pool)])
            if rid is None:
                break
            with lock:
                outstanding[rid] = t_arr
            k += 1
        stop[0] = True
        th.join(timeout=300.0)
        return done, k, vine.serve_clock() - t0

    out = {}
    warm = 3.0
    done, k, t_end = run(None, args.serve_seconds)
    win = [d for d in done if warm <= d[1] <= args.serve_seconds]
    span = args.serve_seconds - warm
    cap_req = len(win) / span
    out["capacity"] = {"requests_per_s": cap_req, "robot_link_steps_per_s": sum(d[2] for d in win) / span,
                       "requests": len(win), "window_s": span}
    rate = max(0.7 * cap_req, 0.2)
    done, k, t_end = run(rate, args.serve_seconds + 2.0)
    kept = [d for d in done if d[0] >= 2.0]
    lat = np.array([d[1] - d[0] for d in kept]) if kept else np.full(1, np.nan)
    win = [d for d in done if 2.0 <= d[1] <= args.serve_seconds + 2.0]
    out["poisson"] = {"offered_requests_per_s": rate, "requests": len(kept),
                      "robot_link_steps_per_s": sum(d[2] for d in win) / args.serve_seconds,
                      "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99))}
    done, k, t_end = run(2000.0, 3.0)
    win = [d for d in done if d[1] <= 3.0]
    out["offered_2000"] = {"offered_requests_per_s": 2000.0, "submitted": k, "completed_in_3s": len(win),
                           "achieved_requests_per_s": len(win) / 3.0,
                           "note": "submission blocks while the slots are full, so arrivals fall behind"}
    st = srv.stats()
    out.update({"slots": st["max_slots"], "steps_per_tick": args.serve_tick, "lanes": args.serve_lanes,
                "launches": st["ticks"], "pool": len(pool),
                "mean_robots_per_request": float(np.mean([s[0] for s in sizes])),
                "mean_robot_link_steps_per_request": float(np.mean([s[1] for s in sizes])),
                "what": "vine_server continuous batching; latency = completion - arrival (queueing included)"})
    srv.close()
    return out


def uneven_leg(args, vine, scenes, torch, stream, flush):
    """Uneven persistent batch (links U{30..300}, 0-8 actuators, 5-200
    obstacles): robot-link-steps/s of vine_simulate with the launch
    configuration picked at creation, then after vine_autotune on a sample.
    Threads per robot from --uneven-threads-per-robot (0: the library's
    choice by robot length, four warps for these robots)."""
    sc = scenes.uneven_batch(args.uneven_robots)
    prm = vine.vine_params_default()
    prm.threads_per_robot = args.uneven_threads_per_robot
    b = vine.Batch(sc, prm, stream=stream)

    def timed(k):
        b.reset(stream)
        b.simulate(stream)  # warm (records the graph)
        torch.cuda.synchronize()
        ms, rls = [], 0
        for _ in range(k):
            flush.zero_()
            b.reset(stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.simulate(stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            rls += b.stats(stream)["robot_link_steps"]
        return rls / (sum(ms) / 1e3), float(np.mean(ms))

    v0, ms0 = timed(2)
    st0 = b.stats(stream)
    cls0 = b.classes()
    t0 = time.perf_counter()
    tune = b.autotune(args.uneven_sample, stream)
    tune_s = time.perf_counter() - t0
    v1, ms1 = timed(2)
    cls1 = b.classes()
    b.close()
    shape = lambda cl: [{k: c[k] for k in ("threads_per_robot", "robots", "robots_per_cta", "max_links")} for c in cl]
    return {"workload": "uneven batch: %d robots, links U{30..300} of U[1,3] cm, 5-200 obstacles, 0-8 actuators"
                        % args.uneven_robots,
            "robot_link_steps_per_step": scenes.robot_link_steps(sc["n_links"]),
            "default": {"value": v0, "ms_per_step": ms0, "classes": shape(cls0),
                        "iters_per_step": st0["iterations"] / max(st0["steps_total"], 1),
                        "robots_maxiter": st0["n_maxiter"]},
            "autotuned": {"value": v1, "ms_per_step": ms1, "classes": shape(cls1), "adopted": tune["adopted"],
                          "list_margin_R": tune["list_margin"], "candidates": tune["candidates"],
                          "sample": tune["sample"], "sample_ms_default": tune["default_ms"],
                          "sample_ms_tuned": tune["best_ms"], "tuning_s": tune_s},
            "what": "one vine_simulate (length classes, one persistent launch each on a parallel graph branch) "
                    "with the classes' team sizes chosen at creation, then after vine_autotune",
            "unit": UNIT}


def robust_leg(args, vine, scenes, torch, stream, flush):
    """Robustness batch with gradients: designs of 150 links and 60 obstacles,
    each perturbed (obstacle centres, actuator ends, pressures); one
    vine_simulate plus one vine_grad (tip-to-goal distance and its
    derivatives w.r.t. every actuator's pressure and span) per step."""
    sc, goals = scenes.robustness_batch(n_designs=args.robust_designs, n_perturb=args.robust_perturb)
    b = vine.Batch(sc, stream=stream)
    g = torch.from_numpy(goals).cuda()
    b.simulate(stream)
    b.grad(g, stream)
    torch.cuda.synchronize()
    ms_f, ms_g, rls = [], [], 0
    for _ in range(args.robust_repeats):
        flush.zero_()
        b.reset(stream)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        b.simulate(stream)
        e1.record(stream)
        out = b.grad(g, stream)
        e2.record(stream)
        torch.cuda.synchronize()
        ms_f.append(e0.elapsed_time(e1))
        ms_g.append(e1.elapsed_time(e2))
        rls += b.stats(stream)["robot_link_steps"]
    st = out["status"].cpu().numpy()
    stats = b.stats(stream)
    b.close()
    return {"workload": "robustness batch: %d designs x %d perturbations, 150 links, 60 obstacles, 2.25 m box"
                        % (args.robust_designs, args.robust_perturb),
            "value": rls / (sum(ms_f) / 1e3), "unit": UNIT, "simulate_ms": float(np.mean(ms_f)),
            "grad_ms": float(np.mean(ms_g)), "grad_ok": int((st == 0).sum()), "robots": int(st.size),
            "iters_per_step": stats["iterations"] / max(stats["steps_total"], 1), "robots_maxiter": stats["n_maxiter"]}


def studies_leg(args):
    """The analysis workloads (Sec. 6.3, 6.4): the robustness sweep (11
    uncertainty levels 0-20 %, 1000 perturbed trials each, obstacle and
    actuation kinds, each kind one vine_simulate over all its levels) and the
    funnelling rollouts (50 start headings x 4 environments, one
    vine_simulate).  Wall time per launch includes batch creation and the
    read-back of the tips."""
    from paper_2509_15180_gb300 import studies
    r = studies.robustness(trials=args.robust_trials)
    f = studies.funnel()
    out = {"robustness": {k: {"success_rate": r[k]["success_rate"], "robots": r[k]["robots"],
                              "not_converged": r[k]["not_converged"], "seconds": r[k]["seconds"],
                              "robot_link_steps_per_s": r[k]["robot_link_steps"] / r[k]["seconds"]}
                          for k in ("obstacles", "actuation")},
           "levels": list(r["levels"]), "trials_per_level": r["trials"], "goal_radius_m": r["goal_radius"],
           "funnel": {"obstacles": f["obstacles"], "rollouts": f["rollouts"],
                      "knn_concentration_ratio": f["ratio"], "seconds": f["seconds"],
                      "not_converged": f["not_converged"]},
           "what": "seeded stand-ins for the paper's environment and design (its figures only); success = grown "
                   "to full length with the tip within the goal radius of the nominal design's tip"}
    return out


def overlapped_leg(args, vine, scenes, torch, sc):
    """The design batch as a stream of independent batches: two batch
    instances alternate on two CUDA streams, so that one batch's last robots
    finish while the next batch fills the freed SMs (as a robustness study
    or a sweep over independent design sets would run).  No L2 flush between
    steps (the working set of a batch is a few MB and the kernel does not
    depend on it)."""
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    prm = vine.vine_params_default()
    prm.threads_per_robot = args.threads_per_robot
    bs = [vine.Batch(sc, prm, stream=streams[q]) for q in range(2)]
    for q in range(2):
        bs[q].simulate(streams[q])
    torch.cuda.synchronize()
    k = max(4, 2 * args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ends = [torch.cuda.Event() for _ in range(2)]
    cur = torch.cuda.current_stream()
    e0.record(cur)
    for q in range(2):
        streams[q].wait_event(e0)
    for i in range(k):
        q = i % 2
        bs[q].reset(streams[q])
        bs[q].simulate(streams[q])
    for q in range(2):
        ends[q].record(streams[q])
        cur.wait_event(ends[q])
    e1.record(cur)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rls = sum(b.stats(streams[q])["robot_link_steps"] for q, b in enumerate(bs))  # last step of each
    for b in bs:
        b.close()
    per = scenes.robot_link_steps(sc["n_links"])
    return {"value": k * (rls / 2.0) / (ms / 1e3), "unit": UNIT, "batches": k, "ms_per_batch": ms / k,
            "robot_link_steps_per_batch": per,
            "what": "two instances of the design batch alternating on two streams; converged robot-link-steps"}


def planner_leg(args, scenes):
    """Batched SST* (Algorithm 2) on the channel planning environment: B
    expansions per iteration, each grown 5-20 links from its parent's stored
    state, pruned against the tree.  Reports the wall time per iteration (the
    paper's "iter time", Sec. 6.2 table: 5-7 s on its machine) split into its
    parts, and the first iteration that reached the goal."""
    from paper_2509_15180_gb300 import planner
    env = scenes.planning_env("channel")
    p = planner.Planner(env, planner.PlanConfig(batch=args.plan_batch, seed=0))
    p.run(2, stop_at_goal=False)  # warm-up: library state, tables, allocator
    p = planner.Planner(env, planner.PlanConfig(batch=args.plan_batch, seed=0))
    t0 = time.perf_counter()
    first_goal = None
    while time.perf_counter() - t0 < args.plan_seconds and p.i <= args.plan_iters:
        h = p.step()
        if h["goal"] and first_goal is None:
            first_goal = (h["iteration"], time.perf_counter() - t0)
    wall = time.perf_counter() - t0
    hist = p.history
    it_s = [h["t_select"] + h.get("t_build", 0.0) + h["t_sim"] + h["t_prune"] + h["t_host"] for h in hist]
    best = p.best_goal()
    rls = sum(h.get("robot_link_steps", 0) for h in hist)
    return {"iterations": len(hist), "batch": args.plan_batch, "wall_s": wall,
            "ms_per_iteration_median": 1e3 * float(np.median(it_s)),
            "ms_parts_median": {k: 1e3 * float(np.median([h.get(k, 0.0) for h in hist]))
                                for k in ("t_select", "t_build", "t_sim", "t_prune", "t_host")},
            "expansions_per_s": sum(h["expanded"] for h in hist) / wall,
            "robot_link_steps_per_s": rls / wall, "tree_nodes": p.size,
            "active_nodes": int(p.active[: p.size].sum()), "radius": p.radius,
            "first_goal": None if first_goal is None else {"iteration": first_goal[0], "seconds": first_goal[1]},
            "best_cost": None if best is None else float(p.cost[best]),
            "what": "channel environment (88 circles, 90-degree bend, goal 1.9 m of corridor away); wall clock "
                    "per iteration including the host tree"}


def synthesis_leg(args):
    """Actuator design synthesis (Sec. 4.2) for a batch of target angles per
    joint: 10 pressures x 61 cell lengths (1 mm grid), the paper's body.
    Wall time of one vine_synthesize call (pair equilibria, choices, host
    copies) after one warm-up call, which builds the grid's FP64 sPAM tables
    (kept for later calls on the grid; its time is reported beside)."""
    from paper_2509_15180_gb300 import vine
    rng = np.random.default_rng(0)
    targets = rng.uniform(0.005, 0.11, args.synth_targets)
    kw = dict(R=0.03335, P_vine=10342.0, l_seg=0.025, pressures=np.arange(10e3, 100e3 + 1, 10e3), l0_min=0.020,
              l0_step=0.001, n_l0=61, tol=0.004)
    t0 = time.perf_counter()
    vine.synthesize(targets[:16], **kw)
    first = time.perf_counter() - t0
    t0 = time.perf_counter()
    out = vine.synthesize(targets, **kw)
    wall = time.perf_counter() - t0
    return {"targets": int(targets.size), "pairs": 610, "ms": 1e3 * wall, "us_per_design": 1e6 * wall / targets.size,
            "first_call_ms": 1e3 * first, "first_call_targets": 16,
            "feasible": float(np.mean(out["p_index"] >= 0)),
            "what": "one vine_synthesize call: 610 pair equilibria and one choice per target, the grid's FP64 sPAM "
                    "tables (61 cell lengths) kept from the first call, which builds them (first_call_ms); paper: "
                    "milliseconds per numerical solve"}


def surrogate_leg(args):
    """The sPAM surrogate of Sec. 4.3: exact-model samples, training (40 000
    samples split 80/10/10, full-batch Adam), held-out normalised MSE
    (paper: 0.003), and throughput of the network against the exact model
    (paper: four orders of magnitude)."""
    import torch
    from paper_2509_15180_gb300 import surrogate, vine
    t0 = time.perf_counter()
    x, y, _ = surrogate.make_dataset(40000, 0)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = surrogate.train(40000, steps=args.surrogate_steps, lr=0.01)
    t_train = time.perf_counter() - t0 - t_data  # train() regenerates the same samples
    n = 1 << 22
    xi = torch.from_numpy(np.tile(x, (n // x.shape[0] + 1, 1))[:n].copy()).cuda()
    vine.surrogate_eval(r["net"], xi)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    vine.surrogate_eval(r["net"], xi)
    e1.record()
    torch.cuda.synchronize()
    net_per_s = n / (e0.elapsed_time(e1) / 1e3)
    exact_per_s = 40000 / t_data
    return {"samples": 40000, "steps": args.surrogate_steps, "train_s": t_train, "test_mse": r["test_mse"],
            "val_mse": r["val_mse"], "paper_mse": 0.003, "eval_per_s": net_per_s, "exact_model_per_s": exact_per_s,
            "speedup": net_per_s / exact_per_s,
            "what": "2-32-2 ReLU network (strain, cell length) -> (m, phi_Rc); exact model: vine_spam_samples "
                    "(FP64, one warp per sample, host round trip included); network: vine_surrogate_eval on "
                    "4M device-resident inputs, CUDA events"}


def cpu_baseline(args, sc, robots=None):
    """The FP64 oracle as it stands, OpenMP over robots on all host cores, on a
    bounded sample of the workload (the first `robots` robots)."""
    import oracle
    from paper_2509_15180_gb300 import scenes

    robots = robots or args.cpu_robots
    sub = scenes.subset(sc, np.arange(robots))
    orc = oracle.Oracle(sub)
    st = orc.new_state()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    orc.run(st, 100, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": float(st["rls"].sum()) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d robots of the workload, all 100 growth steps (%.1f s)" % (robots, dt)}


def cpu_other_configs(args):
    """The oracle on seeded subsets of the uneven batch (config 3) and the
    robustness batch (config 4), robot-link-steps per second of host time:
    the figures extrapolate to the full batches per robot-link-step."""
    import oracle
    from paper_2509_15180_gb300 import scenes

    out = {}
    cores = os.cpu_count() or 1
    k = args.cpu_other_robots
    # the uneven batch's first k robots (robots are drawn one after another);
    # k robustness designs with one perturbation each
    subs = (("uneven", scenes.uneven_batch(k), "the uneven batch's first %d robots"),
            ("robustness", scenes.robustness_batch(n_designs=k, n_perturb=1)[0],
             "%d robustness designs (150 links, 60 obstacles), one perturbation each"))
    for name, sub, what in subs:
        orc = oracle.Oracle(sub)
        st = orc.new_state()
        t0 = time.perf_counter()
        orc.run(st, int(sub["n_links"].max()), threads=cores)
        dt = time.perf_counter() - t0
        out[name] = {"value": float(st["rls"].sum()) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                     "sample": "%s (%.1f s)" % (what % k, dt)}
    return out


def run_reference(args):
    """Reference arm: the oracle on the host cores, same metric and workload."""
    from paper_2509_15180_gb300 import scenes

    ws, rank = _dist()
    if rank != 0:
        return None
    sc = scenes.design_batch(4096)
    vals, times = [], []
    for _ in range(args.warmup):
        cpu_baseline(args, sc, robots=8)
    for _ in range(args.steps):
        r = cpu_baseline(args, sc, robots=args.ref_robots)
        vals.append(r["value"])
        times.append(scenes.robot_link_steps(sc["n_links"][: args.ref_robots]) / r["value"])
    v = float(np.mean(vals))
    cores = os.cpu_count() or 1
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "robots_per_step": args.ref_robots},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "first %d robots of the workload per step" % args.ref_robots},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--robots", type=int, default=4096, help="robots per GPU (the workload has 4096)")
    ap.add_argument("--shard", default="replica", choices=["replica", "lpt"],
                    help="N > 1: a replica of the workload per rank (weak scaling) or one workload split over "
                         "the ranks by LPT on N^2 (K_s n_obs + 8) (strong scaling)")
    ap.add_argument("--threads-per-robot", type=int, default=0, choices=[0, 32, 64, 128],
                    help="design-batch legs: threads per robot (0: the library's choice by robot length)")
    ap.add_argument("--plain-robots", type=int, default=64)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-robots", type=int, default=96)
    ap.add_argument("--ref-robots", type=int, default=48)
    ap.add_argument("--cpu-other-robots", type=int, default=24,
                    help="CPU oracle on this many robots of the uneven and robustness batches (0: skip)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--traffic", type=float, default=None)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-overlap", action="store_true")
    ap.add_argument("--uneven-robots", type=int, default=16384)
    ap.add_argument("--uneven-threads-per-robot", type=int, default=0, choices=[0, 32, 64, 128])
    ap.add_argument("--uneven-sample", type=int, default=2048)
    ap.add_argument("--robust-designs", type=int, default=64)
    ap.add_argument("--robust-perturb", type=int, default=1024)
    ap.add_argument("--robust-repeats", type=int, default=1)
    ap.add_argument("--robust-trials", type=int, default=1000, help="studies leg: trials per uncertainty level (0: skip)")
    ap.add_argument("--plan-seconds", type=float, default=20.0, help="planner leg budget (0: skip)")
    ap.add_argument("--synth-targets", type=int, default=100000, help="design-synthesis leg targets (0: skip)")
    ap.add_argument("--surrogate-steps", type=int, default=3000, help="surrogate leg Adam steps (0: skip)")
    ap.add_argument("--plan-iters", type=int, default=60)
    ap.add_argument("--plan-batch", type=int, default=1024)
    ap.add_argument("--serve-seconds", type=float, default=12.0)
    ap.add_argument("--serve-pool", type=int, default=24)
    ap.add_argument("--serve-slots", type=int, default=32768)
    ap.add_argument("--serve-lanes", type=int, default=4)
    ap.add_argument("--serve-window", type=int, default=0, help="robots per launch and lane (0: the library's default)")
    ap.add_argument("--serve-tick", type=int, default=0, help="growth steps per launch (0: to completion)")
    args = ap.parse_args()
    res = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
