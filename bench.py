"""Throughput of the coupled MPM / rigid-body convex-contact substep on GB300.

Headline workload (the paper's mixed manipulation shape, the largest
single-GPU configuration): 4M particles in 32 objects (16 corotated elastic
with E log-uniform in [1e4, 1e6], 16 Drucker-Prager sand), 12 rigid bodies
(floor, a two-jaw parallel gripper closing on one object, nine static boxes,
capsules and spheres), dx = 2e-3 m on a block-sparse 320 x 184 x 64 grid,
h = 2.5e-5 s, N = 10 substeps per rigid time step, the solver at the paper's
default tolerance (eps_r = 5e-2). One bench step is one rigid time step
(radix sort + 10 substeps, each P2G + grid update + quasi-Newton contact
solve + G2P). The 1M-particle granular scooping workload is measured the same
way and reported under "workloads".

Metric: particle-substeps per second including the contact solve.
  value  device-resident: state in HBM, CUDA events around each mpm_step on the
         library's stream (CUDA-graph replay), L2 flushed (256 MB write)
         between timed steps.
  e2e    the same steps through the C ABI with host buffers: every step uploads
         the current rigid bodies from host memory, runs mpm_step and reads
         back the particle positions (pinned host memory) and the body
         impulses; L2 flushed between steps as above. It replays the first of
         the timed steps from the same start state.
  kernels / roofline  per-kernel CUDA-event times of a replay of the same
         steps with the library's phase events on (direct launches), against
         algorithmic bytes: P2G 96 B per
         particle (x, v, C, F) + 16 B per active grid node, G2P 144 B per
         particle (read x, F; write x, v, C, F).
Rank r of a torchrun job runs an independent replica on its own GPU (a single
scene does not shard); value sums the replicas over the slowest rank's time.

`--impl reference` times the FP64 CPU oracle (oracle/) on the machine's host
cores (its OpenMP build where it exists), one substep of the whole headline
workload per bench step.
"""
import argparse
import functools
import json
import os
import platform
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "particle-substeps/sec incl. contact solve"
UNIT = "particle-substeps/s"
WORKLOAD = "mixed_manipulation_4M"
SECONDARY = "granular_scoop_1M"
# algorithmic bytes (FP32 structure-of-arrays planes)
P2G_BYTES_PER_PARTICLE = 96        # read x, v, C, F
P2G_BYTES_PER_NODE = 16            # one (m, p) reduction per active node
G2P_BYTES_PER_PARTICLE = 144       # read x, F; write x, v, C, F
SOLVE_BYTES_PER_CONTACT = 48       # per QN iteration: the contact record
SOLVE_BYTES_PER_NODE = 60          # per QN iteration and contact node: v, v*, m, g, H, dv
L2_FLUSH_BYTES = 256 * 1024 * 1024


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws):
    """Max of a float over the ranks of the default process group (identity at ws = 1)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, ws):
    """Sum of a float over the ranks of the default process group (identity at ws = 1)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_value(units_per_rank, ws, max_seconds):
    """Units processed by all ranks divided by the slowest rank's time."""
    return units_per_rank * ws / max_seconds


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(kernel, workload, n):
    """DRAM bytes per launch from the committed ncu summary of the current
    kernel build, if one exists (line 'traffic_bytes_per_launch <kernel>
    <workload> <bytes> <particles>'), scaled to n particles."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) == 5 and parts[0] == "traffic_bytes_per_launch" and parts[1] == kernel \
                and parts[2] == workload:
            return float(parts[3]) * n / float(parts[4])
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "bench_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def start(self):
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [q.strip() for q in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


SMALL_SORT_MAX = 8192  # particles the library sorts in one thread block


def kernel_launches_per_step(res, n_substeps, n_bodies=0, n_particles=None):
    """Kernels one mpm_step launches: the sort (above 8,192 particles the
    radix sort: keys, five kernels per 8-bit digit pass, permutation; up to
    it one sorting block and the permutation), per substep P2G, block
    compaction, grid update, the two solve kernels (the cluster one and the
    cooperative one, of which the contact count picks one to work) and G2P,
    and with bodies the rigid update after the substeps."""
    if n_particles is not None and n_particles <= SMALL_SORT_MAX:
        sort = 2
    else:
        blocks = max(-(-int(r) // 4) for r in res)
        morton_bits = max((blocks - 1).bit_length(), 1)
        key_bits = 3 * morton_bits + (6 if 3 * morton_bits + 6 <= 32 else 0)
        sort = 1 + 5 * (-(-key_bits // 8)) + 1
    return sort + 6 * n_substeps + (1 if n_bodies > 0 else 0)


def shard(n_items, rank, ws):
    """The independent items (scenes) rank `rank` of `ws` takes: round robin,
    so that scenes of random size spread evenly."""
    return list(range(rank, n_items, ws))


def workload_name(sc):
    n = sum(len(g["x"]) for g in sc["groups"])
    kind = sc["name"].rsplit("_", 1)[0]
    return "%s_%dM" % (kind, round(n / 1e6)) if n >= 1_000_000 else sc["name"]


def bench_config(sc, n, ws):
    """The workload description shared by both arms' JSON lines."""
    models = sorted({int(g["material"]["model"]) for g in sc["groups"]})
    return {"workload": workload_name(sc), "particles": n,
            "materials": ["corotated_elastic" if m == 0 else "drucker_prager_sand" for m in models],
            "objects": len(sc["groups"]), "bodies": len(sc["bodies"]), "dx": sc["grid"]["dx"],
            "grid": list(sc["grid"]["res"]), "h": sc["h"], "substeps_per_step": sc["substeps"],
            "eps_r": 5e-2,
            "l2": "flushed between timed steps (256 MB write); particle state %d MB" %
                  round(126 * n / 1e6),
            "parallelism": "replica per GPU" if ws > 1 else "single GPU"}


def make_scene(name=WORKLOAD):
    from paper_2503_05046_gb300 import scenes
    if name == SECONDARY:
        return scenes.granular_scoop(n_particles=1_000_000)
    return scenes.mixed_manipulation()


def measure_workload(native, sc, args, ws, stream_flush=True, tight=True):
    """Device-resident throughput, kernel split, end-to-end throughput through
    the C ABI and a tightly solved step of one workload."""
    import torch
    n = sum(len(g["x"]) for g in sc["groups"])
    N = sc["substeps"]
    sim = native.Sim(sc, max_contacts=2 * n)
    stream = sim.torch_stream  # the library's stream: events and the L2 flush go here
    solver = native.solver_params(eps_r=5e-2, max_iters=args.max_iters)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        sim.step(solver=solver, stats=False, check=False)
    # the P2G form that is faster on this workload, timed on ordinary steps
    from paper_2503_05046_gb300 import tune
    (p2g_form, p2g_chunk), form_table = tune.tune_p2g_form(sim, solver, steps=2)
    sim.step(solver=solver, stats=False, check=False)  # records the step's graph again
    sim.step(n_substeps=0, solver=solver, check=False)  # drain warm-up status

    def timed_steps(k, stats=None):
        # stats: a list that takes each step's statistics (the read-back after
        # a step waits for it; only the phase-timed pass asks for them)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        torch.cuda.synchronize()
        for i in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
            starts[i].record(stream)
            _, st_i = native.mpm_step(sim.ctx, sc["h"], N, solver, want_stats=stats is not None)
            ends[i].record(stream)
            if stats is not None:
                stats.append(st_i)
        torch.cuda.synchronize()
        return [s.elapsed_time(e) for s, e in zip(starts, ends)]

    # every leg starts from the same state: the steps they time are the same
    st0, b0 = sim.get_particles(), sim.bodies()

    def restore():
        sim.set_particles(st0["x"], st0["v"], st0["C"], st0["F"])
        sim.set_bodies(b0)

    # --- headline: graph replay, CUDA events around each step
    if ws > 1:
        torch.distributed.barrier()
    step_ms = timed_steps(args.steps)
    if ws > 1:
        torch.distributed.barrier()
    ms = sum(step_ms)
    code_timed, _ = sim.step(n_substeps=0, solver=solver, check=False)
    seconds = max_over_ranks(ms / 1e3, ws)
    value = whole_job_value(float(n) * N * args.steps, ws, seconds)

    # --- e2e through the C ABI with host buffers (current bodies up, x and
    # impulses down every step) over the first of the same steps, with the
    # same L2 policy and graph replay
    restore()
    nb = len(sc["bodies"])
    x_host = torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy()
    imp_host = np.zeros(6 * max(nb, 1))
    arr = (native.RigidBody * max(nb, 1))()
    e2e_steps = max(3, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        native.lib.mpm_get_rigid_bodies(sim.ctx, nb, arr)   # host copy of the current bodies
        native.lib.mpm_set_rigid_bodies(sim.ctx, nb, arr)   # uploaded with the step
        with torch.cuda.stream(stream):
            flush.zero_()
        native.mpm_step(sim.ctx, sc["h"], N, solver, want_stats=False)
        native.mpm_get_particles(sim.ctx, x_host, None, None, None)
        native.lib.mpm_get_rigid_impulses(sim.ctx, imp_host.ctypes.data_as(native._dp), 1)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    e2e_value = whole_job_value(float(n) * N * e2e_steps, ws, e2e_s)
    same_steps_ms = sum(step_ms[:e2e_steps]) if e2e_steps <= len(step_ms) else None

    # --- kernel split: the same steps again with the phase events on
    restore()
    native.mpm_set_option(sim.ctx, native.OPT_PROFILE, 1)
    native.mpm_get_phase_times(sim.ctx, reset=True)
    prof_stats = []
    ms_prof = sum(timed_steps(args.steps, prof_stats))
    phase_ms, phase_n = native.mpm_get_phase_times(sim.ctx, reset=True)
    native.mpm_set_option(sim.ctx, native.OPT_PROFILE, 0)
    # solver statistics of the same steps as the phase times
    subs_p = max(sum(x.substeps for x in prof_stats), 1)
    iters_p = sum(x.iters_total for x in prof_stats)
    ls_p = sum(x.ls_evals_total for x in prof_stats)
    solve_us_p = [sum(x.solve_us[k] for x in prof_stats) / subs_p for k in range(5)]
    act_nodes = max(x.active_blocks_max for x in prof_stats) * 64

    out = {"value": value, "ms_per_step": ms / args.steps, "steps": args.steps,
           "p2g_form": {"chosen": ("gather", "scatter")[p2g_form], "particles_per_block": p2g_chunk,
                        "p2g_us_per_launch": {"%s_%d" % (("gather", "scatter")[f], c): 1e3 * t
                                              for (f, c), t in form_table}},
           "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                   "h2d_bytes_per_step": int(nb * C_sizeof_body(native)),
                   "d2h_bytes_per_step": int(12 * n + 48 * nb),
                   "device_ms_same_steps": same_steps_ms, "host_ms": 1e3 * e2e_s},
           "ms_per_step_profiled": ms_prof / args.steps,
           "phase_ms_per_step": {k: v / args.steps for k, v in phase_ms.items()},
           "solver": {"over": "the %d phase-timed steps" % len(prof_stats),
                      "iters_per_substep": iters_p / subs_p,
                      "ls_passes_per_iter": ls_p / max(iters_p, 1),
                      "contacts_max": max(x.contacts_max for x in prof_stats),
                      "residual_max": max(x.residual_max for x in prof_stats),
                      "active_blocks_max": max(x.active_blocks_max for x in prof_stats),
                      "status_bits": functools.reduce(lambda u, x: u | x.status_bits, prof_stats, 0),
                      "p2g_global_chunks": sum(x.p2g_global_chunks for x in prof_stats),
                      "status_timed": native.STATUS_NAMES[code_timed],
                      "solve_phases_us_per_substep": dict(zip(
                          ("node_list", "gradient_hessian", "node_solve", "line_search", "impulses"),
                          solve_us_p))},
           "launches_per_step": kernel_launches_per_step(sc["grid"]["res"], N, len(sc["bodies"]), n)}

    peak, peak_kind = measured_peak_hbm()
    kern = {}
    for name, per_p, per_node in (("p2g", P2G_BYTES_PER_PARTICLE, P2G_BYTES_PER_NODE),
                                  ("g2p", G2P_BYTES_PER_PARTICLE, 0)):
        launches = max(int(phase_n[name]), 1)
        avg_s = phase_ms[name] / launches / 1e3
        bytes_launch = per_p * n + per_node * act_nodes
        gbps = bytes_launch / avg_s / 1e9 if avg_s > 0 else 0.0
        kern[name] = {"avg_us": avg_s * 1e6, "launches": int(phase_n[name]),
                      "bytes_per_launch": bytes_launch, "GBps": gbps, "frac": gbps / peak}
    solve_launches = max(int(phase_n["solve"]), 1)
    solve_avg_s = phase_ms["solve"] / solve_launches / 1e3
    iters = out["solver"]["iters_per_substep"]
    # per QN iteration: 48 B per contact and 60 B per contact node (v, v*, m,
    # g, H, dv), the latter counted from the step's statistics
    solve_bytes = iters * (SOLVE_BYTES_PER_CONTACT * out["solver"]["contacts_max"] +
                           SOLVE_BYTES_PER_NODE * max(x.contact_nodes_max for x in prof_stats))
    kern["solve"] = {"avg_us": solve_avg_s * 1e6, "launches": int(phase_n["solve"]),
                     "us_per_qn_iter": solve_avg_s * 1e6 / max(iters, 1e-9),
                     "contacts": out["solver"]["contacts_max"],
                     "contact_nodes": max(x.contact_nodes_max for x in prof_stats),
                     "bytes_per_launch": solve_bytes,
                     "GBps": solve_bytes / solve_avg_s / 1e9 if solve_avg_s > 0 else 0.0,
                     "frac": (solve_bytes / solve_avg_s / 1e9 / peak) if solve_avg_s > 0 else 0.0,
                     "bound": "latency (device-wide or cluster barriers and L2 round trips "
                              "per QN iteration, not bytes)"}
    out["kernels"] = kern
    dom = max(("p2g", "g2p"), key=lambda k: phase_ms[k])
    wl = workload_name(sc)
    out["roofline"] = {"kernel": dom, "bound": "hbm", "achieved": kern[dom]["GBps"], "peak": peak,
                       "peak_kind": peak_kind, "unit": "GB/s", "frac": kern[dom]["GBps"] / peak,
                       "traffic": profiled_traffic(
                           dom if dom != "p2g" else "p2g_%s_%d" % (("gather", "scatter")[p2g_form], p2g_chunk),
                           wl, n),
                       "form": ("gather", "scatter")[p2g_form] if dom == "p2g" else None,
                       "note": "the streaming kernel with the largest share of the step; the "
                               "contact solve (%.0f%% of the step) is latency-bound, its "
                               "bytes in kernels.solve" % (100.0 * phase_ms["solve"] /
                                                          max(sum(phase_ms.values()), 1e-9))}

    # --- the same workload solved to the contact residual 1e-6 (one step)
    if tight:
        tsolver = native.solver_params(eps_r=1e-6, eps_a=0.0, max_iters=200000)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        code_t, st_t = native.mpm_step(sim.ctx, sc["h"], N, tsolver, want_stats=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_ms = ev0.elapsed_time(ev1)
        iters = st_t.iters_total / max(st_t.substeps, 1)
        out["tight_solve"] = {
            "eps_r": 1e-6, "value": float(n) * N / (t_ms / 1e3), "unit": UNIT, "ms_per_step": t_ms,
            "iters_per_substep": iters, "contacts_max": st_t.contacts_max,
            "ls_passes_per_iter": st_t.ls_evals_total / max(st_t.iters_total, 1),
            "solve_us_per_qn_iter": sum(st_t.solve_us[1:4]) / max(st_t.iters_total, 1),
            "residual_max": st_t.residual_max, "status": native.STATUS_NAMES[code_t], "steps": 1}
    out["state"] = sim.get_particles()
    out["bodies"] = sim.bodies()
    sim.close()
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2503_05046_gb300 import native
    sc = make_scene(WORKLOAD)
    n = sum(len(g["x"]) for g in sc["groups"])
    clocks = ClockSampler(local)
    clocks.start()
    head = measure_workload(native, sc, args, ws, tight=not args.no_small)
    clk = clocks.stop()
    sc2 = make_scene(SECONDARY)
    second = measure_workload(native, sc2, args, ws, tight=not args.no_small)
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(sc, n, ws),
        "e2e": head["e2e"],
        "gpu_launches": head["launches_per_step"] * args.steps,
        "roofline": head["roofline"],
    }
    for key in ("kernels", "phase_ms_per_step", "ms_per_step_profiled", "solver", "tight_solve", "p2g_form"):
        if key in head:
            line[key] = head[key]
    if clk:
        line["clocks"] = clk
    n2 = sum(len(g["x"]) for g in sc2["groups"])
    line["workloads"] = {SECONDARY: dict(
        {k: v for k, v in second.items() if k not in ("state", "bodies", "launches_per_step")},
        config=bench_config(sc2, n2, ws))}
    if not args.no_small:
        line["small_scenes"] = small_scene_latency(native)
        line["batched"] = batched_throughput(native, ws=ws, rank=rank)
        line["differentiation"] = differentiation(native)
        line["cloth"] = cloth_box_bagging(native)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline({WORKLOAD: (sc, head), SECONDARY: (sc2, second)})
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def small_scene_latency(native, n_steps=10):
    """Latency per substep of the 8,000-particle elastic cube (L2-resident and
    launch-bound, so reported as latency rather than a bandwidth fraction): the
    cube dropped from 0.2 m (free fall over the measured steps) and the same
    cube caught at touch-down on the ground (contacts every substep), the
    latter at the paper's tolerance and at 1e-6, with QN iterations per
    substep."""
    import torch
    from paper_2503_05046_gb300 import scenes
    out = {}
    cases = (("cube_drop_8k", scenes.cube_drop(), 5e-2),
             ("cube_contact_8k", scenes.cube_contact(n_side=20, v0=(0.0, 0.0, -0.05)), 5e-2),
             ("cube_contact_8k_tight", scenes.cube_contact(n_side=20, v0=(0.0, 0.0, -0.05)), 1e-6))
    for name, sc, eps in cases:
        sim = native.Sim(sc)
        solver = native.solver_params(eps_r=eps, max_iters=200000)
        N = sc["substeps"]
        sim.step(solver=solver, check=False)
        st0 = sim.get_particles()
        b0 = sim.bodies()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(sim.torch_stream)
        for _ in range(n_steps):
            native.mpm_step(sim.ctx, sc["h"], N, solver, want_stats=False)
        ev1.record(sim.torch_stream)
        torch.cuda.synchronize()
        us = 1e3 * ev0.elapsed_time(ev1) / (n_steps * N)
        # iteration counts from a repeat of the same steps with statistics
        sim.set_particles(st0["x"], st0["v"], st0["C"], st0["F"])
        sim.set_bodies(b0)
        iters, subs, contacts = 0, 0, 0
        for _ in range(n_steps):
            st = sim.step(solver=solver, check=False)[1]
            iters += st.iters_total
            subs += st.substeps
            contacts = max(contacts, st.contacts_max)
        out[name] = {"us_per_substep": us, "eps_r": eps, "iters_per_substep": iters / max(subs, 1),
                     "contacts_max": contacts, "particles": scenes.n_particles(sc)}
        sim.close()
    return out


def cloth_box_bagging(native, steps=40, warmup=3):
    """The cloth cradle of the box-bagging experiment (Sec. VI): a 30 x 30
    vertex sheet (900 particles) pinned at its corners with a dynamic 8 cm box
    on it, grid 1/64 m, 10 substeps of 2.5e-4 s per step at the paper's
    eps_r = 5e-2: particle-substeps/s, ms per step and the real-time rate,
    with the box moved on the device after each step. The paper's statistics
    table gives 45.3 ms per step of 10 substeps for 2,582 particles (vertices
    and face centroids of the same mesh) on an RTX 4090, its rigid and robot
    side included: context, not a like-for-like figure."""
    import torch
    from paper_2503_05046_gb300 import scenes
    from paper_2503_05046_gb300 import tune
    sc, dyn = scenes.box_bagging()
    solver = native.solver_params(eps_r=5e-2, max_iters=2000)
    N, h = sc["substeps"], sc["h"]
    # the P2G form, chosen on a copy of the scene so that the measured steps
    # start from the same state whichever form wins
    probe = native.Sim(sc)
    probe.set_dynamics(1, dyn)
    (form, chunk), _ = tune.tune_p2g_form(probe, solver, steps=2)
    probe.close()
    sim = native.Sim(sc)
    sim.set_dynamics(1, dyn)
    native.mpm_set_option(sim.ctx, native.OPT_P2G_FORM, form)
    native.mpm_set_option(sim.ctx, native.OPT_P2G_CHUNK, chunk)
    for _ in range(warmup):
        sim.step(solver=solver, check=False)
    st0 = sim.get_particles()
    b0 = sim.bodies()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(sim.torch_stream)
    for _ in range(steps):
        native.mpm_step(sim.ctx, h, N, solver, want_stats=False)
    ev1.record(sim.torch_stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    box_end = sim.bodies()[1]
    # contact and iteration counts from a repeat of the same steps
    sim.set_particles(st0["x"], st0["v"], st0["C"], st0["F"])
    sim.set_bodies(b0)
    sim.set_dynamics(1, dyn)
    iters, subs, contacts, failed = 0, 0, 0, 0
    for _ in range(steps):
        code, st = sim.step(solver=solver, check=False)
        iters += st.iters_total
        subs += st.substeps
        contacts = max(contacts, st.contacts_max)
        failed += int(code != native.OK)
    n = scenes.n_particles(sc)
    out = {"workload": sc["name"], "particles": n, "triangles": len(sc["groups"][0]["tris"]),
           "pins": 4, "substeps_per_step": N, "h_s": h, "steps": steps, "ms_per_step": ms,
           "us_per_substep": 1e3 * ms / N, "particle_substeps_per_s": n * N / (ms * 1e-3),
           "real_time_rate": N * h / (ms * 1e-3), "eps_r": 5e-2, "contacts_max": contacts,
           "iters_per_substep": iters / max(subs, 1), "steps_not_converged": failed,
           "p2g_form": ("gather", "scatter")[form],
           "box_drop_m": float(b0[1]["p"][2] - box_end["p"][2]),
           "paper": {"ms_per_step": 45.3, "particles": 2582, "substeps_per_step": 10,
                     "hardware": "RTX 4090, rigid and robot side included"}}
    sim.close()
    return out


def batched_throughput(native, n_scenes=256, steps=3, warmup=2, ws=1, rank=0):
    """Many independent scenes of uneven size (2k-64k particles each, elastic or
    sand, a gripper jaw and the ground) advanced three ways, each timed by the
    host clock around `steps` steps of every scene, synchronised on both sides:
    - `value`: one batch (mpm_batch_*): a substep of all scenes is one P2G, one
      compaction, one grid-update, one contact-solve and one G2P launch over
      (scene, block) work items, the time step one CUDA graph; launch options
      picked by tune.tune_batch_launch;
    - `concurrent_value`: one context per scene, each on its own stream
      replaying its own step graph, enqueued one after another without
      waiting, SM cap of the solve and P2G block size by tune.tune_batch;
    - `loop_value`: the single-scene path looped (one scene at a time, every
      step waited for, default options).
    On several GPUs the scenes are split round robin over the ranks (they
    are independent: no collective but the timing), each rank times its
    share and the values are all scenes over the slowest rank's time."""
    import torch
    from paper_2503_05046_gb300 import scenes, tune
    mine = shard(n_scenes, rank, ws)
    scs = [scenes.batch_scene(i) for i in mine]
    h, N = scs[0]["h"], scs[0]["substeps"]
    solver = native.solver_params(eps_r=5e-2, max_iters=1000)
    n_total = int(sum_over_ranks(sum(scenes.n_particles(sc) for sc in scs), ws))

    # (1) one batch
    batch = native.Batch(scs, max_contacts=lambda sc: 2 * scenes.n_particles(sc))
    best, table_b = tune.tune_batch_launch(batch, h, N, solver)
    for _ in range(warmup):
        batch.step(h, N, solver)
    batch.synchronize(stats=False)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(steps):
        batch.step(h, N, solver)
    torch.cuda.synchronize()
    t_persist = max_over_ranks(time.perf_counter() - t0, ws)
    code_b, codes_b, stats_b = batch.synchronize()
    contacts_b = [s["contacts_max"] for s in stats_b]
    batch.close()

    # (2) contexts side by side, (3) the loop
    sims = [native.Sim(sc, max_contacts=2 * scenes.n_particles(sc)) for sc in scs]
    (solve_cap, chunk), table = tune.tune_batch(sims, scs, solver)

    def run(cap, wait_each, p2g_chunk=256):
        for sim in sims:
            native.mpm_set_option(sim.ctx, native.OPT_SOLVE_BLOCKS, cap)
            native.mpm_set_option(sim.ctx, native.OPT_P2G_CHUNK, p2g_chunk)
        for _ in range(warmup):
            for sim, sc in zip(sims, scs):
                native.mpm_step(sim.ctx, sc["h"], sc["substeps"], solver, want_stats=False)
        torch.cuda.synchronize()
        for sim in sims:  # clear warm-up status (the touch-down substep may hit max_iters)
            native.mpm_synchronize(sim.ctx)
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(steps):
            for sim, sc in zip(sims, scs):
                native.mpm_step(sim.ctx, sc["h"], sc["substeps"], solver, want_stats=False)
                if wait_each:
                    sim.torch_stream.synchronize()
        torch.cuda.synchronize()
        return max_over_ranks(time.perf_counter() - t0, ws)

    t_conc = run(solve_cap, False, chunk)
    codes = [native.mpm_synchronize(sim.ctx) for sim in sims]
    t_loop = run(0, True)
    for sim in sims:
        sim.close()
    v_persist = n_scenes * steps / t_persist
    v_conc = n_scenes * steps / t_conc
    v_loop = n_scenes * steps / t_loop
    names = {native.BATCH_OPT_P2G_CHUNK: "p2g_chunk", native.BATCH_OPT_G2P_THREADS: "g2p_threads",
             native.BATCH_OPT_GRID_PARTICLES: "grid_particles_per_block",
             native.BATCH_OPT_SOLVE_BLOCKS: "solve_blocks_per_scene"}
    return {"scenes": n_scenes, "particles": n_total, "steps": steps, "substeps_per_step": N,
            "ranks": ws, "scenes_per_rank": len(mine),
            "value": v_persist, "unit": "scene-steps/s",
            "particle_substeps_per_s": n_total * N * steps / t_persist,
            "ms_per_step": 1e3 * t_persist / steps,
            "launches_per_step": 2 + 5 * N,
            "concurrent_value": v_conc, "loop_value": v_loop,
            "speedup_vs_concurrent": v_persist / v_conc, "speedup_vs_loop": v_persist / v_loop,
            "tuned": {names[k]: v for k, v in best.items()},
            "tuning_s_per_2_steps": [[{names[k]: v for k, v in c.items()}, round(t, 4)]
                                     for c, t in table_b],
            "contacts_per_scene": [int(min(contacts_b)), int(max(contacts_b))],
            "status": "ok" if code_b == 0 else
                      "%d scenes reported %s" % (int(np.sum(codes_b != 0)), sorted(set(codes_b.tolist()))),
            "concurrent_tuned": {"solve_cap": solve_cap, "p2g_chunk": chunk,
                                 "candidates_s_per_2_steps": [[c, k, round(t, 4)]
                                                              for c, k, t in table]},
            "status_concurrent": "ok" if all(c == 0 for c in codes) else
                                 "%d scenes reported %s" % (sum(c != 0 for c in codes), sorted(set(codes))),
            "timing": "host clock around the enqueue loop, synchronised on both sides"}


def differentiation(native, steps=20, eps_r=1e-4, fd=True):
    """The differentiation workload: a 65,536-particle elastic cube pushed by a
    kinematic box for 500 substeps (20 rigid steps of 25 substeps, one
    checkpoint per step), loss = squared distance of the centroid to a seeded
    target. Reports the forward rollout (plain, and recording the tape), the
    reverse pass (mpm_backward) and their ratio, the gradient with respect to
    E, nu, each body's mu and the (uniform) initial velocity, and two of
    them against central differences of the CUDA forward. The contact solve
    runs to eps_r = 1e-4 (the implicit gradient is exact at an exact
    minimiser; the block-diagonal quasi-Newton iteration needs ~500
    iterations per substep here for 1e-4 and ~3,000 for 1e-6). The
    difference steps are large enough (1e-2 of E, 1e-3 m/s) for the loss
    change to stand well above the FP32 forward's rounding and solve noise."""
    import torch
    from paper_2503_05046_gb300 import scenes
    sc, target = scenes.push_cube()
    n = scenes.n_particles(sc)
    solver = native.solver_params(eps_r=eps_r, max_iters=20000)
    N = sc["substeps"]

    def forward(sim, tape):
        if tape:
            sim.tape_begin()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            native.mpm_step(sim.ctx, sc["h"], N, solver, want_stats=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if tape:
            sim.tape_end()
        return dt

    def loss_of(sim):
        x = sim.get_particles()["x"].astype(np.float64)
        c = x.mean(0)
        return float(np.sum((c - target) ** 2)), c

    sim = native.Sim(sc)
    st0 = sim.get_particles()
    b0 = sim.bodies()

    def reset(s):
        s.set_particles(st0["x"], st0["v"], st0["C"], st0["F"])
        s.set_bodies(b0)

    forward(sim, False)  # warm-up (graph capture)
    reset(sim)
    t_plain = forward(sim, False)
    code_fwd = native.mpm_synchronize(sim.ctx)
    reset(sim)
    t_taped = forward(sim, True)
    native.mpm_synchronize(sim.ctx)  # (same status as the plain run, reported above)
    L, c = loss_of(sim)
    xbar = np.tile((2.0 * (c - target) / n).astype(np.float32), (n, 1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = sim.backward(x_bar=xbar, check=False)
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    sim.close()
    # central differences of the CUDA forward: E (h = 1e-2 E) and the x
    # component of the uniform initial velocity (h = 1e-3 m/s)
    E = float(sc["groups"][0]["material"]["E"])

    def loss_with(E_rel=0.0, dvx=0.0):
        sc2 = dict(sc)
        g2 = dict(sc["groups"][0])
        g2["material"] = dict(g2["material"], E=E * (1.0 + E_rel))
        g2["v"] = g2["v"] + np.float32([dvx, 0.0, 0.0])
        sc2["groups"] = [g2]
        s2 = native.Sim(sc2)
        forward(s2, False)
        out = loss_of(s2)[0]
        s2.close()
        return out

    tight = None
    if fd:
        # the workload itself, and its lattice variant at the same size (40^3
        # particles at 8 per cell, the outer layers 1e-5 m inside the ground
        # and the box): no particle sits near a contact threshold there
        sc_l, target_l = scenes.push_cube(lattice_side=40, sink=1e-5, box_overlap=1e-5)
        tight = {"random": differentiation_tight(native, sc, target),
                 "lattice": differentiation_tight(native, sc_l, target_l)}
    nan = float("nan")
    dE_fd = (loss_with(E_rel=1e-2) - loss_with(E_rel=-1e-2)) / (2e-2 * E) if fd else nan
    dv_fd = (loss_with(dvx=1e-3) - loss_with(dvx=-1e-3)) / 2e-3 if fd else nan
    dE_adj = float(g["E"][0])
    dv_adj = float(g["v"].astype(np.float64)[:, 0].sum())
    return {"workload": "push_cube_65536: elastic cube pushed by a kinematic box, 500 substeps "
                        "(20 steps x 25), checkpoint per step", "particles": n,
            "substeps": steps * N, "eps_r": eps_r, "loss": L,
            "fwd_s": t_plain, "fwd_taped_s": t_taped, "bwd_s": t_bwd,
            "bwd_over_fwd": t_bwd / t_plain,
            "grad": {"E": float(g["E"][0]), "nu": float(g["nu"][0]),
                     "mu": [float(m) for m in g["mu"]],
                     "v0": [float(v) for v in g["v"].astype(np.float64).sum(0)]},
            "central_differences": {
                "E": {"h": "1e-2 E", "fd": dE_fd, "adjoint": dE_adj,
                      "rel_diff": abs(dE_adj - dE_fd) / max(abs(dE_fd), 1e-300)},
                "v0_x": {"h": "1e-3 m/s", "fd": dv_fd, "adjoint": dv_adj,
                         "rel_diff": abs(dv_adj - dv_fd) / max(abs(dv_fd), 1e-300)}},
            "tight_check": tight,
            "status_fwd": native.STATUS_NAMES[code_fwd],
            "status_bwd": native.STATUS_NAMES[g["status"]],
            "timing": "host clock, synchronised on both sides"}


def differentiation_tight(native, sc, target, steps=2, eps_r=1e-6):
    """The differentiation workload shortened to `steps` rigid steps (50
    substeps) with the contact solve at eps_r = 1e-6 and the adjoint's CG at
    1e-8: dL/dE and dL/dv0_x from mpm_backward against central differences
    of the CUDA forward at two step sizes each (their agreement with each
    other bounds the truncation and noise of the differences). Two losses:
    the workload's own (squared distance of the centroid to the target) and
    the mean squared distance of each particle to its start position moved by
    1 cm along +x, which sees the cube's deformation: the centroid barely
    depends on E (a 1% change of E moves the centroid loss by ~2e-6 of itself,
    the size of the FP32 forward's run-to-run differences), the per-particle
    loss does. The scene keeps its k = 1e3 N/m per contact: its particles are
    ~8x lighter than the 8k cube's, and at 1e4 N/m the block-diagonal
    quasi-Newton iteration needs ~3,000 iterations per substep for 1e-6."""
    import torch
    from paper_2503_05046_gb300 import scenes
    n = scenes.n_particles(sc)
    N = sc["substeps"]
    solver = native.solver_params(eps_r=eps_r, eps_a=0.0, max_iters=200000)
    E = float(sc["groups"][0]["material"]["E"])

    x_goal = (np.asarray(sc["groups"][0]["x"], np.float64) +
              np.array([0.01, 0.0, 0.0]))  # per-particle loss target (id order)

    def losses(x):
        c = x.mean(0)
        return (float(np.sum((c - target) ** 2)),
                float(np.mean(np.sum((x - x_goal) ** 2, axis=1))), c)

    def rollout(scene, tape=False):
        s = native.Sim(scene)
        if tape:
            s.tape_begin()
        iters = 0
        for _ in range(steps):
            code, st = native.mpm_step(s.ctx, scene["h"], N, solver, want_stats=True)
            iters += st.iters_total
        if tape:
            s.tape_end()
        code = native.mpm_synchronize(s.ctx)
        x = s.get_particles()["x"].astype(np.float64)
        return s, x, code, iters

    def losses_with(E_rel=0.0, dvx=0.0):
        sc2 = dict(sc)
        g2 = dict(sc["groups"][0])
        g2["material"] = dict(g2["material"], E=E * (1.0 + E_rel))
        g2["v"] = g2["v"] + np.float32([dvx, 0.0, 0.0])
        sc2["groups"] = [g2]
        s2, x2, _, _ = rollout(sc2)
        s2.close()
        return losses(x2)[:2]

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim, x, code, iters = rollout(sc, tape=True)
    L_c, L_p, c = losses(x)
    bars = {"centroid": np.tile((2.0 * (c - target) / n).astype(np.float32), (n, 1)),
            "per_particle": (2.0 * (x - x_goal) / n).astype(np.float32)}
    adj = {}
    status_bwd = []
    for name, xbar in bars.items():
        g = sim.backward(x_bar=xbar, eps_r=1e-8, max_iters=20000, check=False)
        adj[name] = {"E": float(g["E"][0]), "v0_x": float(g["v"].astype(np.float64)[:, 0].sum())}
        status_bwd.append(native.STATUS_NAMES[g["status"]])
    sim.close()
    out = {"workload": "%s shortened to %d steps x %d substeps" % (sc["name"], steps, N),
           "eps_r": eps_r, "adjoint_cg_eps_r": 1e-8, "contact_k": sc["bodies"][0]["k"],
           "qn_iters_per_substep": iters / float(steps * N),
           "loss": {"centroid": L_c, "per_particle": L_p},
           "status_fwd": native.STATUS_NAMES[code], "status_bwd": status_bwd}
    for key, steps_h in (("E", (1e-2, 5e-3)), ("v0_x", (1e-3, 5e-4))):
        scale = E if key == "E" else 1.0
        rows = {"centroid": [], "per_particle": []}
        for h in steps_h:
            args_p = {"E_rel": h} if key == "E" else {"dvx": h}
            args_m = {"E_rel": -h} if key == "E" else {"dvx": -h}
            lp, lm = losses_with(**args_p), losses_with(**args_m)
            for i, name in enumerate(("centroid", "per_particle")):
                fd_val = (lp[i] - lm[i]) / (2.0 * h * scale)
                a = adj[name][key]
                rows[name].append({"h": h, "fd": fd_val,
                                   "rel_diff": abs(a - fd_val) / max(abs(fd_val), 1e-300)})
        out[key] = {name: {"adjoint": adj[name][key], "central_differences": rows[name]}
                    for name in rows}
    torch.cuda.synchronize()
    out["seconds"] = time.perf_counter() - t0
    return out


def C_sizeof_body(native):
    import ctypes
    return ctypes.sizeof(native.RigidBody)


def oracle_state(sc, state):
    """Oracle particle state (FP64) of a float32 particle state of the scene."""
    import oracle as O
    mass, vol, mat = [], [], []
    for gi, g in enumerate(sc["groups"]):
        k = len(g["x"])
        V = float(np.float32(g["vol"]))
        mass.append(np.full(k, V * float(np.float32(g["material"]["rho"]))))
        vol.append(np.full(k, V))
        mat.append(np.full(k, gi, np.int32))
    return O.Sim.state({"x": state["x"], "v": state["v"], "C": state["C"], "F": state["F"],
                        "mass": np.concatenate(mass), "vol": np.concatenate(vol),
                        "mat": np.concatenate(mat)})


def oracle_runner(sc, bodies=None, openmp=False, eps_r=5e-2):
    """advance(st, k): k oracle substeps of the whole scene on state st (the
    bodies frozen, as within one rigid step); returns the seconds taken."""
    import oracle as O
    _, mats = O.from_scene(sc)
    osim = O.Sim(sc["grid"], openmp=openmp)
    bds = [O.make_body(b) for b in O.bodies_from_scene({"bodies": bodies if bodies is not None
                                                         else sc["bodies"]})]
    S = O.solver(eps_r=eps_r, max_iters=1000)

    def advance(st, k):
        t0 = time.perf_counter()
        for _ in range(k):
            osim.substep(st, mats, bds, sc["h"], S)
        return time.perf_counter() - t0
    return advance


def host_info():
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name") or low.startswith("cpu part"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"host_cores": os.cpu_count(), "cpu": model, "machine": platform.machine()}


def oracle_available(openmp):
    try:
        import oracle as O
        O.lib(openmp)
        return True
    except Exception:
        return False


def cpu_baseline(measured):
    """The FP64 oracle on the machine's host cores, on bounded samples of each
    workload from the state the GPU run left (one substep of the 4M and 1M
    workloads), the 8,000-particle cube drop (cube_drop_8k) whole (200
    substeps) and one checkpoint interval (25 substeps) of the 65,536-particle
    differentiation workload: single-threaded (the oracle as written) and its
    OpenMP build over all host cores."""
    from paper_2503_05046_gb300 import scenes
    import oracle as O
    omp = oracle_available(True)
    builds = [(False, 1)] + ([(True, O.threads(True))] if omp else [])
    samples = []
    for name, (sc, res) in measured.items():
        samples.append((name, sc, res["state"], res["bodies"], 1))
    c1 = scenes.cube_drop()
    samples.append(("cube_drop_8k", c1, None, None, 200))
    c4, _ = scenes.push_cube()
    samples.append(("push_cube_65536", c4, None, None, 25))
    per = {}
    for name, sc, state, bodies, k in samples:
        n = sum(len(g["x"]) for g in sc["groups"])
        row = {"particles": n, "substeps": k}
        for openmp, threads in builds:
            if state is None:
                st, _ = O.from_scene(sc)
            else:
                st = oracle_state(sc, state)
            secs = oracle_runner(sc, bodies, openmp)(st, k)
            row["all_cores" if openmp else "single_thread"] = {
                "value": n * k / secs, "seconds": secs, "threads": threads}
        per[name] = row
    head = per[WORKLOAD]
    best = head.get("all_cores", head["single_thread"])
    out = {"value": best["value"], "unit": UNIT, "cores": best["threads"], "kind": "oracle",
           "sample": "FP64 oracle (%s) on one substep of all %d particles and %d bodies of %s "
                     "from the bench's state; %.1f s" % (
                         "OpenMP build, %d threads" % best["threads"] if "all_cores" in head
                         else "1 thread", head["particles"], len(measured[WORKLOAD][0]["bodies"]),
                         WORKLOAD, best["seconds"]),
           "single_thread": {"value": head["single_thread"]["value"], "cores": 1},
           "workloads": per}
    out.update(host_info())
    if not omp:
        out["all_cores"] = "unavailable: the OpenMP build of the oracle did not compile"
    return out


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores (its OpenMP build where
    it exists), one substep of the whole headline workload (all particles and
    bodies) per bench step."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    sc = make_scene()
    import oracle as O
    omp = oracle_available(True)
    st, _ = O.from_scene(sc)
    n = len(st["x"])
    advance = oracle_runner(sc, openmp=omp)
    advance(st, args.warmup)
    total_s = sum(advance(st, 1) for _ in range(args.steps))
    value = n * args.steps / total_s
    threads = O.threads(True) if omp else 1
    cfg = bench_config(sc, n, ws)
    cfg["sample"] = "one substep of the whole workload per bench step, after %d warm-up substeps" % args.warmup
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "config": cfg,
            "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                                  "sample": cfg["sample"] + ", FP64 oracle on %d host thread%s" % (
                                      threads, "s" if threads > 1 else "")}, **host_info()),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--max-iters", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the small-scene, batched, differentiation and tight-solve legs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
