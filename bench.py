"""Throughput of the ALE compressible lattice Boltzmann step on one GB300.

Headline workload (`value`): the batched airfoil sweep -- 32 NACA 00xx cases
(thickness 8-18%, 20k-300k P2 nodes each, log-uniform; 4,056,108 nodes in
all), Mach 0.1-0.8, rigid pitch 0-5 deg plus plunge 0-0.2c, k 0.05-1,
Re 1e4, chord 1000 lattice units, free-stream start -- advanced together by
the batched step (one launch per phase over all cases, replayed from CUDA
graphs), FP32 populations stored as deviations, FP64 map, departure points
and element decisions.  One step = propagation (departure points, element
location, P2 interpolation, wall/far-field missing populations), moments,
two FE-derivative passes and the collision, for every node of every case.
Cases at Mach >= 0.5 run on the lattice shifted by U = (0.3, 0) (Sec. V.D).

Metric: million node-updates per second.  The FP32 populations of the sweep
(585 MB, double-buffered) are larger than L2, so steps are timed back to
back with CUDA events on the batch's stream.  Beside it: the plain FP64
single-case form (the comparison the metric names) and the FP32 single
case on the 150,400-node plunge (L2 flushed before each of its steps), the
learned proposal on a 2M-node pitching mesh, storage-precision studies,
force histories, and the FP64 oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) the sweep's cases are shared out over the ranks by
node count, each rank steps its own with no exchange (weak scaling in
cases).
"""
import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2002_04353_gb300 import inputs as I  # noqa: E402

METRIC = "M node-updates/s on 1 GB300 (mixed/batched vs FP64 plain) + % HBM roofline"
UNIT = "M node-updates/s"
SHIFT03 = float(np.float32(0.3))  # the transonic case's lattice shift, rounded to FP32
FALLBACK_HBM_GBS = 6800.0


WORKLOADS = {
    # NACA 0012 plunging, Mach 0.2, Re 1e4, 150,400 P2 nodes (the headline case)
    "plunge150k": lambda: I.plunge_case(ni=320, nj=118),
    # the same flow on a 640 x 235 O-mesh, 600,320 P2 nodes (larger than L2;
    # used for counter captures)
    "plunge600k": lambda: I.plunge_case(ni=640, nj=235),
    # NACA 0012 pitching about c/4 on a blended deforming mesh, Mach 0.75,
    # 600,320 P2 nodes
    "pitch600k": lambda: I.pitch_case(ni=640, nj=235),
}


def workload(name="plunge150k"):
    return WORKLOADS[name]()


def kernel_bytes(kernel, n_nodes, n_elems, exact_items, pop_bytes=4, fld_bytes=4, fused=False):
    """Algorithmic bytes of one launch: every value the kernel must read or
    write, each counted once (FP32-deviation form: pop_bytes = fld_bytes = 4;
    16-bit forms: pop_bytes = 2, node fields still 4).

    k_stream_fast   per node: 18 post-collision populations read and (for the
                    settled ones, about all) 18 streamed written, 9 element-
                    cache words, the FP32 hi/lo coordinates (16 B), the
                    boundary distance and the zero-velocity flag (5 B); per
                    element the FP32 inverse Jacobian and edge vectors (32 B)
                    and the connectivity (24 B)
    k_stream_slow   per exact-path population: its work entry, node
                    coordinates, six post-collision values of f and of g,
                    two streamed values, its cache word, the element record
                    (FP32 frame 48 B, inverse Jacobian 32 B, connectivity
                    24 B): 4 + 16 + 12 pop + 2 pop + 4 + 104 B
    k_moments       per node: 18 streamed populations read, Q'_x, Q'_y,
                    mu/(rho T) written
    k_deriv1        per node: Q'_x, Q'_y, mu/(rho T) read (own values and the
                    owner element's, each once), the owner stencil (the
                    owner element's six node numbers, the element and the
                    local index: 32 B), node coordinates (16 B), D_x, D_y
                    written; per element the inverse Jacobian (16 B)
    k_collide       per node: 18 streamed populations read, D_x, D_y, owner
                    stencil, coordinates; 18 populations and rho, u, T
                    written; per element the same 16 B
    k_stream        (FP64 form) per node: 18 populations read and written,
                    Q', mu/(rho T) written, FP64 coordinates, fan entries;
                    per element frame, neighbours, edge info, rank,
                    connectivity (92 B)
    fused           the batched propagation fused with the moments: the
                    propagation also writes Q'_x, Q'_y, mu/(rho T) of its
                    nodes (counted for all N) and lists the pending nodes;
                    the moments kernel reads the list and does the pending
                    nodes only, counted as exact_items nodes (an upper bound:
                    a pending node has at least one listed population)
    """
    N, E, W, p, f = n_nodes, n_elems, exact_items, pop_bytes, fld_bytes
    if kernel == "k_stream_fast":
        return N * (36 * p + 36 + 16 + 5 + (3 * f if fused else 0)) + E * 56
    if kernel == "k_moments" and fused:
        return min(N, W) * (4 + 18 * p + 3 * f + 4)
    if kernel == "k_stream_slow":
        return W * (4 + 16 + 14 * p + 4 + 104)
    if kernel == "k_moments":
        return N * (18 * p + 3 * f)
    if kernel == "k_deriv1":
        return N * (3 * f + 32 + 16 + 2 * f) + E * 16
    if kernel == "k_collide":
        return N * (18 * p + 2 * f + 32 + 16 + 18 * p + 4 * f) + E * 16
    if kernel == "k_stream":
        return N * (36 * p + 3 * f + 16 + 3 * 8 + 4) + E * 92
    return 0


STEP_KERNELS = ("k_stream_fast", "k_stream_slow", "k_moments", "k_deriv1", "k_collide")
SWEEP_NAME = "batched_sweep_32_naca00xx_4.06M"


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# FP32-deviation kernels on the 150,400-node plunge workload, from one ncu
# capture of the current kernels; writes stay in L2 during these launches.
NCU_TRAFFIC_150K = {"k_stream_fast": 23.93e6, "k_stream_slow": 1.48e6, "k_moments": 10.84e6,
                    "k_deriv1": 9.02e6, "k_collide": 19.26e6}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, mean
# of 20 steady-state launches) of the batched phase kernels on the 32-case
# sweep, each launch over all cases as in the per-kernel pass that times
# them, from one ncu capture of the current kernels in the launch form
# named here (profiles/launch_list_sweep32.md); a run whose tuner picks
# another form reports no traffic.
NCU_TRAFFIC_SWEEP_FORM = {"k_stream_fast_directions_per_thread": 9, "k_stream_fast_fused_moments": True}
NCU_TRAFFIC_SWEEP = {"k_stream_fast": 962.6e6, "k_stream_slow": 42.9e6, "k_moments": 14.3e6,
                     "k_deriv1": 265.3e6, "k_collide": 838.0e6}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                d = json.load(f)
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    """The host CPU's model name and logical core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        import platform
        name = platform.processor() or platform.machine()
    return name, os.cpu_count()


def sweep_lattice(flow):
    """The sweep's run options: off-wall missing populations at the mesh
    velocity (flag OFFWALL_VG, the reading that keeps the plunging cases
    stable), and the lattice shifted by U = (0.3, 0) for cases at Mach >= 0.5
    (the paper's set-up for its transonic case)."""
    Ma = math.hypot(*flow.u_inf) / math.sqrt(flow.gamma * flow.T_inf)
    flow = dataclasses.replace(flow, flags=flow.flags | 256)  # ALELB_FLAG_OFFWALL_VG
    return dataclasses.replace(flow, shift=(SHIFT03, 0.0)) if Ma >= 0.5 else flow


def representative_cases(sweep):
    """The smallest, median and largest cases of the sweep by node count."""
    order = sorted(range(len(sweep)), key=lambda k: sweep[k].mesh.n_nodes)
    return [order[0], order[len(order) // 2], order[-1]]


def cpu_baseline(sweep, steps, threads):
    """The FP64 oracle as it stands on the sweep's representative cases
    (smallest, median, largest), `steps` steps each after one untimed step,
    its node loops on `threads` host threads: node-updates/s."""
    import oracle as O
    n0 = O.threads()
    used = O.threads(threads)
    work, dt = 0, 0.0
    try:
        for k in representative_cases(sweep):
            c = sweep[k]
            o = O.Oracle(c.mesh, c.motion, sweep_lattice(c.flow))
            o.step(1)
            for _ in range(steps):
                t0 = time.perf_counter()
                try:
                    o.step(1)
                    dt += time.perf_counter() - t0
                except O.OracleError:
                    # the impulsive start of the faster cases turns non-finite
                    # within these steps (as on the GPU): restart that case from
                    # the free stream, untimed, and go on
                    o = O.Oracle(c.mesh, c.motion, sweep_lattice(c.flow))
                    o.step(1)
                    continue
                work += c.mesh.n_nodes
            del o
    finally:
        O.threads(n0)
    return work / dt / 1e6, dt, used, work


def oracle_rate(case, steps, threads, flow=None):
    """The FP64 oracle on one case: `steps` steps after one untimed step, its
    node loops on `threads` host threads, node-updates/s (a state that turns
    non-finite restarts from the free stream, untimed)."""
    import oracle as O
    n0 = O.threads()
    used = O.threads(threads)
    fl = case.flow if flow is None else flow
    work, dt = 0, 0.0
    try:
        o = O.Oracle(case.mesh, case.motion, fl)
        o.step(1)
        for _ in range(steps):
            t0 = time.perf_counter()
            try:
                o.step(1)
                dt += time.perf_counter() - t0
            except O.OracleError:
                o = O.Oracle(case.mesh, case.motion, fl)
                o.step(1)
                continue
            work += case.mesh.n_nodes
        del o
    finally:
        O.threads(n0)
    return work / dt / 1e6, dt, used


def oracle_timing(threads):
    """The oracle on the paper-form configurations, all host threads: the
    deforming box (200 steps) and a 20-step window of the 150k plunge.  (Its
    set-up grows faster than linearly with the mesh -- 2.7 s at 150k nodes,
    21 s at 600k, 128 s at 2M on an 8-core host -- so the larger meshes are
    left out of the default run; the sweep's largest case, 281k nodes, is in
    the CPU baseline.)"""
    cases = {"box_9216_200_steps": (I.uniform_flow_case(), 200),
             "plunge_150400_20_steps": (I.plunge_case(ni=320, nj=118), 20)}
    out = {}
    for name, (case, steps) in cases.items():
        v, dt, used = oracle_rate(case, steps, threads)
        out[name] = {"value": v, "unit": UNIT, "seconds": dt, "threads": used}
    return out


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (all of them,
    OpenMP over nodes), on the sweep.  One reference step is one oracle step
    of the sweep's median case (80,028 nodes), a bounded sample of a sweep
    step that keeps --steps K --warmup W within a few minutes."""
    world, rank, local = dist_setup()
    if rank != 0:
        return
    import oracle as O
    sweep = I.batched_sweep()
    k = representative_cases(sweep)[1]
    c = sweep[k]
    threads = O.threads(os.cpu_count() or 1)
    o = O.Oracle(c.mesh, c.motion, sweep_lattice(c.flow))
    o.step(max(0, args.warmup))
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = c.mesh.n_nodes * args.steps / dt / 1e6
    model, ncpu = cpu_model()
    sample = (f"{args.steps} oracle steps of sweep case {k} ({c.mesh.n_nodes} nodes, the median case) after "
              f"{args.warmup} warm-up steps, plain FP64 C oracle, OpenMP over nodes on {threads} threads "
              f"({model}, {ncpu} logical cores)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": SWEEP_NAME, "nodes": sum(x.mesh.n_nodes for x in sweep), "cases": len(sweep),
                   "sample_case": k, "sample_nodes": c.mesh.n_nodes},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "cpu_model": model, "nproc": ncpu},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def method_bytes(n_nodes, n_elems):
    """The method's own bytes per step (FP32-deviation storage): every
    population read once and written once (2 x 18 x 4 B per node), the
    derivative passes' node fields (Q'_x, Q'_y, rho T written and read,
    D_x, D_y written and read, rho, u, T written: 56 B per node), the node's
    owner and home element (8 B), and per element the connectivity (24 B),
    neighbours (12 B) and FP64 vertices (48 B); rigid maps need no per-node
    map factors.  About 250 B per node-update on O-meshes (E = N/2)."""
    return n_nodes * (144 + 56 + 8) + n_elems * (24 + 12 + 48)


def run_batched(alelb, torch, dev, world, rank, args, sampler=None):
    """The 32-case airfoil sweep (NACA 00xx, 8-18% thick, 20k-300k P2 nodes
    log-uniform, Mach 0.1-0.8, pitch 0-5 deg, plunge 0-0.2c, k 0.05-1) in
    one batch: FP32-deviation solvers, one launch per phase over all cases,
    steps replayed from captured CUDA graphs.  Cases at Mach 0.5 and above
    run on the lattice shifted by U = (0.3, 0), the paper's set-up for its
    transonic case; on the plain lattice several of them leave the
    admissible range within the timed steps.  Under torchrun the cases are
    shared out by node count (shard.assign_cases) and every rank steps its
    own (no exchange: weak in cases).  Returns the timed result, the
    batched kernels' rooflines and the end-to-end figure (host-resident
    state through the C-ABI)."""
    from paper_2002_04353_gb300 import shard
    sweep = I.batched_sweep(scale=args.sweep_scale)
    mine = shard.assign_cases([c.mesh.n_nodes for c in sweep], world)[rank]
    cases = [sweep[k] for k in mine]
    meshes = [alelb.Mesh(c.mesh, c.motion) for c in cases]
    flows = [sweep_lattice(c.flow) for c in cases]
    solvers = [alelb.Solver(m, fl, alelb.PREC_FP32_DEV) for m, fl in zip(meshes, flows)]
    stream = torch.cuda.Stream(device=dev)
    b = alelb.Batch(solvers, stream=stream.cuda_stream)
    choice = b.tune(reps=3)
    groups = choice["case_groups"]
    if args.choice:  # a fixed launch form (counter captures of one form)
        forced = [int(v) for v in args.choice.split(",")]
        b.set_choice(forced)
        groups = 2 if forced[7] & 512 else 4 if forced[7] & 1024 else 1
        choice = dict(choice, forced=args.choice)
    b.step(max(3, args.warmup) - 1)
    b.sync()
    n_nodes = sum(c.mesh.n_nodes for c in cases)
    n_elems = sum(c.mesh.n_elems for c in cases)
    K = args.steps
    walks0 = sum(s.info()["walks"] for s in solvers)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    torch.cuda.nvtx.range_push("sweep_timed")  # (ncu --nvtx-include selects the timed launches by it)
    e0.record(stream)
    b.step(K)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    finite, nonfinite = 0, []
    for k, (s, fl) in zip(mine, zip(solvers, flows)):
        try:
            s.sync()
            finite += 1
        except alelb.AlelbError:
            nonfinite.append({"case": k, "mach": round(math.hypot(*fl.u_inf) / math.sqrt(fl.gamma * fl.T_inf), 3)})
    n_exact = (sum(s.info()["walks"] for s in solvers) - walks0) / K  # exact-path populations per step
    ms = shard.max_over_ranks(ms, torch, dev)
    n_total = int(shard.sum_over_ranks(n_nodes, torch, dev))
    # per-kernel device times of the batched phases, measured right after
    # the timed region with events around every launch (launched one by one)
    b.profile(True)
    b.step(20)
    kt = b.kernel_times()
    b.profile(False)
    # the persistent form (one cooperative launch per chunk of 64 steps,
    # grid-wide barriers between phases) over the same number of steps
    persistent = None
    if not args.no_persistent:
        b.set_mode(alelb.BATCH_PERSISTENT)
        b.step(3)
        torch.cuda.synchronize()
        e0.record(stream)
        b.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        msp = shard.max_over_ranks(e0.elapsed_time(e1), torch, dev)
        b.set_mode(alelb.BATCH_GRAPHS)
        persistent = {"value": n_total * K / (msp * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": msp / K, "steps": K,
                      "note": "same sweep and steps, one cooperative launch per 64-step chunk with grid-wide "
                              "barriers between phases"}
    kernels = {k: {"ms_per_launch": v[0] / max(1, v[1]), "launches": v[1]} for k, v in kt.items() if v[1]}
    rl = {}  # the phase kernels carry the single-case names (kb_fast runs as k_stream_fast, ...)
    fused = bool(choice.get("k_stream_fast_fused_moments"))
    same_form = all(choice.get(k) == v for k, v in NCU_TRAFFIC_SWEEP_FORM.items()) and args.sweep_scale == 1.0
    for k, v in kernels.items():
        alg = kernel_bytes(k, n_nodes, n_elems, n_exact, fused=fused)
        if alg:
            rl[k] = {"algorithmic_bytes": alg, "achieved_gbs": alg / (v["ms_per_launch"] * 1e-3) / 1e9,
                     "traffic": NCU_TRAFFIC_SWEEP.get(k) if same_form else None}
    b.close()
    for s in solvers:
        s.close()
    # end to end with host buffers: every step uploads every case's
    # populations from pinned host memory, advances the batch one step and
    # reads every case's populations back; a fresh batch from the
    # free-stream start.  The headline figure is alelb_batch_step_host (the
    # FP32-deviation form's stored deviations, exact, 72 B per node each way,
    # uploads, step and read-back pipelined by case group); beside it the
    # same exchange as three calls (alelb_batch_set_pops_stored, _step,
    # _get_pops_stored) and the FP64 exchange (alelb_batch_set_pops /
    # _get_pops: full FP64 values, 144 B).
    e2e = e2e_calls = e2e_fp64 = None
    if not args.no_e2e:
        Ke = args.e2e_steps

        def exchange_loop(dtype, mode):
            # a fresh batch per form, so that both run within the first steps
            # from the impulsive start, where every case stays finite
            solvers = [alelb.Solver(m, fl, alelb.PREC_FP32_DEV) for m, fl in zip(meshes, flows)]
            b = alelb.Batch(solvers, stream=stream.cuda_stream)
            b.tune(reps=1)
            get, put = (b.get_pops, b.set_pops) if mode == "fp64" else (b.get_pops_stored, b.set_pops_stored)
            hf = [torch.empty((9, c.mesh.n_nodes), dtype=dtype).pin_memory().numpy() for c in cases]
            hg = [torch.empty((9, c.mesh.n_nodes), dtype=dtype).pin_memory().numpy() for c in cases]
            get(hf, hg)
            t_now = np.array([s.time()[0] for s in solvers])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(Ke):
                if mode == "pipelined":
                    b.step_host(hf, hg, hf, hg, t=t_now + k)
                else:
                    put(hf, hg, t=t_now + k)
                    b.step(1)
                    get(hf, hg)
            dt = time.perf_counter() - t0
            b.close()
            for s in solvers:
                s.close()
            return dt

        dt = exchange_loop(torch.float32, "pipelined")
        bytes_step = 18 * 4 * n_nodes
        e2e = {"value": world * n_nodes * Ke / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": bytes_step,
               "d2h_bytes_per_step": bytes_step, "steps": Ke,
               "note": "host-resident state: per step one alelb_batch_step_host (every case's stored FP32 "
                       "deviations from and back to pinned host arrays, the copies and the step pipelined by "
                       "case group; fresh batch, free-stream start)"}
        dt = exchange_loop(torch.float32, "calls")
        e2e_calls = {"value": world * n_nodes * Ke / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": bytes_step,
                     "d2h_bytes_per_step": bytes_step, "steps": Ke,
                     "note": "the same as three calls: alelb_batch_set_pops_stored, alelb_batch_step(1), "
                             "alelb_batch_get_pops_stored"}
        dt = exchange_loop(torch.float64, "fp64")
        bytes_step = 18 * 8 * n_nodes
        e2e_fp64 = {"value": world * n_nodes * Ke / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": bytes_step,
                    "d2h_bytes_per_step": bytes_step, "steps": Ke,
                    "note": "the same with the FP64 exchange: alelb_batch_set_pops / alelb_batch_get_pops "
                            "(full FP64 populations)"}
    return {"value": n_total * K / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms / K, "steps": K,
            "cases": len(sweep) if world == 1 else f"{len(cases)} of {len(sweep)} on rank {rank}",
            "nodes": n_total, "elements": n_elems, "cases_finite_after_timing": finite,
            "cases_nonfinite_after_timing": nonfinite,
            "exact_path_per_step": n_exact,
            "cases_on_shifted_lattice": sum(1 for fl in flows if any(fl.shift)), "tuned_launch_shapes": choice,
            "kernels": kernels, "kernel_rooflines": rl, "method_bytes_per_step": method_bytes(n_nodes, n_elems),
            "persistent_form": persistent, "e2e": e2e, "e2e_three_calls": e2e_calls, "e2e_fp64_exchange": e2e_fp64,
            "clocks": clocks,
            # five phase kernels per step (propagation, exact path, moments, first derivative pass,
            # collision) in every case group
            "gpu_launches": 5 * K * groups}


def run_learned(alelb, torch, dev, args):
    """The learned departure-element proposal.  Training data: every query of
    the 600,320-node deforming pitching mesh (Mach 0.75, k = 0.08) at 10
    map times evenly spread over one pitch period (samples depend on the
    map only, not on the flow).  Deployment: the 1,999,200-node pitching
    mesh (1200 x 417 rings) at Mach 0.5, alpha = 2.5 deg sin(omega t),
    stepped with and without the network from the same start; the
    populations must come out bit-identical."""
    import math as _m
    c3 = I.pitch_case(ni=640, nj=235)
    s3 = alelb.Solver(alelb.Mesh(c3.mesh, c3.motion), c3.flow, alelb.PREC_FP32_DEV)
    om = float(c3.motion.params[2])
    period = 2.0 * _m.pi / om
    q = 9 * c3.mesh.n_nodes
    parts = []
    t0 = time.perf_counter()
    for k in range(10):
        feat = torch.empty((q, 6), dtype=torch.float32, device=dev)
        slot = torch.empty(q, dtype=torch.int16, device=dev)
        bary = torch.empty((q, 3), dtype=torch.float32, device=dev)
        nring = torch.empty(q, dtype=torch.uint8, device=dev)
        s3.samples(feat, slot, bary, nring, t=1.0 + k * period / 10.0)
        keep = slot >= 0
        parts.append((feat[keep], slot[keep], bary[keep], nring[keep]))
    s3.close()
    logged = 10 * q
    feat, slot, bary, nring = [torch.cat([p_[k] for p_ in parts]).contiguous() for k in range(4)]
    del parts
    log_s = time.perf_counter() - t0
    net = alelb.Mlp(seed=0)
    n = int(slot.shape[0])
    ps = torch.empty(n, dtype=torch.int32, device=dev)
    t0 = time.perf_counter()
    losses = net.train(feat, slot, bary, nring, epochs=args.mlp_epochs, batch=8192, lr=2e-3, w_bary=0.5, seed=1)
    train_s = time.perf_counter() - t0
    net.predict(feat, nring, ps)
    train_hit = (ps == slot.int()).float().mean().item()
    del feat, slot, bary, nring, ps
    c5 = I.pitch_case(ni=1200, nj=417, Ma=0.5, alpha0_deg=0.0)
    m5 = alelb.Mesh(c5.mesh, c5.motion)
    N = c5.mesh.n_nodes
    stream = torch.cuda.Stream(device=dev)
    res = {}
    pops = {}
    def one_step(s):
        """One step timed alone, with the proposal counters it moved."""
        a0 = s.mlp_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        with torch.cuda.stream(stream):
            s.lb_step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        s.sync()
        a1 = s.mlp_stats()
        d = {k: a1[k] - a0[k] for k in a1}
        return {"ms": e0.elapsed_time(e1), "exact_path": d["exact_path"], "proposed": d["proposed"],
                "accepted": d["accepted"], "hit_rate": d["accepted"] / max(1, d["proposed"])}

    for label, use in (("without", False), ("with", True)):
        s = alelb.Solver(m5, c5.flow, alelb.PREC_FP32_DEV, stream=stream.cuda_stream)
        if use:
            s.set_mlp(net)
        # the first step runs with an empty element cache: every population
        # takes the exact path, where a proposal can save the walk
        cold = one_step(s)
        s.lb_step(max(3, args.warmup) - 1)
        s.sync()
        st0 = s.mlp_stats()
        K = args.mlp_steps
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for k in range(K):
                evs[k][0].record(stream)
                s.lb_step(1)
                evs[k][1].record(stream)
        torch.cuda.synchronize()
        s.sync()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        st1 = s.mlp_stats()
        # a jump of the map time: the cached elements belong to another map
        t_now = s.time()[0]
        fj, gj = s.get_pops()
        s.set_pops(fj, gj, t=t_now + 2000.0)
        jump = one_step(s)
        s.profile(True)
        s.lb_step(3)
        kt = s.kernel_times()
        s.profile(False)
        exact = st1["exact_path"] - st0["exact_path"]
        prop = st1["proposed"] - st0["proposed"]
        acc = st1["accepted"] - st0["accepted"]
        res[label] = {"value": N * K / (ms * 1e-3) / 1e6, "ms_per_step": ms / K,
                      "exact_path_per_step": exact / K, "cold_cache_step": cold, "time_jump_step": jump,
                      "kernels": {k_: {"ms_per_launch": v[0] / max(1, v[1]), "launches": v[1]}
                                  for k_, v in kt.items() if v[1]}}
        if use:
            res[label].update({"proposals_per_step": prop / K, "hit_rate": acc / max(1, prop),
                               "fallback_rate": 1.0 - acc / max(1, exact)})
        pops[label] = s.get_pops()
        s.close()
    identical = bool(np.array_equal(pops["with"][0], pops["without"][0]) and
                     np.array_equal(pops["with"][1], pops["without"][1]))
    net.close()
    return {"unit": UNIT, "workload": f"pitch {N} nodes, Mach 0.5, alpha 2.5 deg sin(wt), k 0.08",
            "steps": args.mlp_steps, "without": res["without"], "with": res["with"],
            "gain": res["with"]["value"] / res["without"]["value"],
            "bit_identical_populations": identical,
            "training": {"samples_logged": logged, "samples_in_ring": n, "epochs": args.mlp_epochs,
                         "loss_per_epoch": [round(float(x), 4) for x in losses], "hit_rate_on_training_data": train_hit,
                         "log_seconds": log_s, "train_seconds": train_s,
                         "source": f"pitch mesh {c3.mesh.n_nodes} nodes, 10 map times over one period"}}


def run_precision(alelb, torch, dev, args, Ma, shift=(0.0, 0.0), flags=0):
    """Storage precision on the 600,320-node deforming pitching mesh
    (alpha = 0.1 + 2.5 deg sin(omega t), k = 0.08, Mach Ma, lattice shift
    `shift`, solver flags `flags`): the
    FP64, FP32-deviation, BF16-deviation and FP16-deviation forms advance
    the same free-stream start by the same steps.  Each deviation form
    reports its throughput over the last `--prec-steps` steps (L2 flushed
    before each) and the error of rho, u, T against the FP64 form (max and
    RMS over the nodes, normalised by rho_inf, |u_inf| and T_inf) twice:
    after 20 steps, where it is the storage rounding, and at the end, where
    the start transient next to the suction side has amplified it (every
    form, FP32 included, differs there from FP64 by far more than its
    rounding).  A form whose state leaves the admissible range is reported
    as diverged."""
    case = I.pitch_case(ni=640, nj=235, Ma=Ma)
    case = dataclasses.replace(case, flow=dataclasses.replace(case.flow, shift=shift, flags=flags))
    mesh = alelb.Mesh(case.mesh, case.motion)
    N, E = case.mesh.n_nodes, case.mesh.n_elems
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    W, K = max(20, args.warmup), args.prec_steps
    U = math.hypot(*case.flow.u_inf)
    out, ref, ref_early = {}, None, None

    def errors(mo, base):
        err = {}
        for k, sc in (("rho", case.flow.rho_inf), ("ux", U), ("uy", U), ("T", case.flow.T_inf)):
            d = (mo[k] - base[k]) / sc
            err[k] = {"max": float(np.abs(d).max()), "rms": float(np.sqrt(np.mean(d * d)))}
        return err

    forms = (("fp64", alelb.PREC_FP64, 8), ("fp32_dev", alelb.PREC_FP32_DEV, 4),
             ("bf16_dev", alelb.PREC_BF16_DEV, 2), ("fp16_dev", alelb.PREC_FP16_DEV, 2))
    for label, prec, pb in forms:
        s = alelb.Solver(mesh, case.flow, prec, stream=stream.cuda_stream)
        s.lb_step(W)
        try:
            s.sync()
        except alelb.AlelbError as e:
            out[label] = {"diverged": str(e), "within_steps": W}
            s.close()
            continue
        early = s.moments()
        walks0 = s.info()["walks"]
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for k in range(K):
                flush.fill_(float(k))
                evs[k][0].record(stream)
                s.lb_step(1)
                evs[k][1].record(stream)
        torch.cuda.synchronize()
        try:
            s.sync()
        except alelb.AlelbError as e:
            out[label] = {"diverged": str(e), "within_steps": W + K}
            s.close()
            continue
        ms = sum(a.elapsed_time(b) for a, b in evs)
        n_exact = (s.info()["walks"] - walks0) / K
        mo = s.moments()
        s.close()
        r = {"value": N * K / (ms * 1e-3) / 1e6, "ms_per_step": ms / K, "pop_bytes": pb}
        if prec != alelb.PREC_FP64:
            step_bytes = sum(kernel_bytes(k, N, E, n_exact, pop_bytes=pb) for k in STEP_KERNELS)
            r["algorithmic_bytes_per_step"] = step_bytes
            r["achieved_gbs"] = step_bytes / (ms / K * 1e-3) / 1e9
        if prec == alelb.PREC_FP64:
            ref, ref_early = mo, early
        elif ref is None:
            r["error_vs_fp64"] = None
        else:
            r[f"error_vs_fp64_step{W}"] = errors(early, ref_early)
            r[f"error_vs_fp64_step{W + K}"] = errors(mo, ref)
        out[label] = r
    walls = ("slip walls, equilibrium missing populations" if flags == (alelb.FLAG_SLIP_WALL | alelb.FLAG_BC_EQUILIBRIUM)
             else "the paper's wall condition" if flags == 0 else f"flags {flags}")
    return {"unit": UNIT, "workload": f"pitch600k: deforming O-mesh {N} nodes, Mach {Ma}, "
                                      f"alpha 0.1 + 2.5 deg sin(wt), k 0.08, lattice shift {shift}, {walls}",
            "steps": W + K, "timed_steps": K,
            "errors": f"normalised by rho_inf, |u_inf|, T_inf; max and RMS over nodes after {W} and {W + K} steps",
            **out}


def run_precision_growth(alelb, args):
    """How the flow amplifies rounding: on the 150,400-node plunge (paper's
    wall targets, and off-wall targets at the mesh velocity, R8c) and the
    600,320-node blended pitch at Mach 0.3, three runs from the same start
    -- FP64, FP64 with every f population changed in its last bit, and the
    FP32-deviation form -- compared at several step counts: the largest of
    the field errors (rho and T relative per node, u relative to the
    largest speed) of FP32 against FP64 and of the perturbed FP64 run
    against FP64.  When their ratio stays near the ratio of the formats'
    unit roundoffs, the FP32 difference is rounding amplified by the flow."""
    def field_err(mo, ref):
        umax = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
        return max(float((np.abs(mo["rho"] - ref["rho"]) / ref["rho"]).max()),
                   float(np.abs(mo["ux"] - ref["ux"]).max() / umax),
                   float(np.abs(mo["uy"] - ref["uy"]).max() / umax),
                   float((np.abs(mo["T"] - ref["T"]) / ref["T"]).max()))

    out = {}
    runs = (("plunge150k_paper", I.plunge_case(), 0, (20, 100, 200, 300, 500)),
            ("plunge150k_R8c", I.plunge_case(), alelb.FLAG_OFFWALL_VG, (20, 200, 1000, 2000)),
            ("pitch600k_ma03", I.pitch_case(Ma=0.3), 0, (20, 50, 100, 150, 220)))
    for name, case, flags, marks in runs:
        fl = dataclasses.replace(case.flow, flags=flags)
        m = alelb.Mesh(case.mesh, case.motion)
        sol = {k: alelb.Solver(m, fl, p) for k, p in (("fp64", alelb.PREC_FP64), ("fp64_perturbed", alelb.PREC_FP64),
                                                        ("fp32_dev", alelb.PREC_FP32_DEV))}
        for k, s in sol.items():
            f, g = s.get_pops()
            if k == "fp64_perturbed":
                f = f * (1.0 + np.random.default_rng(0).choice([-1.0, 1.0], size=f.shape) * 2.0 ** -52)
            s.set_pops(f, g, t=0.0)
        rows, done = [], 0
        for n in marks:
            try:
                for s in sol.values():
                    s.lb_step(n - done)
                mo = {k: s.moments() for k, s in sol.items()}
            except alelb.AlelbError as e:
                rows.append({"step": n, "diverged": str(e)})
                break
            done = n
            a, b = field_err(mo["fp32_dev"], mo["fp64"]), field_err(mo["fp64_perturbed"], mo["fp64"])
            rows.append({"step": n, "fp32_vs_fp64": a, "fp64_perturbed_vs_fp64": b, "ratio": a / max(b, 1e-300)})
        for s in sol.values():
            s.close()
        out[name] = rows
    return out


def run_force_history(alelb, args):
    """Lift and drag histories over whole runs on the 150,400-node plunging
    and pitching NACA 0012 (Sec. V.B, V.C), FP32 populations, off-wall missing populations at
    the mesh velocity (flag OFFWALL_VG, which keeps these runs stable):
    config 2 (h = 0.1c, k = 1, Ma 0.2, Re 1e4) over its 5 plunge periods, and
    the paper's slow (h = 0.08c, Sr = 0.46) and fast (h = 0.12c, Sr = 1.5)
    plunges at Ma 0.2, Re 1850 over 3 and 5 periods.  Sr = h omega / u_inf
    (Sec. V.B), so k = omega c / (2 u_inf) = Sr c / (2 h); the chord is 1000
    lattice units (the paper's is 200; Re, Ma, h/c and Sr are the paper's).
    The paper's two cases run without the correction phi (flag PHI_OFF; at
    Ma 0.2 and T 0.3 Q' carries the factor 1 - 3T = 0.1): with it their
    impulsive start, at plunge speeds 0.46 and 1.5 u_inf, diverges within
    200 steps.  c_D and c_L are sampled every 100 steps and reported per
    period (mean, range)."""
    out = {}
    V, P = alelb.FLAG_OFFWALL_VG, alelb.FLAG_PHI_OFF
    runs = (("config2_plunge", dict(Re=1e4, k=1.0, h_frac=0.1), 5.0, V),
            ("paper_slow_plunge", dict(Re=1850.0, k=0.46 / (2 * 0.08), h_frac=0.08), 3.0, V | P),
            ("paper_fast_plunge", dict(Re=1850.0, k=1.5 / (2 * 0.12), h_frac=0.12), 5.0, V | P))
    # the paper's pitching cases (Sec. V.C): rigid pitch about c/4, A = 2 deg,
    # Re 12000, k = omega c / (2 u_inf) = 6.68 and 10, at its Ma 0.2 (at its
    # Ma 0.08 the relaxation rate is 1.94 and these runs diverge)
    runs += (("paper_pitch_k6.68", dict(Re=12000.0, k=6.68, Ma=0.2, pitch=True), 3.0, V | P),
             ("paper_pitch_k10", dict(Re=12000.0, k=10.0, Ma=0.2, pitch=True), 3.0, V | P))
    for name, kw, periods, flags in runs:
        if kw.get("pitch"):
            case = I.pitch_case(ni=320, nj=118, Ma=kw["Ma"], Re=kw["Re"], k=kw["k"], alpha0_deg=0.0, amp_deg=2.0,
                                blended=False, periods=periods)
        else:
            case = I.plunge_case(ni=320, nj=118, Ma=0.2, periods=periods, **kw)
        fl = dataclasses.replace(case.flow, flags=flags)
        s = alelb.Solver(alelb.Mesh(case.mesh, case.motion), fl, alelb.PREC_FP32_DEV)
        T = 2.0 * math.pi / (2.0 * kw["k"] * fl.u_inf[0] / fl.chord)
        hist, done, status = [], 0, "completed"
        t0 = time.perf_counter()
        while done < case.steps:
            n = min(100, case.steps - done)
            s.lb_step(n)
            done += n
            try:
                F = s.forces()
            except alelb.AlelbError as e:
                status = f"diverged by step {done}: {e}"
                break
            hist.append((done, F[4], F[5]))
        wall = time.perf_counter() - t0
        s.close()
        h = np.array(hist).reshape(-1, 3)
        per = []
        for p in range(int(periods)):
            sel = (h[:, 0] > p * T) & (h[:, 0] <= (p + 1) * T)
            if sel.any():
                per.append({"cd_mean": float(h[sel, 1].mean()), "cl_mean": float(h[sel, 2].mean()),
                            "cd_range": [float(h[sel, 1].min()), float(h[sel, 1].max())],
                            "cl_range": [float(h[sel, 2].min()), float(h[sel, 2].max())]})
        out[name] = {"nodes": case.mesh.n_nodes, "steps": done, "period_steps": T, "status": status,
                     "wall_seconds": wall, "per_period": per,
                     "workload": (f"rigid pitch about c/4, A 2 deg, k {kw['k']:g}, Ma {kw['Ma']}, Re {kw['Re']:g}"
                                  if kw.get("pitch") else
                                  f"plunge h {kw['h_frac']}c, k {kw['k']:.4f}, Ma 0.2, Re {kw['Re']:g}"),
                     "flags": flags}
    return out


def run_sweep_seeds(alelb, torch, dev, args, seeds=(1, 2), steps=300):
    """The same sweep drawn with other seeds (case sizes, Mach numbers and
    motions differ): tuned, then `steps` graph-replayed steps timed with CUDA
    events, as the headline."""
    out = {}
    for seed in seeds:
        sweep = I.batched_sweep(seed=seed)
        solvers = [alelb.Solver(alelb.Mesh(c.mesh, c.motion), sweep_lattice(c.flow), alelb.PREC_FP32_DEV)
                   for c in sweep]
        stream = torch.cuda.Stream(device=dev)
        b = alelb.Batch(solvers, stream=stream.cuda_stream)
        choice = b.tune(reps=3)
        b.step(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        n = sum(c.mesh.n_nodes for c in sweep)
        out[f"seed{seed}"] = {"value": n / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms, "steps": steps,
                              "nodes": n, "fused_form": bool(choice.get("k_stream_fast_fused_moments")),
                              "directions_per_thread": choice.get("k_stream_fast_directions_per_thread")}
        b.close()
        for s_ in solvers:
            s_.close()
    return out


def run_element_stability(alelb, args):
    """How far the paper's airfoil runs get under its own wall targets (R8,
    correction phi on) on triangles and on the same rings as 9-node
    quadrilaterals (150,400 nodes each), FP32 populations, up to
    args.stability_steps steps with the forces read every 100 steps (a
    non-finite state stops the run): config 2's plunge, the paper's slow
    plunge (also with R8c) and its pitch at k = 6.68."""
    V = alelb.FLAG_OFFWALL_VG
    runs = (("config2_plunge", dict(Re=1e4, k=1.0, h_frac=0.1), 0),
            ("paper_slow_plunge", dict(Re=1850.0, k=0.46 / (2 * 0.08), h_frac=0.08), 0),
            ("paper_slow_plunge_R8c", dict(Re=1850.0, k=0.46 / (2 * 0.08), h_frac=0.08), V),
            ("paper_pitch_k6.68", dict(Re=12000.0, k=6.68, pitch=True), 0))
    out = {}
    for elem in ("p2", "q2"):
        for name, kw, flags in runs:
            if kw.get("pitch"):
                case = I.pitch_case(ni=320, nj=118, Ma=0.2, Re=kw["Re"], k=kw["k"], alpha0_deg=0.0, amp_deg=2.0,
                                    blended=False, elem=elem)
            else:
                case = I.plunge_case(ni=320, nj=118, Ma=0.2, elem=elem, **kw)
            fl = dataclasses.replace(case.flow, flags=flags)
            s = alelb.Solver(alelb.Mesh(case.mesh, case.motion), fl, alelb.PREC_FP32_DEV)
            done, status = 0, "completed"
            while done < args.stability_steps:
                s.lb_step(100)
                done += 100
                try:
                    s.forces()
                except alelb.AlelbError:
                    status = f"diverged by step {done}"
                    break
            s.close()
            out[f"{elem}:{name}"] = {"status": status, "steps": done, "nodes": case.mesh.n_nodes}
    return out


def run_bulk_stability(alelb, args):
    """Where the scheme itself stops being stable: a periodic box of 48 x 48
    cells with jittered P2 nodes and no walls, uniform flow at Ma 0.2 with
    every population perturbed by 1% (seeded), FP32 populations, 3,000
    steps per free-stream temperature and relaxation frequency omega (the
    viscosity set from omega); then the still 150k NACA 0012 at Re 1e4 and
    12000 (T 0.3, the paper's wall targets, phi on).  A non-finite state
    stops a run."""
    out = {}

    def run(s, steps, check):
        done = 0
        while done < steps:
            s.lb_step(100)
            done += 100
            try:
                check()
            except alelb.AlelbError:
                return {"status": f"diverged by step {done}", "steps": done}
        return {"status": "completed", "steps": done}

    m = alelb.Mesh(I.periodic_box(48, 96.0, 0.2, seed=1), I.Motion.make(I.MOTION_NONE))
    rng = np.random.default_rng(2)
    for T in (0.25, 0.3):
        for om in (1.8, 1.85, 1.9, 1.95):
            s = alelb.Solver(m, I.flow_params(0.2, T_inf=T, mu=(1.0 / om - 0.5) * T), alelb.PREC_FP32_DEV)
            f, g = s.get_pops()
            s.set_pops(f * (1 + 0.01 * rng.standard_normal(f.shape)), g * (1 + 0.01 * rng.standard_normal(g.shape)))
            out[f"box_T{T}_omega{om}"] = run(s, 3000, s.sync)
            s.close()
    m.close()
    m = alelb.Mesh(I.naca_omesh(320, 118, chord=1000.0, R=20000.0, first=1.0), I.Motion.make(I.MOTION_NONE))
    for Re in (1e4, 12000.0):
        flow = I.flow_params(0.2, T_inf=0.3, Re=Re, chord=1000.0)
        s = alelb.Solver(m, flow, alelb.PREC_FP32_DEV)
        r = run(s, 3000, s.forces)
        r["omega"] = round(1.0 / (flow.mu / (flow.rho_inf * flow.T_inf) + 0.5), 3)
        out[f"still_airfoil_Re{int(Re)}"] = r
        s.close()
    m.close()
    return out


def run_single(alelb, torch, dev, world, args):
    """The 150,400-node plunge (h = 0.1c, k = 1, Mach 0.2, Re 1e4): the
    FP32-deviation form and the plain FP64 form, one case.  Its working set
    fits in L2, so L2 is flushed (a 512 MiB write) before every timed step
    and only the step is timed.  Also the end-to-end figure of one case
    (host-resident state through the C-ABI)."""
    case = workload("plunge150k")
    mesh = alelb.Mesh(case.mesh, case.motion)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(prec, steps, warmup, profile):
        s = alelb.Solver(mesh, case.flow, prec, stream=stream.cuda_stream)
        s.lb_step(warmup)
        s.sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize()
        walks0 = s.info()["walks"]
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.fill_(float(k))
                evs[k][0].record(stream)
                s.lb_step(1)
                evs[k][1].record(stream)
        torch.cuda.synchronize()
        s.sync()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        info = s.info()
        info["walks_timed"] = info["walks"] - walks0
        kt = {}
        if profile:
            s.profile(True)
            with torch.cuda.stream(stream):
                for k in range(min(steps, 10)):
                    flush.fill_(float(k))
                    s.lb_step(1)
            torch.cuda.synchronize()
            kt = s.kernel_times()
            s.profile(False)
        s.close()
        return ms, kt, info

    W, K = max(3, args.warmup), args.single_steps
    ms32, kt32, info32 = timed(alelb.PREC_FP32_DEV, K, W, True)
    K64 = max(2, K // 4)
    ms64, kt64, _ = timed(alelb.PREC_FP64, K64, W, True)
    N, E = case.mesh.n_nodes, case.mesh.n_elems
    n_exact = info32["walks_timed"] / K
    per_kernel = {k: {"ms_per_launch": v[0] / v[1], "algorithmic_bytes": kernel_bytes(k, N, E, n_exact),
                      "achieved_gbs": kernel_bytes(k, N, E, n_exact) / (v[0] / v[1] * 1e-3) / 1e9}
                  for k, v in kt32.items() if v[1]}
    e2e = None
    if not args.no_e2e:
        # the stored FP32 deviations (exact, 72 B per node each way), then the
        # FP64 exchange (144 B) from the same solver
        s = alelb.Solver(mesh, case.flow, alelb.PREC_FP32_DEV, stream=stream.cuda_stream)
        Ke = max(3, K // 4)
        e2e = {}
        for name, dtype, get, put in (("stored", torch.float32, s.get_pops_stored, s.set_pops_stored),
                                      ("fp64", torch.float64, s.get_pops, s.set_pops)):
            f = torch.empty((9, N), dtype=dtype).pin_memory().numpy()
            g = torch.empty((9, N), dtype=dtype).pin_memory().numpy()
            get(f, g)
            t0 = time.perf_counter()
            for k in range(Ke):
                put(f, g, t=float(k))
                s.lb_step(1)
                get(f, g)
            dt = time.perf_counter() - t0
            nb = 18 * N * f.itemsize
            e2e[name] = {"value": world * N * Ke / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": nb,
                         "d2h_bytes_per_step": nb}
        s.close()
        e2e = dict(e2e["stored"], fp64_exchange=e2e["fp64"])
    return {
        "workload": case.name, "nodes": N, "elements": E,
        "fp32_dev": {"value": world * N * K / (ms32 * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms32 / K,
                     "steps": K, "kernels": per_kernel,
                     "step_algorithmic_gbs": sum(kernel_bytes(k, N, E, n_exact) for k in STEP_KERNELS)
                     / (ms32 / K * 1e-3) / 1e9,
                     "method_bytes_frac": method_bytes(N, E) / (ms32 / K * 1e-3) / 1e9 / measured_peaks()[0],
                     "walks_per_step": n_exact,
                     "verified_previous_element_rate": 1.0 - n_exact / (9.0 * N),
                     "traffic_ncu_per_launch": NCU_TRAFFIC_150K,
                     "l2": "flushed (512 MiB write) before every timed step; only the step is timed"},
        "fp64_plain": {"value": world * N * K64 / (ms64 * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms64 / K64,
                       "steps": K64,
                       "kernels": {k: {"ms_per_launch": v[0] / max(1, v[1])} for k, v in kt64.items() if v[1]}},
        "e2e": e2e,
    }


def run_q2(alelb, torch, dev, args):
    """The paper's own element: the 150,400-node plunging NACA 0012 O-mesh
    of 9-node quadrilaterals (the same rings as the triangle mesh, each cell
    kept whole), FP32-deviation and FP64 forms, L2 flushed before each
    timed step.  Every population takes the exact path (FP64 departure
    point, exact walk over quadrilaterals, Newton for Eq. NonLinear_Eq)."""
    case = I.plunge_case(elem="q2")
    mesh = alelb.Mesh(case.mesh, case.motion)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"workload": case.name, "nodes": case.mesh.n_nodes, "elements": case.mesh.n_elems}
    for label, prec in (("fp32_dev", alelb.PREC_FP32_DEV), ("fp64", alelb.PREC_FP64)):
        s = alelb.Solver(mesh, case.flow, prec, stream=stream.cuda_stream)
        s.lb_step(max(3, args.warmup))
        s.sync()
        K = args.q2_steps
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for k in range(K):
                flush.fill_(float(k))
                evs[k][0].record(stream)
                s.lb_step(1)
                evs[k][1].record(stream)
        torch.cuda.synchronize()
        s.sync()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        s.profile(True)
        with torch.cuda.stream(stream):
            s.lb_step(3)
        torch.cuda.synchronize()
        kt = s.kernel_times()
        s.profile(False)
        s.close()
        out[label] = {"value": case.mesh.n_nodes * K / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms / K,
                      "steps": K, "kernels": {k: {"ms_per_launch": v[0] / v[1]} for k, v in kt.items() if v[1]}}
    return out


def run_ours(args):
    import torch
    from paper_2002_04353_gb300 import alelb

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peak, peak_src = measured_peaks()
    W, K = max(3, args.warmup), args.steps
    if args.only_part:
        # one part alone (for counter captures of its kernels): no headline
        part = {"single": lambda: run_single(alelb, torch, dev, world, args),
                "q2": lambda: run_q2(alelb, torch, dev, args),
                "learned": lambda: run_learned(alelb, torch, dev, args)}[args.only_part]()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": UNIT, "part": args.only_part, "result": part}), flush=True)
        return

    # headline: the batched sweep, clocks sampled during its timed region
    sampler = ClockSampler(local)
    bat = run_batched(alelb, torch, dev, world, rank, args, sampler)
    ms_step = bat["ms_per_step"]
    top = max(bat["kernels"], key=lambda k: bat["kernels"][k]["ms_per_launch"])
    top_rl = bat["kernel_rooflines"].get(top, {})
    roofline = {"bound": "hbm", "kernel": top, "achieved": top_rl.get("achieved_gbs"), "peak": peak,
                "unit": "GB/s", "frac": (top_rl.get("achieved_gbs") or 0.0) / peak, "peak_source": peak_src,
                "traffic": top_rl.get("traffic"), "algorithmic_bytes_per_launch": top_rl.get("algorithmic_bytes"),
                "launch_ms": bat["kernels"][top]["ms_per_launch"],
                "note": ("achieved = algorithmic bytes of one launch over the sweep / its CUDA-event duration "
                         "(launched one by one right after the timed region); traffic = ncu dram bytes of one "
                         "launch on this workload")}
    mb = bat["method_bytes_per_step"]
    step_rl = {"method_bytes_per_step": mb, "method_bytes_per_node": mb / bat["nodes"],
               "achieved_gbs": mb / (ms_step * 1e-3) / 1e9, "frac": mb / (ms_step * 1e-3) / 1e9 / peak,
               "note": "the method's own bytes (populations once each way, derivative-pass fields, geometry)"}

    seeds = None if (args.only_batched or world > 1) else run_sweep_seeds(alelb, torch, dev, args)
    single = None if args.no_single else run_single(alelb, torch, dev, world, args)
    q2 = None if (args.no_q2 or world > 1) else run_q2(alelb, torch, dev, args)
    learned = None if (args.no_mlp or world > 1) else run_learned(alelb, torch, dev, args)
    forces = None if (args.no_forces or world > 1) else run_force_history(alelb, args)
    growth = None if (args.no_precision or world > 1) else run_precision_growth(alelb, args)
    stability = run_element_stability(alelb, args) if (args.stability and world == 1) else None
    bulk = run_bulk_stability(alelb, args) if (args.stability and world == 1) else None
    precision = precision_low = None
    if not (args.no_precision or world > 1):
        # config 3 at its own Mach number: the shifted lattice of the transonic
        # case and the inviscid-wall variant (equilibrium missing populations)
        precision = run_precision(alelb, torch, dev, args, args.prec_mach, (SHIFT03, 0.0),
                                  alelb.FLAG_SLIP_WALL | alelb.FLAG_BC_EQUILIBRIUM)
        # the paper's wall condition on the plain lattice, at a Mach number it holds
        precision_low = run_precision(alelb, torch, dev, args, 0.3)

    cpu = cpu1 = oracle_cfg = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sweep = I.batched_sweep()
        model, ncpu = cpu_model()
        reps = representative_cases(sweep)
        nodes = [sweep[k].mesh.n_nodes for k in reps]
        v, dt, used, work = cpu_baseline(sweep, args.cpu_steps, ncpu or 1)
        cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "cpu_model": model, "nproc": ncpu,
               "sample": f"{args.cpu_steps} steps each of the sweep's smallest, median and largest cases "
                         f"({nodes} nodes) after one untimed step, plain FP64 C oracle, OpenMP over nodes on "
                         f"{used} threads ({dt:.1f} s; {work} node-updates; a case whose state turns non-finite "
                         f"restarts from the free stream, untimed)"}
        v1, dt1, used1, _ = cpu_baseline(sweep, args.cpu_steps_1core, 1)
        cpu1 = {"value": v1, "unit": UNIT, "cores": used1, "kind": "oracle", "cpu_model": model,
                "sample": f"{args.cpu_steps_1core} steps each of the same three cases, one thread ({dt1:.1f} s)"}
        oracle_cfg = oracle_timing(ncpu or 1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": bat["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "precision": "FP32 populations (deviations) and arithmetic; FP64 map, "
                                         "departure points and element decisions",
            "data": "synthetic",
            "config": {"workload": SWEEP_NAME, "cases": 32, "nodes": bat["nodes"], "elements": bat["elements"],
                       "mach": "0.1-0.8 (cases >= 0.5 on the lattice shifted by (0.3, 0))", "re": 1e4,
                       "chord": 1000.0, "motion": "rigid pitch 0-5 deg + plunge 0-0.2c, k 0.05-1",
                       "l2": "inputs larger than L2 (FP32 populations of all cases 585 MB, double-buffered); "
                             "steps timed back to back",
                       "parallelism": f"cases sharded over {world} GPU(s)" if world > 1 else "single GPU"},
            "roofline": roofline,
            "step_roofline": step_rl,
            "batched": {k: v for k, v in bat.items() if k not in ("e2e", "clocks")},
            "batched_other_seeds": seeds,
            "fp64_plain": None if single is None else dict(single["fp64_plain"], workload=single["workload"]),
            "single_case": None if single is None else dict(single["fp32_dev"], workload=single["workload"],
                                                            e2e=single["e2e"]),
            "q2_single_case": q2,
            "gpu_launches": bat["gpu_launches"],
            "learned_proposal": learned,
            "precision_study": precision,
            "force_history": forces,
            "precision_study_ma03": precision_low,
            "precision_growth": growth,
            "element_stability": stability,
            "bulk_stability": bulk,
            "e2e": bat["e2e"],
            "cpu_baseline": cpu,
            "cpu_baseline_1core": cpu1,
            "oracle_timing": oracle_cfg,
            "clocks": bat["clocks"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000, help="timed steps of the batched sweep (the headline)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=64)
    ap.add_argument("--cpu-steps-1core", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--single-steps", type=int, default=40)
    ap.add_argument("--no-single", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-mlp", action="store_true")
    ap.add_argument("--mlp-epochs", type=int, default=2)
    ap.add_argument("--mlp-steps", type=int, default=10)
    ap.add_argument("--prec-steps", type=int, default=200)
    ap.add_argument("--prec-mach", type=float, default=0.75)
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-forces", action="store_true")
    ap.add_argument("--no-persistent", action="store_true")
    ap.add_argument("--no-q2", action="store_true")
    ap.add_argument("--q2-steps", type=int, default=10)
    ap.add_argument("--stability", action="store_true",
                    help="also run the paper's airfoil cases on triangles and quadrilaterals until they diverge")
    ap.add_argument("--stability-steps", type=int, default=3000)
    ap.add_argument("--sweep-scale", type=float, default=1.0,
                    help="node counts of the sweep's cases times this (1: the workload; smaller for counter captures)")
    ap.add_argument("--only-part", choices=["single", "q2", "learned"],
                    help="run one part alone, without the headline (for counter captures of its kernels)")
    ap.add_argument("--choice", default="",
                    help="after tuning, set the batch's launch shapes to these 8 values (alelb_batch_set_choice)")
    ap.add_argument("--only-batched", action="store_true",
                    help="the headline alone (no single case, e2e, network, precision, forces, CPU baseline)")
    args = ap.parse_args()
    if args.only_batched:
        args.no_single = args.no_e2e = args.no_mlp = args.no_precision = args.no_forces = args.no_q2 = True
        args.no_cpu_baseline = True
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
