"""Benchmark: node-updates per second per SSP-RK3 stage of the limited 2D Euler update.

Workload (N=1): 2D Euler, gamma = 1.4, 1024 x 1024 elements at p = 3 (16,777,216 nodes x 4
fields), blast data (rho = 1, v = 0, p = 1e-5 + 1e3 exp(-r^2/0.01^2) at the centre), outflow
sides, CFL 1/2, subcell convex limiting, mixed precision (float32 state and stage arithmetic,
float64 dt reduction).  The state (268 MB per buffer) is larger than L2, so no flush is needed.

One step = dt reduction + 3 SSP-RK3 stages (CUDA graph replay).  value = nodes * 3 * K / time.
Also reported: the same workload in float64 ("fp64"), the stage kernel's roofline, the same
workload on a curved (warped, periodic) mesh ("curved", Sec. 2.3 and 3.1), an end-to-end figure
through the C-ABI with host buffers, and the oracle's CPU rate.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank advances its own copy of the workload (independent problems: weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-updates/s per RK stage (Euler 2D p=3), mixed vs FP64; % HBM roofline"
UNIT = "node-updates/s"
# Counters of the two mixed-precision stage kernels (the library's tile autotuner picks one of
# them), from ncu captures of the 768x768 p=3 blast (stages 1-3 of one step): DRAM bytes (read +
# write) per node and launch averaged over the three stages, executed FP32 flops (2 x FFMA + FADD +
# FMUL) and warp instructions per node of stages 1, 2, 3.  "current" is False once the kernel has
# changed since its capture: its traffic is then reported as null.
STAGE_COUNTERS = {
    "node": {"kernel": "k_stage<3, TX, TY, LawEuler<float>, float, subcell>", "current": False,
             "dram_bytes_per_node": 39.3, "fp32_flop_per_node": (363.9, 371.9, 371.9),
             "warp_instr_per_node": (27.2, 27.2, 27.2)},
    # the line kernel issues paired float32 operations (fma/add/mul on register pairs), which the
    # thread-level FFMA/FADD/FMUL counters do not count: no FP32 flop figure; its FMA pipe was
    # active 36.5% of the cycles of stage 2 in the capture
    "line": {"kernel": "k_stage_lines<3, TX, TY, LawEuler<float>, float>", "current": True,
             "dram_bytes_per_node": 39.2, "fp32_flop_per_node": None,
             "warp_instr_per_node": (16.31, 16.30, 16.31)},
}
# The float64 stage kernel's executed FP64 flops per node (2 x DFMA + DADD + DMUL), stages 1-3,
# from an ncu capture of the same workload in float64: its FP64-pipe roofline.
FP64_STAGE_FLOP_PER_NODE = (1198.0, 1197.6, 1197.8)
SMS, SCHEDULERS_PER_SM = 152, 4
# DRAM traffic per node and launch (stages 1-3 averaged) of the two curved-mesh stage kernels, from
# ncu captures of the 768x768 curved leg; "current" is False once the kernel has changed since.
CURVED_COUNTERS = {
    "node": {"kernel": "k_stage_curved<3, LawEuler<float>, float>", "dram_bytes_per_node": 93.4, "current": False},
    "line": {"kernel": "k_stage_curved_lines<3, LawEuler<float>, float>", "dram_bytes_per_node": 93.9,
             "current": True},
}
NEL, P = 1024, 3
WORKLOAD = "2D Euler blast, 1024x1024 elements, p=3 (16.8M nodes x 4 fields), outflow, CFL 0.5, subcell convex limiting"
WORKLOAD_CURVED = ("2D Euler blast on a curved mesh: 1024x1024 elements, p=3, nodes warped by "
                   "x, y += 0.05 sin(2 pi x) sin(2 pi y), periodic, subcell convex limiting")
HBM_FALLBACK = 6800.0


def workload_label(nel):
    """The headline workload's description at nel x nel elements."""
    if nel == 1024:
        return WORKLOAD
    nodes = nel * nel * (P + 1) ** 2
    return WORKLOAD.replace("1024x1024", f"{nel}x{nel}").replace("16.8M nodes", f"{nodes / 1e6:.1f}M nodes")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu, self.rows, self.proc = gpu, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def blast_state(sv):
    from paper_2004_08503_gb300 import inputs
    x, y = sv.node_coords()
    return inputs.blast(x, y)


def make_solver(precision, stream):
    from paper_2004_08503_gb300 import sidp
    return sidp.Solver(stream=stream, law="euler", p=P, nx=NEL, ny=NEL, precision=precision,
                       domain=(0.0, 1.0, 0.0, 1.0), bc=("outflow",) * 4, cfl=0.5, gamma=1.4, limiter="subcell")


def max_over_ranks(torch, seconds, dist, device):
    """Slowest rank's time (the job's time); identity on one process."""
    if not dist:
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units processed by all ranks divided by the job's time (weak scaling: each rank its own copy)."""
    return units_per_rank * world / seconds


# untimed steps before the warm-up: the library's tile autotuner times its candidates at the first
# step and once more at step 10 (past the workload's initial transient)
SETTLE_STEPS = 10


def time_steps(torch, sv, stream, steps, warmup, dist=None, clocks_gpu=None):
    """Graph-replayed steps after SETTLE_STEPS untimed steps and `warmup` more; returns
    (max-over-ranks seconds, clock summary)."""
    sv.step(SETTLE_STEPS)
    sv.step(warmup)
    sv.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(clocks_gpu) if clocks_gpu is not None else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clk:
        clk.__enter__()
        time.sleep(0.3)
    ev0.record(stream)
    sv.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    if clk:
        clk.__exit__()
    sec = max_over_ranks(torch, ev0.elapsed_time(ev1) / 1e3, dist, "cuda")
    return sec, (clk.summary() if clk else None)


def other_ceilings(nodes, kt, clk, fp32_peak, ctr):
    """FP32 pipe (against the measured FMA throughput) and instruction-issue (nominal: 4
    schedulers per SM at the sampled SM clock) fractions of the stage kernel (counters `ctr`)."""
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz")
    if not mhz or not all(kt) or not ctr["current"]:
        return None
    hz = 1e6 * float(mhz)
    out = {"sm_mhz": float(mhz)}
    if ctr["fp32_flop_per_node"] is not None:
        fl = ctr["fp32_flop_per_node"]
        flops = sum(f * nodes for f in fl) / sum(kt)
        out["fp32"] = {"achieved": flops / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
                       "frac": flops / fp32_peak, "flop_per_node": list(fl),
                       "peak_kind": "measured (sidp_fma_peak, float32)"}
    if ctr["warp_instr_per_node"] is not None:
        wi = ctr["warp_instr_per_node"]
        issue = sum(w * nodes for w in wi) / sum(kt)
        issue_peak = SMS * SCHEDULERS_PER_SM * hz
        out["issue"] = {"achieved": issue / 1e12, "peak": issue_peak / 1e12, "unit": "T warp-instr/s",
                        "frac": issue / issue_peak, "warp_instr_per_node": list(wi),
                        "peak_kind": "nominal at the sampled clock"}
    return out


def stage_kernel_times(torch, sv, stream, reps):
    """Average device time of each stage-kernel launch (CUDA events on the launch stream)."""
    from paper_2004_08503_gb300 import sidp
    dt = sv.compute_dt()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    tot = [0.0, 0.0, 0.0]
    for _ in range(reps):
        evs[0].record(stream)
        for k in (1, 2, 3):
            sidp.sidp_stage(sv.ctx, k, dt)
            evs[k].record(stream)
        evs[3].synchronize()
        for k in (1, 2, 3):
            tot[k - 1] += evs[k - 1].elapsed_time(evs[k]) / 1e3
    return [t / reps for t in tot]


def run_curved(torch, sidp, stream, steps, warmup, hbm, peak_kind):
    """The same workload on a curved mesh (Sec. 2.3 metric terms, Sec. 3.1 corrected metric):
    the nodes of the Cartesian mesh moved by the periodic warp x += 0.05 s, y += 0.05 s,
    s = sin(2 pi x) sin(2 pi y) (inputs.warped_coords), periodic sides, mixed precision."""
    from paper_2004_08503_gb300 import inputs
    sv = sidp.Solver(stream=stream, law="euler", p=P, nx=NEL, ny=NEL, precision="mixed", domain=(0.0, 1.0, 0.0, 1.0),
                     bc=("periodic",) * 4, cfl=0.5, gamma=1.4, limiter="subcell")
    x, y = sv.node_coords()
    xw, yw = inputs.warped_coords(x, y, 0.05)
    t0 = time.time()
    sv.set_geometry(xw, yw)
    setup = time.time() - t0
    sv.set_state(inputs.blast(xw, yw))
    sv.set_stats(False)
    nodes = sv.N
    sec, _ = time_steps(torch, sv, stream, steps, warmup)
    value = nodes * 3 * steps / sec
    kt = stage_kernel_times(torch, sv, stream, reps=10)
    ctr = CURVED_COUNTERS["line" if sv.tile()[2] >= 4 else "node"]
    # untimed: three steps with the statistics variant of the curved stage kernel
    sv.set_stats(True)
    sv.step(3)
    d = sv.diag()
    sv.close()
    # algorithmic bytes per node and launch: state (u_in, u_out; u^n in stages 2-3) plus the
    # geometry each node reads: 8 metric rows and m_i, and the face normals on face nodes
    # (2 of every p+1 nodes along each direction carry a normal pair)
    s, n = 4, P + 1
    geo = s * (9 + 2 * (2.0 / n) * 2)
    per_node = [2 * 4 * s + geo, 3 * 4 * s + geo, 3 * 4 * s + geo]
    ach = sum(b * nodes for b in per_node) / sum(kt) / 1e9
    return {"workload": WORKLOAD_CURVED.replace("1024x1024", f"{NEL}x{NEL}"), "value": value, "unit": UNIT,
            "steps": steps, "ms_per_step": 1e3 * sec / steps, "stage_ms": [1e3 * t for t in kt],
            "geometry_setup_s": setup,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "traffic": ctr["dram_bytes_per_node"] * nodes if ctr["current"] else None,
                         "kernel": ctr["kernel"],
                         "bytes_per_node": per_node, "peak_kind": peak_kind},
            "invariants": {k: d[k] for k in ("rho_min", "p_min", "nonfinite", "max_bound_violation",
                                             "max_entropy_violation", "rootfind_max_iters", "rootfind_cap_hits",
                                             "bound_nudges")}}


def _oracle_strip(args):
    """One worker of cpu_baseline: the oracle's forward-Euler stage on a strip of element rows of
    the workload (its own blast data and outflow sides; every element of the strip is computed).
    Returns (nodes, seconds of the stage alone)."""
    nel, row0, rows, dt = args
    from oracle import laws, scheme
    from paper_2004_08503_gb300 import inputs
    h = 1.0 / nel
    pb = scheme.Problem(laws.Euler(1.4), P, nel, rows, domain=(0.0, 1.0, row0 * h, (row0 + rows) * h),
                        bc=("outflow",) * 4)
    X, Y = pb.node_coords()
    U = inputs.blast(X, Y)
    del X, Y
    t0 = time.perf_counter()
    pb.fe_stage(U, dt)
    return pb.Ne * (P + 1) ** 2, time.perf_counter() - t0


def cpu_baseline():
    """The oracle as it stands on all host cores: one forward-Euler stage of the whole workload,
    its element rows split into one strip per core (a process each, spawned; numpy runs one
    thread per process here).  Rate = all nodes / the slowest strip's time."""
    import multiprocessing as mp
    from oracle import laws, scheme
    from paper_2004_08503_gb300 import inputs
    cores = max(1, os.cpu_count() or 1)
    # the workload's time step: its largest wave speeds sit in the blast centre
    pb = scheme.Problem(laws.Euler(1.4), P, NEL, NEL, bc=("outflow",) * 4)
    c = NEL // 2
    centre = np.array([(c + dy) * NEL + c + dx for dy in range(-8, 8) for dx in range(-8, 8)])
    X, Y = pb.node_coords()
    U = inputs.blast(X, Y)
    del X, Y
    tot = pb.sum_dhat(U, centre)
    dt = pb.cfl * float(np.min(pb.mass[None, :] / (2.0 * tot)))
    del U, pb
    bounds = np.linspace(0, NEL, cores + 1).astype(int)
    jobs = [(NEL, int(a), int(b - a), dt) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_oracle_strip, jobs)
    nodes = sum(r[0] for r in res)
    sec = max(r[1] for r in res)
    return {"value": nodes / sec, "unit": UNIT, "cores": len(jobs), "kind": "oracle",
            "sample": f"one forward-Euler stage of the FP64 numpy oracle over the whole {NEL}x{NEL} p={P} blast "
                      f"({nodes} nodes), split into {len(jobs)} strips of element rows, one spawned process per "
                      f"host core (numpy single-threaded); rate = nodes / slowest strip's stage time "
                      f"({sec:.1f} s)"}


def run_reference(args):
    """The oracle arm: bounded samples of the same workload on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import laws, scheme
    from paper_2004_08503_gb300 import inputs
    pb = scheme.Problem(laws.Euler(1.4), P, NEL, NEL, bc=("outflow",) * 4)
    X, Y = pb.node_coords()
    U = inputs.blast(X, Y)
    del X, Y
    c = NEL // 2
    centre = np.array([(c + dy) * NEL + c + dx for dy in range(-8, 8) for dx in range(-8, 8)])
    rng = np.random.default_rng(1)
    sel = np.unique(np.concatenate([centre, rng.integers(0, pb.Ne, 256)]))
    tot = pb.sum_dhat(U, centre)
    dt = pb.cfl * float(np.min(pb.mass[None, :] / (2.0 * tot)))
    U0 = U[:, sel]

    def one_step():
        # one SSP-RK3 step on the sample (stage inputs restricted to the sample's elements)
        for k in (1, 2, 3):
            pb.fe_stage(U, dt, elems=sel)

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    sec = time.perf_counter() - t0
    nodes = len(sel) * (P + 1) ** 2
    value = nodes * 3 * args.steps / sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_elements": int(len(sel)), "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step = 3 forward-Euler stages of the FP64 numpy oracle on "
                                       f"{len(sel)} elements ({nodes} nodes) of the workload, single thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_e2e(torch, sidp, sv, U, stream, args, dist, world, nodes):
    """The same metric through the C-ABI with host buffers: every step uploads the state from
    pinned host memory, runs one SSP-RK3 step and downloads the new state."""
    host_in = torch.from_numpy(U.astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    sv.set_stats(False)
    e_steps = max(3, min(args.steps, 30))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sidp.sidp_upload_state(sv.ctx, host_in.data_ptr())
    sv.step(1)
    sv.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(e_steps):
        sidp.sidp_upload_state(sv.ctx, host_in.data_ptr())
        sv.step(1)
        sidp.sidp_download_state(sv.ctx, 0, host_out.data_ptr())
    ev1.record(stream)
    ev1.synchronize()
    e_sec = max_over_ranks(torch, ev0.elapsed_time(ev1) / 1e3, dist, "cuda")
    return {"value": whole_job_rate(nodes * 3 * e_steps, world, e_sec), "unit": UNIT,
            "h2d_bytes_per_step": int(host_in.numel() * 4), "d2h_bytes_per_step": int(host_out.numel() * 4),
            "steps": e_steps}


def _batch_rate(torch, sidp, stream, cfgs, states, steps, warmup):
    """Create a batch, set the states (a function of (batch, i) or a list), time `steps` steps."""
    b = sidp.sidp_batch_create(cfgs, stream)
    for i in range(len(cfgs)):
        sidp.sidp_batch_set_state(b, i, states(b, i) if callable(states) else states[i])
    sidp.sidp_batch_set_stats(b, False)
    nodes = sidp.sidp_batch_total_nodes(b)
    sidp.sidp_batch_step(b, warmup)
    sidp.sidp_batch_synchronize(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sidp.sidp_batch_step(b, steps)
    e1.record(stream)
    e1.synchronize()
    return b, nodes, e0.elapsed_time(e1) / 1e3


def run_batched(torch, sidp, stream, steps, warmup, hbm, peak_kind, seed=0, count=512):
    """Batched workload: `count` independent Euler problems, elements per side from {8,16,32,64}
    and p from {2..7} (seeded), seeded four-quadrant data, mixed precision, outflow sides.  The
    default launch structure (one launch per degree group, the groups on concurrent graph
    branches) is timed, and beside it the single degree-switching launch per stage."""
    from paper_2004_08503_gb300 import inputs
    shapes = inputs.batch_shapes(seed, count)
    cfgs = [sidp.make_config(law="euler", p=p, nx=nel, ny=nel, precision="mixed", bc=("outflow",) * 4)
            for nel, p in shapes]
    states = []

    def initial(b, i):
        x, y = sidp.sidp_batch_node_coords(b, i)
        states.append(inputs.four_quadrant(x, y, seed * 100003 + i))
        return states[-1]

    prev = os.environ.pop("SIDP_BATCH_LAUNCH", None)
    b, nodes, sec = _batch_rate(torch, sidp, stream, cfgs, initial, steps, warmup)
    sidp.sidp_batch_set_stats(b, True)
    sidp.sidp_batch_step(b, 2)
    worst = {"rho_min": 1e300, "p_min": 1e300, "max_bound_violation": 0.0, "max_entropy_violation": 0.0}
    for i in range(0, count, max(1, count // 32)):
        d = sidp.sidp_batch_get_diag(b, i)
        worst["rho_min"] = min(worst["rho_min"], d["rho_min"])
        worst["p_min"] = min(worst["p_min"], d["p_min"])
        worst["max_bound_violation"] = max(worst["max_bound_violation"], d["max_bound_violation"])
        worst["max_entropy_violation"] = max(worst["max_entropy_violation"], d["max_entropy_violation"])
    sidp.sidp_batch_destroy(b)
    os.environ["SIDP_BATCH_LAUNCH"] = "single"
    bs, _, sec_single = _batch_rate(torch, sidp, stream, cfgs, states, steps, warmup)
    sidp.sidp_batch_destroy(bs)
    os.environ.pop("SIDP_BATCH_LAUNCH")
    if prev is not None:
        os.environ["SIDP_BATCH_LAUNCH"] = prev
    # whole step on 3 nc s = 48 bytes per node and stage (state passes of the three stages and the
    # time step, Euler float32)
    gbs = 48.0 * nodes * 3 * steps / sec / 1e9
    return {"value": nodes * 3 * steps / sec, "unit": UNIT, "instances": count, "nodes": nodes, "steps": steps,
            "ms_per_step": 1e3 * sec / steps, "launches_per_step": "4 per degree group + 1",
            "single_launch": {"value": nodes * 3 * steps / sec_single, "unit": UNIT,
                              "ms_per_step": 1e3 * sec_single / steps, "launches_per_step": 5,
                              "note": "one degree-switching launch per stage (SIDP_BATCH_LAUNCH=single)"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "bytes_per_node_stage": 48, "scope": "whole graph-replayed step", "peak_kind": peak_kind},
            "invariants_sampled": worst, "workload": f"{count} Euler instances, elements per side in {{8,16,32,64}}, "
            f"p in {{2..7}} (seed {seed}), four-quadrant data, mixed precision, one CUDA graph per step, degree groups on concurrent graph branches"}


def run_dmr(sidp, nx, t_end, image=None, chunk=100, max_seconds=600.0, stats_from=0.0):
    """The double Mach reflection of Sec. 5.7 on nx x nx/4 elements of [0,4] x [0,1], p = 3, mixed
    precision, to t_end (the paper runs 2400 x 600 to t = 0.275).  Split boundaries: post-shock
    inflow (west), post-shock then slip wall from x = 1/6 (south), the moving incident shock
    (north), outflow (east).  Reports throughput, invariants and where the incident shock meets the
    top boundary against its exact position; `image`: element-mean density as a binary PGM."""
    import time
    from paper_2004_08503_gb300 import inputs
    ny = nx // 4
    sv = sidp.Solver(law="euler", p=3, nx=nx, ny=ny, precision="mixed", domain=(0.0, 4.0, 0.0, 1.0),
                     bc=("split", "outflow", "split", "split"))
    for side, sp in inputs.double_mach_boundaries().items():
        sv.set_split(side, sp["s0"], sp["speed"], sp["a"], sp["b"])
    x, y = sv.node_coords()
    sv.set_state(inputs.double_mach(x, y))
    # statistics (bound and entropy violations) over t >= stats_from * t_end (0: the whole run)
    sv.set_stats(stats_from <= 0.0)
    steps, t = 0, 0.0
    sv.synchronize()
    t0 = time.perf_counter()
    stop = "t_end reached"
    while t < t_end:
        sv.step(chunk)
        steps += chunk
        d = sv.diag()
        if d["nonfinite"] or not d["t"] > t:
            stop = "stopped: non-finite state or time not advancing"
            t = d["t"]
            break
        t = d["t"]
        if stats_from > 0.0 and t >= stats_from * t_end:
            sv.set_stats(True)
        if steps % (50 * chunk) == 0:
            print(f"dmr: {steps} steps, t = {t:.5f}, {time.perf_counter() - t0:.1f} s", file=sys.stderr, flush=True)
        if time.perf_counter() - t0 > max_seconds:
            stop = f"stopped at the {max_seconds:.0f} s wall-clock cap"
            break
    sec = time.perf_counter() - t0
    d = sv.diag()
    u = sv.get_state(0)
    top = np.abs(y - 1.0) < 1e-12
    order = np.argsort(x[top])
    xs, rs = x[top][order], u[0][top][order]
    cross = float(xs[np.argmax(rs < 0.5 * (inputs.DMR_PRE[0] + inputs.DMR_POST[0]))])
    if image:
        rho = u[0].reshape(ny, nx, 16).mean(axis=2)[::-1]
        lo_, hi_ = float(rho.min()), float(rho.max())
        g = np.clip((rho - lo_) / max(hi_ - lo_, 1e-30) * 255.0, 0, 255).astype(np.uint8)
        with open(image, "wb") as f:
            f.write(b"P5\n%d %d\n255\n" % (nx, ny))
            f.write(g.tobytes())
    out = {"elements": [nx, ny], "p": 3, "nodes": sv.N, "t": t, "steps": steps, "seconds": sec,
           "value": sv.N * 3 * steps / sec, "unit": UNIT, "rho_min": d["rho_min"], "p_min": d["p_min"],
           "rho_max": float(u[0].max()), "max_bound_violation": d["max_bound_violation"],
           "max_entropy_violation": d["max_entropy_violation"], "rootfind_cap_hits": d["rootfind_cap_hits"],
           "nonfinite": d["nonfinite"], "top_shock_x": cross, "top_shock_x_exact": float(inputs.dmr_shock_x(1.0, t)),
           "element_width": 4.0 / nx, "end": stop, "statistics_from_t": stats_from * t_end,
           "timing": "wall clock around sidp_step and diag calls (every %d steps)" % chunk}
    sv.close()
    return out


def run_accuracy(sidp, stream, stages=198):
    """Mixed (float32) against float64 after `stages` RK stages on the two mixed-precision
    configurations (256x256 p=3 and 128x128 p=7, seeded four-quadrant data, outflow), with the
    violation statistics of the mixed run (density bounds and entropy minimum, measured in float64
    on the stored state, over every stage).  The float64 path is the one the parity tests hold to
    the FP64 oracle (including a sampled check of this float64 trajectory's final state)."""
    from paper_2004_08503_gb300 import inputs
    out = []
    for nel, p in ((256, 3), (128, 7)):
        res = {}
        for prec in ("fp64", "mixed"):
            sv = sidp.Solver(stream=stream, law="euler", p=p, nx=nel, ny=nel, precision=prec, bc=("outflow",) * 4)
            x, y = sv.node_coords()
            sv.set_state(inputs.four_quadrant(x, y, 0))
            sv.set_stats(True)
            sv.step(stages // 3)
            res[prec] = (sv.get_state(0), sv.diag())
            sv.close()
        a, b = res["mixed"][0], res["fp64"][0]
        w = np.abs(b).max(axis=1)
        d = res["mixed"][1]
        node_stages = a.shape[1] * 3 * (stages // 3)
        out.append({"config": f"{nel}x{nel} p={p}", "stages": 3 * (stages // 3),
                    "linf_rel": (np.abs(a - b).max(axis=1) / w).tolist(),
                    "l1_rel": (np.abs(a - b).mean(axis=1) / np.abs(b).mean(axis=1)).tolist(),
                    "rho_min": d["rho_min"], "p_min": d["p_min"], "max_bound_violation": d["max_bound_violation"],
                    "max_entropy_violation": d["max_entropy_violation"],
                    "bound_nudges": d["bound_nudges"], "bound_nudge_share": d["bound_nudges"] / node_stages,
                    "rootfind_cap_hits": d["rootfind_cap_hits"], "fp64_rootfind_cap_hits": res["fp64"][1]["rootfind_cap_hits"]})
    return out


def main():
    global NEL
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64 leg (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--nel", type=int, default=NEL, help="elements per side (profiling runs only)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched leg")
    ap.add_argument("--no-curved", action="store_true", help="skip the curved-mesh leg")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the mixed-vs-float64 accuracy leg")
    ap.add_argument("--dmr", type=int, default=0, help="also run the double Mach reflection on N x N/4 elements")
    ap.add_argument("--dmr-t", type=float, default=0.275, help="final time of the double Mach reflection")
    ap.add_argument("--dmr-image", default=None, help="write its element-mean density as a PGM file")
    ap.add_argument("--dmr-max-seconds", type=float, default=600.0, help="wall-clock cap of the double Mach run")
    ap.add_argument("--dmr-stats-from", type=float, default=0.0,
                    help="collect violation statistics only from this fraction of the final time on")
    args = ap.parse_args()
    NEL = args.nel
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2004_08503_gb300 import build, sidp
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    sidp.load()
    stream = torch.cuda.Stream()
    hbm, peak_kind = peaks()
    fp32_peak = sidp.sidp_fma_peak("mixed", stream)
    fp64_peak = sidp.sidp_fma_peak("fp64", stream)

    # ---------------- mixed precision: the headline
    sv = make_solver("mixed", stream)
    U = blast_state(sv)
    sv.set_state(U)
    sv.set_stats(False)
    nodes = sv.N
    sec, clk = time_steps(torch, sv, stream, args.steps, args.warmup, dist, clocks_gpu=local)
    value = whole_job_rate(nodes * 3 * args.steps, world, sec)
    # stage-kernel roofline: algorithmic bytes per launch = reads of u_in (and u^n in stages 2, 3)
    # plus the write of u_out, nc = 4 fields of s = 4 bytes per node
    kt = stage_kernel_times(torch, sv, stream, reps=20)
    s = 4
    bytes_stage = [2 * 4 * s * nodes, 3 * 4 * s * nodes, 3 * 4 * s * nodes]
    # the stage kernel the autotuner chose, and its DRAM traffic per launch (average over stages
    # 1-3) from one ncu capture of the 768x768 case scaled to this launch by nodes
    tx, ty, tidx = sv.tile()
    ctr = STAGE_COUNTERS["line" if tidx >= 4 else "node"]
    kname = ctr["kernel"].replace("TX", str(tx)).replace("TY", str(ty))
    traffic = ctr["dram_bytes_per_node"] * nodes if (ctr["current"] and ctr["dram_bytes_per_node"]) else None
    ach = sum(bytes_stage) / sum(kt) / 1e9
    # whole step on the per-node figure 3 * nc * s bytes per node per stage (dt pass included)
    step_gbs = 3 * 4 * s * nodes * 3 * args.steps / sec / 1e9
    # invariants of the workload (statistics on, a separate short run)
    sv.set_state(U)
    sv.set_stats(True)
    sv.step(3)
    d = sv.diag()
    diag_stats = {k: d[k] for k in ("rho_min", "p_min", "max_bound_violation", "max_entropy_violation",
                                   "rootfind_max_iters", "rootfind_cap_hits", "nonfinite")}
    e2e = None if args.no_e2e else run_e2e(torch, sidp, sv, U, stream, args, dist, world, nodes)
    sv.close()

    # ---------------- the plain FP64 single-instance form on the same GPU
    fp64 = None
    if not args.no_fp64:
        sv64 = make_solver("fp64", stream)
        sv64.set_state(U)
        sv64.set_stats(False)
        sec64, _ = time_steps(torch, sv64, stream, args.fp64_steps, 2, dist)
        fp64_value = whole_job_rate(nodes * 3 * args.fp64_steps, world, sec64)
        kt64 = stage_kernel_times(torch, sv64, stream, reps=2)
        sv64.close()
        fl64 = sum(f * nodes for f in FP64_STAGE_FLOP_PER_NODE) / sum(kt64)
        fp64 = {"value": fp64_value, "unit": UNIT, "steps": args.fp64_steps,
                "stage_ms": [1e3 * t for t in kt64], "speedup_mixed_over_fp64": value / fp64_value,
                "roofline": {"bound": "fp64", "achieved": fl64 / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                             "frac": fl64 / fp64_peak, "flop_per_node": list(FP64_STAGE_FLOP_PER_NODE),
                             "kernel": "k_stage<3, LawEuler<double>, double>",
                             "peak_kind": "measured (sidp_fma_peak, float64 fused multiply-add)"}}

    curved = None
    if not args.no_curved:
        curved = run_curved(torch, sidp, stream, max(20, args.steps // 4), 3, hbm, peak_kind)

    batched = None
    if not args.no_batched:
        batched = run_batched(torch, sidp, stream, max(10, args.steps // 4), 2, hbm, peak_kind)
    accuracy = None if args.no_accuracy else run_accuracy(sidp, stream)
    dmr = (run_dmr(sidp, args.dmr, args.dmr_t, args.dmr_image, max_seconds=args.dmr_max_seconds,
                   stats_from=args.dmr_stats_from) if args.dmr else None)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": workload_label(NEL),
                           "nodes_per_gpu": nodes, "precision": "mixed (f32 state/stage, f64 dt)",
                           "l2": "state >= 151 MB per buffer > L2 (no flush needed)",
                           "parallelism": "independent replica per GPU"},
                "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                             "traffic": traffic, "kernel": kname, "tile_index": tidx,
                             "stage_ms": [1e3 * t for t in kt], "peak_kind": peak_kind,
                             "whole_step_gbs": step_gbs, "whole_step_frac": step_gbs / hbm,
                             "other_ceilings": other_ceilings(nodes, kt, clk, fp32_peak, ctr)},
                "fp64": fp64, "curved": curved, "batched": batched, "invariants": diag_stats, "accuracy": accuracy, "dmr": dmr,
                "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
                "gpu_launches": 5 * args.steps}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
