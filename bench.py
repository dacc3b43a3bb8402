#!/usr/bin/env python
"""Throughput of adaptive SDC on the 3D monodomain slab (201x71x31 nodes,
442,401 dofs, M = 4 Radau nodes, dt = 0.05 ms, 5 sweeps, TOL = 1e-5, 1 ms
corner stimulus) on one GB300, through the library's C ABI.

One benchmark step = one SDC time step (all sweeps, all node solves, the
selection and extraction of the nested active sets).  The K timed steps are the
first K steps of the trajectory from t = 0 (K = 1000 covers the workload's
50 ms).  Between timed steps L2 is flushed by writing a 256 MiB buffer; each
step is timed with CUDA events on the library's stream.

Printed as one JSON line: steps/s (value), active-dof sweeps/s, the plain-SDC
run at the same dt with its speedup and both errors against a 12-sweep
reference, the live roofline of the dominant kernel (restricted PCG), the
end-to-end rate through the host-buffer entry point, the CPU oracle timed on a
bounded sample of the same trajectory, and the SM clocks seen meanwhile.

--impl reference times the CPU oracle alone (single thread) on the same
workload and prints the same line with "impl": "reference".
"""

from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "SDC steps/s & active-dof sweeps/s (3D slab), adaptive vs plain at equal err; HBM GB/s"


def metric_of(wl):
    """The headline metric for the 3D slab; the same quantity named per workload otherwise."""
    if wl.name.startswith("w1_slab"):
        return METRIC
    return "SDC steps/s & active-dof sweeps/s (%s), adaptive TOL=%g vs plain; HBM GB/s" % (
        wl.name, wl.tol)
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 1000 for w1, 50 = 1 ms for w2, 300 for "
                         "w1l/w5, 100 for w0/w3, 200 for w4)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["w1", "w1l", "w0", "w5", "w2", "w3", "w4", "sweet",
                                           "sweet_emi", "order"],
                    default="w1",
                    help="w2: cell-by-cell (EMI) bricks; w3: 96-instance batch, batched launches "
                         "vs per-instance launches; w4: gradient by the discrete adjoint vs "
                         "finite differences; sweet / sweet_emi: final error vs drop tolerance "
                         "for several SDC tolerances on the 2D square / the 2D branched "
                         "cell-by-cell myocytes (energy-norm stop); order: error vs device "
                         "time for M = 2..6 and dt = 0.025..0.2 ms on the slab")
    ap.add_argument("--fd-directions", type=int, default=16)
    ap.add_argument("--ref-sweeps", type=int, default=12)
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip plain/reference/e2e runs")
    ap.add_argument("--emi-w-frozen", action="store_true", help="w2: hold the gating at w = 0")
    ap.add_argument("--emi-cells", default="8,4,4",
                    help="w2: brick cells along x,y,z (default 8,4,4 = 1,471,260 dofs)")
    ap.add_argument("--emi-coarse", default="16,4,4",
                    help="w2: two-level preconditioner of the node solves over blocks = the "
                         "cells and the extracellular space cut into this many boxes "
                         "(x,y,z); 'off' for Jacobi alone")
    ap.add_argument("--emi-coarse-min-rows", type=int, default=100000,
                    help="w2 with coarse blocks: sweeps with fewer active rows solve with "
                         "Jacobi alone (0: every sweep two-level)")
    ap.add_argument("--emi-order", choices=["block", "natural"], default="block",
                    help="w2 with coarse blocks: number the dofs block by block (block) or "
                         "keep the mesh's numbering (natural)")
    ap.add_argument("--autotune", type=int, choices=[0, 1], default=None,
                    help="pick the node solves' launch shape with sdc_autotune before timing "
                         "(default: on for the batch w3, off otherwise)")
    ap.add_argument("--reorder", type=int, choices=[0, 1], default=None,
                    help="library-internal Morton numbering of the dofs (default: on for the "
                         "randomly numbered tissue mesh w5, off otherwise)")
    args = ap.parse_args()
    if args.reorder is None:
        args.reorder = 1 if args.workload == "w5" else 0
    if args.autotune is None:
        args.autotune = 1 if args.workload == "w3" else 0
    if args.steps is None:
        args.steps = {"w1": 1000, "w2": 50, "w1l": 300, "w5": 300, "w0": 100, "w3": 100,
                      "w4": 200, "sweet": 100, "sweet_emi": 125, "order": 80}[args.workload]
    return args


def make_workload(name):
    return {"w1": W.w1_slab, "w1l": W.w1l_slab, "w0": W.w0_square, "w5": W.w5_tissue}[name]()


def config_of(wl, K, reorder=0):
    return {"workload": wl.name, "n_dofs": wl.n, "M": wl.M, "dt_ms": wl.dt, "sweeps": wl.sweeps,
            "TOL": wl.tol, "alpha": wl.alpha, "cg_rtol": wl.cg_rtol,
            "dof_numbering": "library Morton order" if reorder else "as generated",
            "simulated_ms": round(K * wl.dt, 6),
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"}


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_id):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", device_id, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        sm, mx, reasons = [], [], set()
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(self.NAMES, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.tmp.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- distributed
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "gb300" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle
def host_info():
    """The host the oracle ran on: logical cores and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model or platform.machine()}


def oracle_steps(wl, states, budget_s):
    """Time single oracle steps from the given (step index, v, w) states until the
    budget is used.  Returns (steps done, seconds, per-step results)."""
    import oracle
    S = oracle.System.from_mesh(wl.mesh, wl.sigma, wl.dof_scale)
    done, secs, outs = 0, 0.0, []
    for (n, v, w) in states:
        t0 = time.perf_counter()
        r = S.step(wl.ionic, wl.M, v, w, wl.dt, wl.sweeps, wl.tol, alpha=wl.alpha,
                   cg_rtol=wl.cg_rtol, istim=wl.stim_vector(n * wl.dt))
        secs += time.perf_counter() - t0
        done += 1
        outs.append((n, r))
        if r["status"] != 0:
            raise RuntimeError("oracle step failed with status %d" % r["status"])
        if secs >= budget_s:
            break
    return done, secs, outs


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    wl = make_workload(args.workload)
    import oracle
    S = oracle.System.from_mesh(wl.mesh, wl.sigma, wl.dof_scale)
    v, w = wl.v0.copy(), wl.w0.copy()
    # warm-up: W oracle steps on a copy of the initial state (untimed)
    wv, ww = v.copy(), w.copy()
    for n in range(min(args.warmup, 1)):
        r = S.step(wl.ionic, wl.M, wv, ww, wl.dt, wl.sweeps, wl.tol, alpha=wl.alpha,
                   cg_rtol=wl.cg_rtol, istim=wl.stim_vector(n * wl.dt))
    budget = max(10.0, min(120.0, args.cpu_budget * 3))
    done, secs, nact = 0, 0.0, 0
    while done < args.steps and secs < budget:
        t0 = time.perf_counter()
        r = S.step(wl.ionic, wl.M, v, w, wl.dt, wl.sweeps, wl.tol, alpha=wl.alpha,
                   cg_rtol=wl.cg_rtol, istim=wl.stim_vector(done * wl.dt))
        secs += time.perf_counter() - t0
        if r["status"] != 0:
            print(json.dumps({"impl": "reference", "unavailable": "oracle step failed: %d"
                              % r["status"]}))
            return 0
        v, w = r["v"], r["w"]
        nact += sum(r["stats"].n_active[:wl.sweeps])
        done += 1
    value = done / secs
    sample = ("first %d of the %d requested steps from t = 0 (single-threaded FP64 oracle, "
              "time budget %.0f s)" % (done, args.steps, budget))
    line = {"impl": "reference", "metric": metric_of(wl), "value": value, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": done, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / done, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, done),
            "active_dof_sweeps_per_s": nact / secs,
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_info()},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
FP64_LANES_PER_CYCLE = 304          # whole GPU, ncu dfma peak_sustained on GB300
# measured warp FP64 issue rate as a fraction of that peak (a warp FP64 instruction holds a
# sub-partition's FP64 unit for ~76 cycles: 1.68 of 2.0 lanes per cycle per SM)
FP64_ISSUE_FRACTION = 0.84
SIZE_CLASSES = ((1, 10_000, "<=10k rows"), (10_001, 300_000, "10k-300k rows"),
                (300_001, 1 << 62, ">300k rows"))
CG_SOURCES = ("step.cu", "device_common.cuh")
# DRAM traffic of the dominant kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the first node solve of a slab step, all 442,401 rows, scaled to
# the average launch by algorithmic bytes.  `source_sha` is the hash of the CG sources the
# capture was taken with (kernel_source_sha()); once they change, the figure is withheld.
ERR_NORM = ("max over ten checkpoints evenly spaced in the window (the last step included) of "
            "max_i |v_i(t) - v_ref,i(t)|")
ERR_NORM_U = ERR_NORM.replace("|v_i(t) - v_ref,i(t)|", "|u_i(t) - u_ref,i(t)|")


# ---- equal-error pairs (host logic) -----------------------------------------------
# plain: {fixed sweeps: (err, ms)}; adapt: [(TOL, err, ms)] in the order run.

def plain_partner(plain, err):
    """The plain run with the fewest sweeps whose error is within 1.1x of err (the most
    sweeps when none is)."""
    cands = [kp for kp in sorted(plain) if plain[kp][0] <= 1.1 * err]
    return cands[0] if cands else max(plain)


def closest_pair(plain, adapt):
    """(j, kp) of the adaptive and plain runs whose errors are closest in log."""
    return min(((j, kp) for j in range(len(adapt)) for kp in plain),
               key=lambda q: abs(np.log(max(adapt[q[0]][1], 1e-300)
                                        / max(plain[q[1]][0], 1e-300))))


def interp_plain_ms(plain, err):
    """Plain time at error err, log-log between the two plain runs whose errors bracket
    it; None outside their range."""
    pts = sorted((e, m) for e, m in plain.values() if e > 0)
    for (e_lo, m_lo), (e_hi, m_hi) in zip(pts, pts[1:]):
        if e_lo <= err <= e_hi and e_hi > e_lo:
            f = np.log(err / e_lo) / np.log(e_hi / e_lo)
            return float(np.exp(np.log(m_lo) + f * np.log(m_hi / m_lo)))
    return None

PCG_TRAFFIC = {"w1": {"dram_bytes": 64.25e6 + 10.65e6, "algorithmic_bytes": 1.735e9,
                      "kernel": "k_pcg_scaled<1024>", "source_sha": "f6df4e0ce07892df",
                      "capture": "profiles/pcg_scaled_w1_slab_full_solve.md"}}


def kernel_source_sha():
    """Hash of the CG kernel sources (the code the ncu traffic figure describes)."""
    import hashlib
    h = hashlib.sha256()
    for f in CG_SOURCES:
        with open(os.path.join(ROOT, "paper_2311_07206_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def pcg_ops(st, M, sweeps, extra_per_row=0.0):
    """Algorithmic FP64 operations (lane instructions) of the PCG solves of one
    step: per iteration and active row zbar + 8 (SpMV zbar + 1, p and q updates,
    two dot products, x and r updates, z = r / diag), plus extra_per_row (the
    two-level preconditioner: 2, the piece sum of Y'w and u = r + Y y)."""
    ops = 0.0
    for k in range(st.sweeps_run):
        n = st.n_active[k]
        if n == 0:
            continue
        nnz = st.nnz_active[k] + n
        per_iter = nnz + (8.0 + extra_per_row) * n
        for m in range(M):
            ops += st.cg_iters[k][m] * per_iter
    return ops


def pcg_bytes(st, M, sweeps, extra_per_row=0.0):
    """Algorithmic bytes of the restricted PCG solves of one step: per iteration
    and active row 12 zbar + 104 B (zbar = stored entries per row incl. the
    diagonal; FP64 values, int32 indices, fused vector traffic), plus
    extra_per_row (the two-level preconditioner: 20 B, the row's position in the
    block order, Y_i, and the store of u)."""
    b = 0.0
    for k in range(st.sweeps_run):
        n = st.n_active[k]
        if n == 0:
            continue
        nnz = st.nnz_active[k] + n
        per_iter = 12.0 * nnz + (104.0 + extra_per_row) * n
        for m in range(M):
            b += st.cg_iters[k][m] * per_iter
    return b


class SolveTable:
    """Node solves of a run grouped by active-set size: count, mean iterations,
    device microseconds per iteration, the FP64 floor of an iteration (zbar + 8
    operations per row at the measured issue rate) and the share of PCG time."""

    def __init__(self, sm_mhz):
        self.rate = FP64_LANES_PER_CYCLE * FP64_ISSUE_FRACTION * sm_mhz * 1e6   # lane-op/s
        self.c = {label: [0, 0, 0.0, 0.0, 0.0] for _, _, label in SIZE_CLASSES}

    def add(self, st, M):
        for k in range(st.sweeps_run):
            n = st.n_active[k]
            if n == 0:
                continue
            ops_it = st.nnz_active[k] + n + 8.0 * n
            label = [lb for lo, hi, lb in SIZE_CLASSES if lo <= n <= hi][0]
            e = self.c[label]
            for m in range(M):
                it = st.cg_iters[k][m]
                e[0] += 1
                e[1] += it
                e[2] += st.cg_ms[k][m]
                e[3] += it * ops_it / self.rate * 1e3
                e[4] += it * ops_it

    def table(self):
        tot = sum(e[2] for e in self.c.values()) or 1.0
        out = []
        for _, _, label in SIZE_CLASSES:
            solves, iters, ms, floor_ms, ops = self.c[label]
            if solves == 0:
                continue
            out.append({"class": label, "solves": solves, "mean_iters": iters / solves,
                        "us_per_iter": 1e3 * ms / max(1, iters),
                        "fp64_floor_us_per_iter": 1e3 * floor_ms / max(1, iters),
                        "share_of_pcg": ms / tot,
                        "fp64_frac": ops / (ms * 1e-3) / (self.rate / FP64_ISSUE_FRACTION)
                        if ms > 0 else None})
        return out


def run_gb300(args):
    """The headline slab (and the other monodomain workloads): timed windows of
    adaptive SDC with the plain run, equal-error pairs, roofline and baselines."""
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2311_07206_gb300 import Context, default_options

    wl = make_workload(args.workload)
    K, Wm = args.steps, args.warmup
    stream = torch.cuda.current_stream(dev)

    def new_ctx(**kw):
        o = default_options(profile=1, cg_rtol=wl.cg_rtol, alpha=wl.alpha, reorder=args.reorder)
        for k, v in kw.items():
            setattr(o, k, v)
        return Context.from_workload(wl, options=o, stream=stream.cuda_stream)

    ctx = new_ctx()
    v0 = torch.tensor(wl.v0, dtype=torch.float64, device=dev)
    w0 = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    peaks = {}
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as f:
            peaks = json.load(f)
    hbm_peak = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    tune = None
    if args.autotune:
        tune = ctx.autotune(v0.clone(), w0.clone(), 0.0, wl.dt, wl.sweeps, wl.tol, trial_steps=3)

    def checkpoints(steps):
        """Step offsets after which errors are measured: ten, evenly spaced, the last
        step included (a long window's final state alone can sit at rest)."""
        return sorted({max(0, (j * steps) // 10 - 1) for j in range(1, 11)})

    def trajectory(c, vs, ws, n0, steps, tol, sweeps, timed, table=None, ref=None,
                   record=False):
        """`steps` steps of context c from (vs, ws) at step index n0 (inputs kept).
        record: also return v at the checkpoints (device copies, taken outside the
        timed region); ref: such a record, against which the run's error (max over
        the checkpoints of max |v - v_ref|) is returned instead."""
        v, w = vs.clone(), ws.clone()
        ck = set(checkpoints(steps)) if (record or ref is not None) else set()
        snaps, err = [], None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)] if timed else None
        agg = {"active_dof_sweeps": 0, "pcg_ms": 0.0, "pcg_launches": 0, "pcg_bytes": 0.0,
               "pcg_ops": 0.0, "launches": 0, "phase_ms": np.zeros(5), "sweeps": 0}
        for i in range(steps):
            n = n0 + i
            if timed:
                flush.fill_(n)
                ev[i][0].record(stream)
            st = c.step(v, w, n * wl.dt, wl.dt, sweeps, tol)
            if timed:
                ev[i][1].record(stream)
            agg["active_dof_sweeps"] += sum(st.n_active[:st.sweeps_run])
            agg["sweeps"] += st.sweeps_run
            agg["pcg_ms"] += st.phase_ms[1]
            agg["pcg_launches"] += st.phase_launches[1]
            agg["pcg_bytes"] += pcg_bytes(st, wl.M, sweeps)
            agg["pcg_ops"] += pcg_ops(st, wl.M, sweeps)
            agg["launches"] += st.kernel_launches
            agg["phase_ms"] += np.array(st.phase_ms[:5])
            if table is not None:
                table.add(st, wl.M)
            if i in ck:
                if record:
                    snaps.append(v.clone())
                else:
                    e = (v - ref[len(snaps)]).abs().max()
                    snaps.append(None)
                    err = e if err is None else torch.maximum(err, e)
        torch.cuda.synchronize(dev)
        total_ms = sum(a.elapsed_time(b) for a, b in ev) if timed else None
        if record:
            return v, w, total_ms, agg, snaps
        if ref is not None:
            return v, w, total_ms, agg, float(err)
        return v, w, total_ms, agg

    def roofline_of(agg, ms_step_total):
        alu_peak = FP64_LANES_PER_CYCLE * sm_max * 1e6 / 1e9            # G op/s
        pcg_s = agg["pcg_ms"] / 1e3
        launches = max(1, agg["pcg_launches"])
        ach_ops = agg["pcg_ops"] / pcg_s / 1e9 if pcg_s > 0 else None
        ach_gbs = agg["pcg_bytes"] / pcg_s / 1e9 if pcg_s > 0 else None
        avg_ms = agg["pcg_ms"] / launches
        r = {"kernel": "k_pcg_scaled / k_pcg* (restricted Jacobi-PCG, symmetrically scaled "
                       "form, one cooperative launch per node solve)",
             "bound": "alu", "achieved": ach_ops, "peak": alu_peak, "unit": "G FP64 lane-op/s",
             "frac": ach_ops / alu_peak if ach_ops else None,
             "peak_source": "304 FP64 lanes/cycle (ncu dfma peak_sustained) x %.0f MHz max SM "
                            "clock" % sm_max,
             "traffic": None, "traffic_source": None,
             "algorithmic_ops_per_launch": agg["pcg_ops"] / launches,
             "algorithmic_bytes_per_launch": agg["pcg_bytes"] / launches,
             "avg_launch_ms": avg_ms, "launches": agg["pcg_launches"],
             "share_of_step": agg["pcg_ms"] / ms_step_total,
             # algorithmic bytes over time: what the kernel moves through L2 and DRAM together
             "effective_view": {"achieved": ach_gbs, "unit": "GB/s",
                                "note": "algorithmic bytes / time; the solves' working set "
                                        "is L2-resident, so this is not an HBM rate"},
             "dram_view": None}
        tr = PCG_TRAFFIC.get(args.workload)
        if tr is not None and agg["pcg_launches"] > 0:
            sha = kernel_source_sha()
            if tr["source_sha"] == sha:
                r["traffic"] = tr["dram_bytes"] / tr["algorithmic_bytes"] * (
                    agg["pcg_bytes"] / launches)
                r["traffic_source"] = (
                    "ncu DRAM bytes of one full-size %s launch (%.1f MB for %.3f GB "
                    "algorithmic; %s; CG sources %s), scaled to the average launch by "
                    "algorithmic bytes" % (tr["kernel"], tr["dram_bytes"] / 1e6,
                                           tr["algorithmic_bytes"] / 1e9, tr["capture"], sha))
                gbs = r["traffic"] / (avg_ms / 1e3) / 1e9
                r["dram_view"] = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                  "frac": gbs / hbm_peak,
                                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"
                                  if "hbm_gbs" in peaks else "fallback 6.8 TB/s"}
            else:
                r["traffic_source"] = ("withheld: the CG sources (%s) changed since the ncu "
                                       "capture (%s)" % (sha, tr["source_sha"]))
        return r

    def err_of(snaps, ref):
        return max(float((a - b).abs().max()) for a, b in zip(snaps, ref))

    def equal_error(vs, ws, n0, steps, ref, err_a, ms_a):
        """(fixed) adaptive with the workload's sweeps against plain SDC with the fewest
        fixed sweeps whose error is within 1.1x; the adaptive TOL is halved (up to five
        times) until its error is within 1.1x of that partner's.  (energy_stop) the
        energy-norm stop of Sec. 3.2 at the same TOL (rho = 0.05, at most 12 sweeps),
        no dropping (alpha = 0) against alpha = 0.1, TOL halved on the adaptive side the
        same way.  All errors against plain SDC with 12 sweeps from the same state."""
        plain = {}
        for kp in range(1, wl.sweeps + 3):
            _, _, ms, _, e = trajectory(ctx, vs, ws, n0, steps, 0.0, kp, timed=True, ref=ref)
            plain[kp] = (e, ms)
        adapt = [(wl.tol, err_a, ms_a)]
        pick = None
        for j in range(6):
            if j > 0:
                tol_j = wl.tol / 2 ** j
                _, _, ms, _, e = trajectory(ctx, vs, ws, n0, steps, tol_j, wl.sweeps,
                                            timed=True, ref=ref)
                adapt.append((tol_j, e, ms))
            e_a = adapt[j][1]
            kp = plain_partner(plain, e_a)
            if e_a <= 1.1 * plain[kp][0]:
                pick = (j, kp)
                break
        matched = pick is not None
        j, kp = pick if matched else closest_pair(plain, adapt)
        interp = interp_plain_ms(plain, adapt[j][1])
        fixed = {"adaptive": {"TOL": adapt[j][0], "sweeps": wl.sweeps, "err": adapt[j][1],
                              "ms_per_step": adapt[j][2] / steps},
                 "speedup_interpolated": interp / adapt[j][2] if interp else None,
                 "interpolation": "plain ms/step at the adaptive error, log-log between the "
                                  "two fixed-sweep plain runs whose errors bracket it",
                 "plain": {"sweeps": kp, "err": plain[kp][0],
                           "ms_per_step": plain[kp][1] / steps},
                 "matched_within_1.1x": matched,
                 "speedup": plain[kp][1] / adapt[j][2],
                 "plain_sweep_scan": {str(k): {"err": e, "ms_per_step": m / steps}
                                      for k, (e, m) in plain.items()},
                 "adaptive_tol_scan": [{"TOL": t, "err": e, "ms_per_step": m / steps}
                                       for t, e, m in adapt]}
        # energy-norm stop pair
        es_ctx = {a: new_ctx(alpha=a, energy_stop=1, sdc_rho=0.05) for a in (0.0, wl.alpha)}
        _, _, ms0, agg0, e0 = trajectory(es_ctx[0.0], vs, ws, n0, steps, wl.tol, 12,
                                         timed=True, ref=ref)
        scan = []
        for j in range(5):
            tol_j = wl.tol / 2 ** j
            _, _, ms1, agg1, e1 = trajectory(es_ctx[wl.alpha], vs, ws, n0, steps, tol_j, 12,
                                             timed=True, ref=ref)
            scan.append({"TOL": tol_j, "err": e1, "ms_per_step": ms1 / steps,
                         "mean_sweeps": agg1["sweeps"] / steps})
            if scan[-1]["err"] <= 1.1 * e0:
                break
        best = scan[-1]
        energy = {"non_adaptive": {"TOL": wl.tol, "alpha": 0.0, "err": e0,
                                   "ms_per_step": ms0 / steps,
                                   "mean_sweeps": agg0["sweeps"] / steps},
                  "adaptive": dict(best, alpha=wl.alpha),
                  "matched_within_1.1x": best["err"] <= 1.1 * e0,
                  "speedup": (ms0 / steps) / best["ms_per_step"],
                  "adaptive_tol_scan": scan}
        for c in es_ctx.values():
            c.close()
        return {"fixed_sweeps": fixed, "energy_stop": energy,
                "reference": "plain SDC, %d sweeps, same dt, same start" % args.ref_sweeps,
                "norm": ERR_NORM}

    def window(vs, ws, n0, steps, extras, table):
        """Timed adaptive run of `steps` steps from (vs, ws) at step n0, then (extras) the
        plain run, the errors, and the equal-error pairs."""
        trajectory(ctx, vs, ws, n0, Wm, wl.tol, wl.sweeps, timed=False)   # warm-up
        props = torch.cuda.get_device_properties(dev)
        dev_id = str(getattr(props, "uuid", "")) or str(local)
        if dev_id and not dev_id.startswith("GPU-") and len(dev_id) > 8:
            dev_id = "GPU-" + dev_id
        barrier(world)
        torch.cuda.synchronize(dev)
        clocks = Clocks(dev_id)
        res = trajectory(ctx, vs, ws, n0, steps, wl.tol, wl.sweeps, timed=True, table=table,
                         record=bool(extras))
        va, wa, ms_a, agg_a = res[:4]
        snaps_a = res[4] if extras else None
        torch.cuda.synchronize(dev)
        barrier(world)
        clk = clocks.stop()
        ms_a = max_over_ranks(ms_a, world)
        out = {"value": world * steps / (ms_a / 1e3), "ms_per_step": ms_a / steps,
               "active_dof_sweeps_per_s": world * agg_a["active_dof_sweeps"] / (ms_a / 1e3),
               "agg": agg_a, "clocks": clk, "va": va, "wa": wa}
        if extras:
            _, _, _, _, ref = trajectory(ctx, vs, ws, n0, steps, 0.0, args.ref_sweeps,
                                         timed=False, record=True)
            _, _, ms_p, agg_p, err_p = trajectory(ctx, vs, ws, n0, steps, 0.0, wl.sweeps,
                                                  timed=True, ref=ref)
            err_a = err_of(snaps_a, ref)
            del snaps_a
            out["plain"] = {"value": steps / (ms_p / 1e3), "unit": "steps/s",
                            "ms_per_step": ms_p / steps,
                            "active_dof_sweeps_per_s": agg_p["active_dof_sweeps"] / (ms_p / 1e3)}
            out["speedup_vs_plain"] = ms_p / ms_a
            out["err_vs_ref"] = {"adaptive": err_a, "plain": err_p,
                                 "reference": "plain SDC, %d sweeps, same dt" % args.ref_sweeps,
                                 "norm": ERR_NORM}
            out["equal_error"] = equal_error(vs, ws, n0, steps, ref, err_a, ms_a)
        return out

    # ---- window 1: the first K steps from t = 0 (the headline value)
    table0 = SolveTable(sm_max)
    win0 = window(v0, w0, 0, K, not args.no_extras, table0)
    agg_a, ms_adapt = win0["agg"], win0["ms_per_step"] * K
    value = win0["value"]
    extras = {k: win0[k] for k in ("plain", "speedup_vs_plain", "err_vs_ref", "equal_error")
              if k in win0}

    # ---- end to end through the host-buffer entry point (pinned host arrays)
    samples = sorted({s for s in (0, K // 5, 2 * K // 5, 3 * K // 5, 4 * K // 5) if s + 1 < K})
    snaps = {}
    hv_t = torch.tensor(wl.v0, dtype=torch.float64).pin_memory()
    hw_t = torch.tensor(wl.w0, dtype=torch.float64).pin_memory()
    hv, hw = hv_t.numpy(), hw_t.numpy()
    torch.cuda.synchronize(dev)
    barrier(world)
    e2e_s = 0.0
    for n in range(K):
        if n in samples or n - 1 in samples:
            snaps[n] = (hv.copy(), hw.copy())      # outside the timed call
        t0 = time.perf_counter()
        ctx.step_host(hv, hw, n * wl.dt, wl.dt, wl.sweeps, wl.tol)
        e2e_s += time.perf_counter() - t0
    e2e = {"value": world * K / max_over_ranks(e2e_s, world), "unit": "steps/s",
           "h2d_bytes_per_step": 2 * 8 * wl.n, "d2h_bytes_per_step": 2 * 8 * wl.n,
           "api": "sdc_step_host (pinned host v, w)"}

    roofline = roofline_of(agg_a, ms_adapt)
    roofline["size_classes"] = table0.table()

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        states = [(s, snaps[s][0], snaps[s][1]) for s in samples if s in snaps]
        done, secs, outs = oracle_steps(wl, states, args.cpu_budget)
        cpu = {"value": done / secs, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": "%d single steps of the same trajectory, started from the GPU states at "
                         "steps %s (single-threaded FP64 oracle)"
                         % (done, [s for s, _ in outs]), "host": host_info()}
        diffs = []
        for s, r in outs:
            if s + 1 in snaps:
                gv = snaps[s + 1][0]
                diffs.append(float(np.abs(gv - r["v"]).max() / max(1.0, np.abs(r["v"]).max())))
        parity = {"max_rel_diff_v_vs_oracle": max(diffs) if diffs else None, "steps": len(diffs)}

    # ---- window 2: the propagating front, from the state at t = 20 ms (slab only)
    win20 = None
    if args.workload == "w1" and not args.no_extras:
        n20 = int(round(20.0 / wl.dt))
        steps20 = max(1, min(K, wl.steps - n20))
        v20, w20 = v0.clone(), w0.clone()
        t_adv = time.perf_counter()
        n_adv = 0
        while n_adv < n20 and time.perf_counter() - t_adv < 30.0:
            ctx.step(v20, w20, n_adv * wl.dt, wl.dt, wl.sweeps, wl.tol, want_stats=False)
            n_adv += 1
        torch.cuda.synchronize(dev)
        table20 = SolveTable(sm_max)
        w2 = window(v20, w20, n_adv, steps20, True, table20)
        rf = roofline_of(w2["agg"], w2["ms_per_step"] * steps20)
        rf["size_classes"] = table20.table()
        win20 = {"t_start_ms": n_adv * wl.dt, "steps": steps20,
                 "advance": "untimed adaptive steps from t = 0 (capped at 30 s)",
                 "value": w2["value"], "unit": "steps/s", "ms_per_step": w2["ms_per_step"],
                 "active_dof_sweeps_per_s": w2["active_dof_sweeps_per_s"],
                 **{k: w2[k] for k in ("plain", "speedup_vs_plain", "err_vs_ref", "equal_error")},
                 "phase_ms_per_step": dict(zip(("residual", "pcg", "update", "select",
                                                "extract"),
                                               (w2["agg"]["phase_ms"] / steps20).round(4)
                                               .tolist())),
                 "roofline": rf, "clocks": w2["clocks"]}
        if rank == 0 and world == 1:
            # one oracle step from the window's start state against the library's step
            import oracle
            S = oracle.System.from_mesh(wl.mesh, wl.sigma, wl.dof_scale)
            hv20, hw20 = v20.cpu().numpy(), w20.cpu().numpy()
            vg, wg = v20.clone(), w20.clone()
            ctx.step(vg, wg, n_adv * wl.dt, wl.dt, wl.sweeps, wl.tol)
            acts_g = [ctx.active(k) for k in range(wl.sweeps)]
            t0 = time.perf_counter()
            r = S.step(wl.ionic, wl.M, hv20, hw20, wl.dt, wl.sweeps, wl.tol, alpha=wl.alpha,
                       cg_rtol=wl.cg_rtol, istim=wl.stim_vector(n_adv * wl.dt), want_log=True)
            secs = time.perf_counter() - t0
            vgn, wgn = vg.cpu().numpy(), wg.cpu().numpy()
            same = (r["status"] == 0 and len(r["active"]) <= len(acts_g) and all(
                np.array_equal(a, b) for a, b in zip(r["active"], acts_g)))
            win20["oracle_step"] = {
                "status": r["status"], "seconds": secs,
                "max_rel_diff_v": float(np.abs(vgn - r["v"]).max()
                                        / max(1.0, np.abs(r["v"]).max())),
                "max_rel_diff_w": float(np.abs(wgn - r["w"]).max()
                                        / max(1.0, np.abs(r["w"]).max())),
                "active_sets_identical": bool(same),
                "n_active": list(r["stats"].n_active[:r["stats"].sweeps_run])}

    phase = dict(zip(("residual", "pcg", "update", "select", "extract"),
                     (agg_a["phase_ms"] / K).round(4).tolist()))
    line = {"metric": metric_of(wl), "value": value, "unit": "steps/s", "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": ms_adapt / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config_of(wl, K, args.reorder), autotune=tune),
            "active_dof_sweeps_per_s": win0["active_dof_sweeps_per_s"],
            **extras,
            "phase_ms_per_step": phase,
            "roofline": roofline, "cpu_baseline": cpu, "oracle_parity_on_sample": parity,
            "e2e": e2e, "clocks": win0["clocks"], "gpu_launches": agg_a["launches"]}
    if win20 is not None:
        line["window_t20"] = win20
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


def run_emi(args):
    """Cell-by-cell (EMI) bricks: 8x4x4 myocytes of 100x20x20 um on 2 um voxels
    (1,471,260 dofs, 277,264 membrane pairs), M = 3, dt = 0.02 ms, 4 sweeps,
    TOL = 1e-5, Aliev-Panfilov gating on the cell-bath pairs (--emi-w-frozen
    holds w = 0 as in the paper's own EMI runs); the first cell starts
    excited.  Adaptive vs plain SDC, as for the slab."""
    import torch
    from workloads.emi import emi_bricks

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2311_07206_gb300 import Context, default_options

    frozen = bool(args.emi_w_frozen)
    cells = tuple(int(x) for x in args.emi_cells.split(","))
    wl = emi_bricks(cells=cells, w_frozen=frozen)
    K, Wm = args.steps, args.warmup
    stream = torch.cuda.current_stream(dev)
    opts = default_options(profile=1, cg_rtol=wl.cg_rtol, alpha=wl.alpha, w_frozen=int(frozen),
                           cg_maxit=100000, coarse_min_rows=args.emi_coarse_min_rows)
    blocks = None
    if args.emi_coarse != "off":
        from workloads.emi import block_major, coarse_blocks, renumber
        blocks = coarse_blocks(wl, split=tuple(int(x) for x in args.emi_coarse.split(",")))
        if args.emi_order == "block":
            # the same problem with its dofs numbered block by block: each block's rows
            # are contiguous in memory
            order, blocks = block_major(wl, blocks)
            wl = renumber(wl, order)
    ctx = Context.from_emi(wl, options=opts, stream=stream.cuda_stream)
    if blocks is not None:
        ctx.set_coarse_blocks(blocks)
    u0 = torch.tensor(wl.u0, dtype=torch.float64, device=dev)
    w0 = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
    tune = None
    if args.autotune:
        tune = ctx.autotune(u0.clone(), w0.clone(), 0.0, wl.dt, wl.sweeps, wl.tol, trial_steps=1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def trajectory(tol, sweeps, steps, timed, ref=None, record=False):
        """record: also return u at ten checkpoints (outside the timed region); ref: such
        a record, against which the run's error is returned instead."""
        u, w = u0.clone(), w0.clone()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)] if timed else None
        agg = {"active_dof_sweeps": 0, "pcg_ms": 0.0, "pcg_launches": 0, "pcg_bytes": 0.0,
               "pcg_ops": 0.0, "launches": 0, "phase_ms": np.zeros(5), "row_iters": 0.0,
               "iters_max": 0}
        ck = set(sorted({max(0, (j * steps) // 10 - 1) for j in range(1, 11)})) \
            if (record or ref is not None) else set()
        snaps, err = [], None
        for n in range(steps):
            if timed:
                flush.fill_(n)
                ev[n][0].record(stream)
            st = ctx.step(u, w, n * wl.dt, wl.dt, sweeps, tol)
            if timed:
                ev[n][1].record(stream)
            agg["active_dof_sweeps"] += sum(st.n_active[:st.sweeps_run])
            agg["pcg_ms"] += st.phase_ms[1]
            agg["pcg_launches"] += st.phase_launches[1]
            agg["pcg_bytes"] += pcg_bytes(st, wl.M, sweeps, 20.0 if blocks is not None else 0.0)
            agg["pcg_ops"] += pcg_ops(st, wl.M, sweeps, 2.0 if blocks is not None else 0.0)
            agg["launches"] += st.kernel_launches
            agg["phase_ms"] += np.array(st.phase_ms[:5])
            for k in range(st.sweeps_run):
                for m in range(wl.M):
                    agg["row_iters"] += st.n_active[k] * st.cg_iters[k][m]
                    agg["iters_max"] = max(agg["iters_max"], st.cg_iters[k][m])
            if n in ck:
                if record:
                    snaps.append(u.clone())
                else:
                    e = (u - ref[len(snaps)]).abs().max()
                    snaps.append(None)
                    err = e if err is None else torch.maximum(err, e)
        torch.cuda.synchronize(dev)
        total_ms = sum(a.elapsed_time(b) for a, b in ev) if timed else None
        if record:
            return u, w, total_ms, agg, snaps
        if ref is not None:
            return u, w, total_ms, agg, float(err)
        return u, w, total_ms, agg

    trajectory(wl.tol, wl.sweeps, Wm, timed=False)
    props = torch.cuda.get_device_properties(dev)
    dev_id = str(getattr(props, "uuid", "")) or str(local)
    if dev_id and not dev_id.startswith("GPU-") and len(dev_id) > 8:
        dev_id = "GPU-" + dev_id
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks = Clocks(dev_id)
    res = trajectory(wl.tol, wl.sweeps, K, timed=True, record=not args.no_extras)
    ua, _, ms_adapt, agg_a = res[:4]
    snaps_a = res[4] if not args.no_extras else None
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    ms_adapt = max_over_ranks(ms_adapt, world)
    value = world * K / (ms_adapt / 1e3)

    extras = {}
    if not args.no_extras:
        _, _, _, _, ref = trajectory(0.0, args.ref_sweeps, K, timed=False, record=True)
        _, _, ms_plain, agg_p, err_p = trajectory(0.0, wl.sweeps, K, timed=True, ref=ref)
        err_a = max(float((a - b).abs().max()) for a, b in zip(snaps_a, ref))
        del snaps_a
        # equal error: adaptive against the plain run with the fewest fixed sweeps whose
        # error is within 1.1x, the adaptive TOL halved (up to four times) until its error
        # is within 1.1x of that partner's
        plain = {}
        for kp in range(1, wl.sweeps + 2):
            _, _, ms_k, _, e_k = trajectory(0.0, kp, K, timed=True, ref=ref)
            plain[kp] = (e_k, ms_k)
        adapt = [(wl.tol, err_a, ms_adapt)]
        pick = None
        for j in range(5):
            if j > 0:
                tol_j = wl.tol / 2 ** j
                _, _, ms_j, _, e_j = trajectory(tol_j, wl.sweeps, K, timed=True, ref=ref)
                adapt.append((tol_j, e_j, ms_j))
            kp = plain_partner(plain, adapt[j][1])
            if adapt[j][1] <= 1.1 * plain[kp][0]:
                pick = (j, kp)
                break
        matched = pick is not None
        j, kp = pick if matched else closest_pair(plain, adapt)
        interp = interp_plain_ms(plain, adapt[j][1])
        extras = {"plain": {"value": K / (ms_plain / 1e3), "unit": "steps/s",
                            "ms_per_step": ms_plain / K,
                            "active_dof_sweeps_per_s": agg_p["active_dof_sweeps"] / (ms_plain / 1e3)},
                  "speedup_vs_plain": ms_plain / ms_adapt,
                  "err_vs_ref": {"adaptive": err_a, "plain": err_p,
                                 "reference": "plain SDC, %d sweeps, same dt" % args.ref_sweeps,
                                 "norm": ERR_NORM_U},
                  "equal_error": {"fixed_sweeps": {
                      "adaptive": {"TOL": adapt[j][0], "sweeps": wl.sweeps, "err": adapt[j][1],
                                   "ms_per_step": adapt[j][2] / K},
                      "plain": {"sweeps": kp, "err": plain[kp][0], "ms_per_step": plain[kp][1] / K},
                      "matched_within_1.1x": matched,
                      "speedup": plain[kp][1] / adapt[j][2],
                      "speedup_interpolated": interp / adapt[j][2] if interp else None,
                      "interpolation": "plain ms/step at the adaptive error, log-log between "
                                       "the two fixed-sweep plain runs whose errors bracket it",
                      "plain_sweep_scan": {str(k): {"err": e, "ms_per_step": m / K}
                                           for k, (e, m) in plain.items()},
                      "adaptive_tol_scan": [{"TOL": t, "err": e, "ms_per_step": m / K}
                                            for t, e, m in adapt]},
                      "reference": "plain SDC, %d sweeps, same dt, same start" % args.ref_sweeps,
                      "norm": ERR_NORM_U}}

    # end to end through the host-buffer entry point (pinned host u, w)
    hu_t = torch.tensor(wl.u0, dtype=torch.float64).pin_memory()
    hw_t = torch.tensor(wl.w0, dtype=torch.float64).pin_memory()
    hu, hw = hu_t.numpy(), hw_t.numpy()
    barrier(world)
    e2e_s = 0.0
    for n in range(K):
        t0 = time.perf_counter()
        ctx.step_host(hu, hw, n * wl.dt, wl.dt, wl.sweeps, wl.tol)
        e2e_s += time.perf_counter() - t0
    e2e = {"value": world * K / max_over_ranks(e2e_s, world), "unit": "steps/s",
           "h2d_bytes_per_step": 8 * (wl.n + wl.n_pairs),
           "d2h_bytes_per_step": 8 * (wl.n + wl.n_pairs),
           "api": "sdc_step_host (pinned host u, w)"}

    peaks = {}
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as f:
            peaks = json.load(f)
    hbm_peak = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = FP64_LANES_PER_CYCLE * sm_max * 1e6 / 1e9
    pcg_s = agg_a["pcg_ms"] / 1e3
    launches = max(1, agg_a["pcg_launches"])
    ach_ops = agg_a["pcg_ops"] / pcg_s / 1e9 if pcg_s > 0 else None
    ach_gbs = agg_a["pcg_bytes"] / pcg_s / 1e9 if pcg_s > 0 else None
    kname = ("k_pcgcs_coarse (two-level: Jacobi + block coarse space)" if blocks is not None
             else "k_pcg* (Jacobi)")
    roofline = {"kernel": kname + " on the EMI node operator (K + membrane pair slots)",
                "bound": "alu", "achieved": ach_ops, "peak": alu_peak,
                "unit": "G FP64 lane-op/s", "frac": ach_ops / alu_peak if ach_ops else None,
                "peak_source": "304 FP64 lanes/cycle (ncu dfma peak_sustained) x %.0f MHz max SM clock"
                               % sm_max,
                "traffic": None,
                "algorithmic_ops_per_launch": agg_a["pcg_ops"] / launches,
                "algorithmic_bytes_per_launch": agg_a["pcg_bytes"] / launches,
                "avg_launch_ms": agg_a["pcg_ms"] / launches, "launches": agg_a["pcg_launches"],
                "share_of_step": agg_a["pcg_ms"] / ms_adapt,
                "effective_view": {"achieved": ach_gbs, "unit": "GB/s",
                                   "note": "algorithmic bytes / time (L2 and DRAM together); "
                                           "no DRAM capture is stored for this workload"}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = emi_cpu_baseline(args.cpu_budget, agg_a["row_iters"] / K, frozen)

    phase = dict(zip(("residual", "pcg", "update", "select", "extract"),
                     (agg_a["phase_ms"] / K).round(4).tolist()))
    cfg = {"workload": wl.name, "n_dofs": wl.n, "n_pairs": wl.n_pairs, "M": wl.M,
           "dt_ms": wl.dt, "sweeps": wl.sweeps, "TOL": wl.tol, "alpha": wl.alpha,
           "cg_rtol": wl.cg_rtol,
           "gating": "held at w = 0" if frozen else "Aliev-Panfilov on cell-bath pairs", "simulated_ms": round(K * wl.dt, 6),
           "preconditioner": ("two-level: Jacobi + %d blocks (cells, extracellular space in "
                              "%s boxes)" % (int(blocks.max()) + 1, args.emi_coarse)
                              if blocks is not None else "Jacobi"),
           "coarse_min_rows": args.emi_coarse_min_rows if blocks is not None else None,
           "dof_order": ("block by block (workloads.emi.renumber)"
                         if blocks is not None and args.emi_order == "block" else "mesh"),
           "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas",
           "autotune": tune}
    line = {"metric": "SDC steps/s & active-dof sweeps/s (cell-by-cell bricks), adaptive "
                      "TOL=%g vs plain; HBM GB/s" % wl.tol,
            "value": value, "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": Wm,
            "ms_per_step": ms_adapt / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "active_dof_sweeps_per_s": world * agg_a["active_dof_sweeps"] / (ms_adapt / 1e3),
            "cg_iters_max": agg_a["iters_max"], **extras, "phase_ms_per_step": phase,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": agg_a["launches"]}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


def emi_cpu_baseline(budget_s, gpu_row_iters_per_step, frozen):
    """The oracle's EMI step on a two-cell instance of the same construction
    (100x20x20 um bricks, 2 um voxels), single thread, within the budget; its
    rate in CG row-iterations/s converted to steps/s of the full workload with
    the full workload's row-iterations per step measured on the GPU."""
    import oracle
    from workloads.emi import emi_bricks
    wl = emi_bricks(cells=(2, 1, 1), w_frozen=frozen)
    S = oracle.System.from_mesh(wl.mesh)
    u, w = wl.u0.copy(), wl.w0.copy()
    done, secs, row_iters = 0, 0.0, 0.0
    while secs < budget_s and done < 10:
        t0 = time.perf_counter()
        r = S.step_emi(wl, u, w, w_frozen=frozen)
        secs += time.perf_counter() - t0
        if r["status"] != 0:
            raise RuntimeError("oracle EMI step failed with status %d" % r["status"])
        st = r["stats"]
        row_iters += sum(st.n_active[k] * st.cg_iters[k * 8 + m]
                         for k in range(st.sweeps_run) for m in range(wl.M))
        u, w = r["u"], r["w"]
        done += 1
    rate = row_iters / secs
    return {"value": rate / gpu_row_iters_per_step, "unit": "steps/s", "cores": 1,
            "kind": "oracle", "same_config": False,
            "sample": "different configuration: %d oracle steps of a 2-cell instance of the same "
                      "construction (%d dofs) in %.1f s, %.3g CG row-iterations/s, divided by "
                      "the full workload's %.3g row-iterations per step (one oracle step of the "
                      "full workload takes minutes)"
                      % (done, wl.n, secs, rate, gpu_row_iters_per_step),
            "sample_steps_per_s": done / secs, "host": host_info()}



def run_sweet(args):
    """Sweet-line study (Sec. 5.2): final error against the drop tolerance
    TOL_drop = alpha TOL for several SDC tolerances TOL, the sweeps ended by the
    energy-norm test of Sec. 3.2 with the paper's rho = 0.05 (at most 12); the
    reference is plain SDC with 12 sweeps.  Per TOL also the non-adaptive run
    (alpha = 0: same stop, no dropping), whose time over the adaptive one at
    alpha = 0.1 is the speedup of the adaptivity, and the a priori drop
    tolerance of Sec. 4.1 (drop_rule 1, same rho).

    sweet: the 2D monodomain square (65x65 nodes, M = 3, dt = 0.1, 100 steps to
    t = 10).  sweet_emi: the 2D cell-by-cell branched myocytes of
    emi_branched_2d on 2.5 um pixels (28,809 dofs), gating held at w = 0 as in
    the paper's EMI runs, M = 3, dt = 0.02 ms, 125 steps to t = 2.5 ms (the time
    of the paper's EMI sweet-line figure).  The paper finds TOL_drop = TOL / 10
    close to the largest drop tolerance that leaves the accuracy unchanged."""
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2311_07206_gb300 import Context, default_options

    emi = args.workload == "sweet_emi"
    if emi:
        from workloads.emi import emi_branched_2d
        wl = emi_branched_2d(h=2.5)
        x0, y0 = wl.u0, wl.w0
    else:
        wl = W.w0_square()
        x0, y0 = wl.v0, wl.w0
    K, Wm = args.steps, args.warmup
    stream = torch.cuda.current_stream(dev)

    def run(tol, alpha, energy_stop, sweeps, drop_rule=0, keep_active=False):
        opts = default_options(alpha=alpha, energy_stop=int(energy_stop), sdc_rho=0.05,
                               cg_rtol=wl.cg_rtol, drop_rule=drop_rule,
                               w_frozen=int(emi), cg_maxit=100000)
        ctx = (Context.from_emi(wl, options=opts, stream=stream.cuda_stream) if emi else
               Context.from_workload(wl, options=opts, stream=stream.cuda_stream))
        v = torch.tensor(x0, dtype=torch.float64, device=dev)
        w = torch.tensor(y0, dtype=torch.float64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ads, swp, tds, act = 0, 0, [], []
        e0.record(stream)
        for n in range(K):
            st = ctx.step(v, w, n * wl.dt, wl.dt, sweeps, tol)
            ads += sum(st.n_active[:st.sweeps_run])
            swp += st.sweeps_run
            tds.append(st.tol_drop)
            if keep_active:
                act.append(list(st.n_active[:st.sweeps_run]))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ctx.close()
        return v.cpu().numpy(), e0.elapsed_time(e1), ads, swp, float(np.mean(tds)), act

    for _ in range(max(1, Wm)):
        run(1e-4, 0.1, True, 12)
    ref = run(0.0, 0.1, False, 12)[0]
    rows, active_profile = [], None
    for tol in (1e-3, 1e-4, 1e-5, 1e-6):
        for alpha, rule in ((0.0, 0), (0.001, 0), (0.01, 0), (0.1, 0), (1.0, 0), (10.0, 0),
                            (None, 1)):
            keep = tol == 1e-4 and alpha == 0.1
            v, ms, ads, swp, td, act = run(tol, alpha if alpha is not None else 0.1, True, 12,
                                           drop_rule=rule, keep_active=keep)
            if keep:
                active_profile = act
            rows.append({"TOL": tol, "TOL_drop": td, "alpha": alpha,
                         "drop_rule": "a priori (Sec. 4.1)" if rule else "alpha TOL",
                         "err": float(np.abs(v - ref).max()), "ms_per_step": ms / K,
                         "mean_sweeps": swp / K, "active_dof_sweeps_per_step": ads / K})
    for r in rows:
        base = [q for q in rows if q["TOL"] == r["TOL"] and q["alpha"] == 0.0][0]
        r["speedup_vs_alpha0"] = base["ms_per_step"] / r["ms_per_step"]
    at = [r for r in rows if r["TOL"] == 1e-4 and r["alpha"] == 0.1][0]
    # mean active dofs per sweep index over the steps (the paper's active-dof figure)
    mean_active = []
    if active_profile:
        for k in range(max(len(a) for a in active_profile)):
            mean_active.append(float(np.mean([a[k] if k < len(a) else 0 for a in active_profile])))
    what = ("2D cell-by-cell branched myocytes, w = 0" if emi else "2D monodomain square")
    line = {"metric": "sweet-line study: max error at t = %g ms vs TOL_drop (%s, energy-norm "
                      "stop, rho = 0.05)" % (K * wl.dt, what),
            "value": 1e3 / at["ms_per_step"], "unit": "steps/s at TOL = 1e-4, TOL_drop = 1e-5",
            "n_gpus": world, "steps": K, "warmup": Wm, "ms_per_step": at["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "n_dofs": wl.n, "M": wl.M, "dt_ms": wl.dt,
                       "max_sweeps": 12, "rho": 0.05, "reference": "plain SDC, 12 sweeps",
                       "speedup_alpha_0.1_vs_non_adaptive": at["speedup_vs_alpha0"]},
            "mean_active_dofs_per_sweep_at_TOL_1e-4_alpha_0.1": mean_active,
            "table": rows}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_order(args):
    """Collocation order against step size (the speedup lever of Sec. 6: higher
    M with larger dt trades sweeps against order).  The slab of the headline
    workload (201x71x31 nodes, 1 ms corner stimulus) is integrated to t = 4 ms
    with M = 2, 3, 4, 6 nodes and dt = 0.025 .. 0.2 ms, adaptive (alpha = 0.1)
    with the energy-norm stop (rho = 0.05, at most 12 sweeps) at TOL = 1e-5;
    the error is max |v(4) - v_ref(4)| against plain SDC with M = 4, dt =
    0.0125 ms and 12 sweeps (order 7 once converged).  Each row gives the
    device time per simulated ms; rows that no other row beats in both error and
    time are marked pareto."""
    import dataclasses

    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2311_07206_gb300 import Context, default_options

    base = W.w1_slab()
    T, tol = 4.0, 1e-5
    stream = torch.cuda.current_stream(dev)

    def run(M, dt, tol, sweeps, energy_stop):
        wl = dataclasses.replace(base, M=M, dt=dt)
        opts = default_options(alpha=0.1, energy_stop=int(energy_stop), sdc_rho=0.05,
                               cg_rtol=1e-12)
        ctx = Context.from_workload(wl, options=opts, stream=stream.cuda_stream)
        v = torch.tensor(wl.v0, dtype=torch.float64, device=dev)
        w = torch.tensor(wl.w0, dtype=torch.float64, device=dev)
        steps = int(round(T / dt))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        swp, ads = 0, 0
        e0.record(stream)
        for n in range(steps):
            st = ctx.step(v, w, n * dt, dt, sweeps, tol)
            swp += st.sweeps_run
            ads += sum(st.n_active[:st.sweeps_run])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ctx.close()
        return v.cpu().numpy(), e0.elapsed_time(e1), swp / steps, ads / steps

    for _ in range(max(1, args.warmup)):
        run(3, 0.2, tol, 12, True)
    ref = run(4, 0.0125, 0.0, 12, False)[0]
    rows = []
    for M in (2, 3, 4, 6):
        for dt in (0.025, 0.05, 0.1, 0.2):
            v, ms, sw, ads = run(M, dt, tol, 12, True)
            rows.append({"M": M, "dt_ms": dt, "err": float(np.abs(v - ref).max()),
                         "ms_per_simulated_ms": ms / T, "mean_sweeps": sw,
                         "active_dof_sweeps_per_step": ads})
    for r in rows:
        r["pareto"] = not any(q["err"] <= r["err"] and q["ms_per_simulated_ms"] <
                              r["ms_per_simulated_ms"] for q in rows if q is not r)
    head = [r for r in rows if r["M"] == 4 and r["dt_ms"] == 0.05][0]
    line = {"metric": "collocation order vs step size: max error at t = 4 ms vs device time "
                      "(slab 201x71x31, adaptive, energy-norm stop)",
            "value": 1e3 / head["ms_per_simulated_ms"],
            "unit": "simulated ms per s at M = 4, dt = 0.05 ms",
            "n_gpus": world, "steps": int(round(T / 0.05)), "warmup": args.warmup,
            "ms_per_step": head["ms_per_simulated_ms"] * 0.05, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": base.name, "n_dofs": base.n, "TOL": tol, "alpha": 0.1,
                       "rho": 0.05, "max_sweeps": 12, "t_end_ms": T, "cg_rtol": 1e-12,
                       "reference": "plain SDC, M = 4, dt = 0.0125 ms, 12 sweeps"},
            "table": rows}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_batch(args):
    """96 2D instances (sides log-uniform in [64, 512], D ~ U[0.5, 2]): one
    batched step of all instances vs the same steps as per-instance launches."""
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2311_07206_gb300 import Batch, Context, default_options

    insts = W.batch_instances()
    wl0 = insts[0]
    K, Wm = args.steps, args.warmup
    stream = torch.cuda.current_stream(dev)
    opts = default_options(profile=0)
    batch = Batch(insts, options=opts, stream=stream.cuda_stream)
    solos = [Context.from_workload(wl, options=opts, stream=stream.cuda_stream) for wl in insts]
    t64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    v0 = np.concatenate([wl.v0 for wl in insts])
    w0 = np.concatenate([wl.w0 for wl in insts])

    def run_batched(steps, timed):
        v, w = t64(v0), t64(w0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)] if timed else []
        ads = 0
        for n in range(steps):
            if timed:
                ev[n][0].record(stream)
            st = batch.step(v, w, n * wl0.dt, wl0.dt, wl0.sweeps, wl0.tol)
            if timed:
                ev[n][1].record(stream)
            ads += sum(st.n_active[:st.sweeps_run])
        torch.cuda.synchronize(dev)
        return v, (sum(a.elapsed_time(b) for a, b in ev) if timed else None), ads

    def run_solo(steps, timed):
        vs = [t64(wl.v0) for wl in insts]
        ws = [t64(wl.w0) for wl in insts]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for n in range(steps):
            for b, wl in enumerate(insts):
                solos[b].step(vs[b], ws[b], n * wl.dt, wl.dt, wl.sweeps, wl.tol, want_stats=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return vs, (e0.elapsed_time(e1) if timed else None)

    tune = None
    if args.autotune:
        # launch shape of the batched solves picked by timing steps from the start state
        tv, tw = t64(v0), t64(w0)
        tune = batch.autotune(tv, tw, 0.0, wl0.dt, wl0.sweeps, wl0.tol, trial_steps=10)
    run_batched(Wm, False)
    run_solo(Wm, False)
    barrier(world)
    clocks = Clocks(str(local))
    vb, ms_b, ads = run_batched(K, True)
    clk = clocks.stop()
    vs, ms_s = run_solo(K, True)
    vbh = vb.cpu().numpy()
    diff = max(float(np.abs(vbh[batch.offsets[b]:batch.offsets[b + 1]] - vs[b].cpu().numpy()).max())
               for b in range(len(insts)))
    ms_b = max_over_ranks(ms_b, world)
    line = {"metric": "batched SDC steps/s, 96 2D instances (one step = every instance)",
            "value": world * K / (ms_b / 1e3), "unit": "steps/s", "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": ms_b / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batch_96_2d_instances", "n_dofs": int(batch.n),
                       "instances": len(insts), "M": wl0.M, "dt_ms": wl0.dt,
                       "sweeps": wl0.sweeps, "TOL": wl0.tol, "l2": "inputs larger than L2",
                       "autotune": tune},
            "instance_steps_per_s": world * K * len(insts) / (ms_b / 1e3),
            "active_dof_sweeps_per_s": world * ads / (ms_b / 1e3),
            "per_instance_launches": {"value": K / (ms_s / 1e3), "unit": "steps/s",
                                      "ms_per_step": ms_s / K},
            "speedup_vs_per_instance": ms_s / ms_b,
            "max_abs_diff_batched_vs_per_instance": diff,
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line))
    batch.close()
    for c in solos:
        c.close()
    return 0


def run_grad(args):
    """W4 (101x36x16 slab, M = 3, 200 steps): gradient of the probe loss with
    respect to the per-node conductivity scale and (k, a) by the discrete
    adjoint with checkpoints every 20 steps, checked against central
    differences on random directions with the active sets replayed."""
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2311_07206_gb300 import Context, default_options
    from paper_2311_07206_gb300.autodiff import TrajectoryLoss, _set_params, replayed_loss

    wl = W.w4_slab()
    steps = min(args.steps, wl.steps)
    ck = 20
    stream = torch.cuda.current_stream(dev)
    ctx = Context.from_workload(wl, options=default_options(cg_rtol=1e-12),
                                stream=stream.cuda_stream)
    t64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    probes = t64(wl.meta["probes"]).long()
    k0, a0 = wl.ionic["ga"], wl.ionic["a"]
    s_init = wl.dof_scale.copy()
    # target: the run with s = 1 and the nominal (k, a)
    _set_params(ctx, wl, t64(np.ones(wl.n)), k0, a0)
    v, w = t64(wl.v0), t64(wl.w0)
    targets = []
    for n in range(steps):
        ctx.step(v, w, n * wl.dt, wl.dt, wl.sweeps, wl.tol, want_stats=False)
        targets.append(v[probes].clone())
    for _ in range(max(1, args.warmup)):
        sc = t64(s_init).requires_grad_(True)
        ka = t64([k0, a0]).requires_grad_(True)
        TrajectoryLoss.apply(sc, ka, ctx, wl, min(steps, ck), probes, targets, ck).backward()
    torch.cuda.synchronize(dev)
    sc = t64(s_init).requires_grad_(True)
    ka = t64([k0, a0]).requires_grad_(True)
    t0 = time.perf_counter()
    L = TrajectoryLoss.apply(sc, ka, ctx, wl, steps, probes, targets, ck)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    L.backward()
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    gs, gka = sc.grad.cpu().numpy(), ka.grad.cpu().numpy()
    # finite differences with the forward's active sets replayed
    _set_params(ctx, wl, t64(s_init), k0, a0)
    v0, w0 = t64(wl.v0), t64(wl.w0)
    tapes = []
    v, w = v0.clone(), w0.clone()
    for n in range(steps):
        tp = ctx.new_tape(wl.sweeps, dev)
        ctx.step_taped(v, w, n * wl.dt, wl.dt, wl.sweeps, wl.tol, tp)
        tapes.append(tp)
    rng = np.random.default_rng(SEED_FD)
    errs = []
    h = 1e-5 * float(np.linalg.norm(s_init))
    tf0 = time.perf_counter()
    for _ in range(args.fd_directions):
        d = rng.standard_normal(wl.n)
        d /= np.linalg.norm(d)
        lp, lm = [], []
        for sgn, out in ((1, lp), (-1, lm)):
            _set_params(ctx, wl, t64(s_init + sgn * h * d), k0, a0)
            out.append(replayed_loss(ctx, wl, v0, w0, steps, probes, targets, tapes))
        fd = (lp[0] - lm[0]) / (2 * h)
        ad = float(gs @ d)
        errs.append(abs(fd - ad) / max(abs(fd), abs(ad), 1e-300))
    tf1 = time.perf_counter()
    del tapes
    line = {"metric": "adjoint gradient evaluations/s, W4 slab 101x36x16 (200 steps)",
            "value": 1.0 / (t2 - t0), "unit": "gradients/s", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * (t2 - t0) / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "n_dofs": wl.n, "M": wl.M, "dt_ms": wl.dt,
                       "sweeps": wl.sweeps, "TOL": wl.tol, "checkpoint_every": ck,
                       "probes": int(probes.numel()), "cg_rtol": 1e-12},
            "loss": L.item(), "forward_s": t1 - t0, "backward_s": t2 - t1,
            "grad_norm_scale": float(np.linalg.norm(gs)), "grad_k_a": gka.tolist(),
            "fd_check": {"directions": args.fd_directions, "step": h,
                         "max_rel_err": max(errs) if errs else None,
                         "median_rel_err": float(np.median(errs)) if errs else None,
                         "masks": "replayed from the forward", "seconds": tf1 - tf0}}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


SEED_FD = 2311_07206 + 40


def main():
    args = parse()
    if args.impl == "reference" and args.workload in ("w2", "w3", "w4", "sweet", "sweet_emi",
                                                      "order"):
        print(json.dumps({"impl": "reference", "unavailable":
                          "the reference arm times the oracle on the monodomain workloads only"}))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "w3":
        return run_batch(args)
    if args.workload == "w4":
        return run_grad(args)
    if args.workload in ("sweet", "sweet_emi"):
        return run_sweet(args)
    if args.workload == "order":
        return run_order(args)
    if args.workload == "w2":
        return run_emi(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
