"""Benchmark: elements bisected per second of full recursive spectral bisection.

Default workload (the largest single-GPU configuration): the 256^3 box hex mesh
with a seeded 5 % of its elements deleted (largest connected component kept,
15,938,356 elements), vertex-adjacency dual graph with weights 4/2/1 shared
vertices (26 neighbours), bisected to 1024 parts (10 levels) by Lanczos in mixed
precision (FP32 vectors and SpMV, FP64 Gram-Schmidt coefficients, projected
matrix, Rayleigh quotient and polish); every level's subgraphs are batched in
one set of launches, the tile rows and launch mode picked by rsb_autotune before
the timed region.  A step is one full rsb_partition call from device-resident
CSR to part ids.  metric = (sum over levels and split segments of their element
count) / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload c1|c2|c3|c4|c5] [--precision mixed|fp64]
                    [--forms fp64 fp64_plain spmv cpu]
    python bench.py --case lanczos|spmv|partition ...   (small fixed cases for ncu)

Other workloads: c1 16x8x4 face box -> 8 parts; c2 64x64x32 face box -> 64;
c3 192x128x96 box, 10 % deleted, vertex adjacency, inverse iteration -> 256;
c4 512 face boxes with sides drawn from [8, 96], 16 parts each in one batched
call.  Under torchrun each rank runs the same workload on its own GPU
(independent replicas, no collective on the data path); the value is all
ranks' elements bisected divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "elements bisected/s (full RSB to P parts)"
UNIT = "elements/s"

WORKLOADS = {
    "c1": {"kind": "box", "dims": (16, 8, 4), "adjacency": "face", "parts": 8,
           "opts": {"method": "lanczos", "degenerate_policy": "resolve"},
           "name": "box 16x8x4 hex mesh, face-adjacency dual graph, unit weights, 512 elements "
                   "-> 8 parts (3 levels)"},
    "c2": {"kind": "box", "dims": (64, 64, 32), "adjacency": "face", "parts": 64,
           "opts": {"method": "lanczos", "degenerate_policy": "resolve"},
           "name": "box 64x64x32 hex mesh, face-adjacency dual graph, unit weights, 131072 "
                   "elements -> 64 parts (6 levels)"},
    "c3": {"kind": "deleted", "dims": (192, 128, 96), "frac": 0.10, "seed": 20260,
           "adjacency": "vertex", "parts": 256,
           "opts": {"method": "inverse", "degenerate_policy": "none", "polish_cycles": 8},
           "name": "box 192x128x96 hex mesh with a seeded 10% of elements deleted (largest "
                   "component, 2123367 elements), vertex-adjacency dual graph, weights 4/2/1, "
                   "inverse iteration with CG -> 256 parts (8 levels)"},
    "c4": {"kind": "batch", "count": 512, "lo": 8, "hi": 96, "seed": 2026, "adjacency": "face",
           "parts": 16, "opts": {"method": "lanczos", "degenerate_policy": "resolve"},
           "name": "batch of 512 box hex meshes with sides drawn from [8, 96], face adjacency, "
                   "unit weights, 16 parts each (4 levels), one batched call"},
    "c5": {"kind": "deleted", "dims": (256, 256, 256), "frac": 0.05, "seed": 20261,
           "adjacency": "vertex", "parts": 1024,
           "opts": {"method": "lanczos", "degenerate_policy": "none"},
           "name": "box 256x256x256 hex mesh with a seeded 5% of elements deleted (largest "
                   "component, 15938356 elements), vertex-adjacency dual graph, weights 4/2/1, "
                   "mixed-precision Lanczos -> 1024 parts (10 levels)"},
}
DEFAULT_FORMS = {"c1": ["fp64", "fp64_plain", "spmv", "cpu"],
                 "c2": ["fp64", "fp64_plain", "spmv", "cpu"],
                 "c3": ["fp64", "spmv", "cpu"], "c4": ["fp64", "cpu"],
                 "c5": ["fp64", "spmv", "cpu", "frows"]}
# bounded samples for the CPU oracle: meshes of the same kind as the workload
# (same generator, adjacency, weights and deletion fraction), small enough for
# a few to a few tens of seconds of host time
CPU_SAMPLES = {
    "c5": {"dims": (32, 32, 32), "frac": 0.05, "seed": 20261, "adjacency": "vertex", "parts": 8,
           "ref_dims": (32, 32, 16), "ref_parts": 2,
           "opts": {"method": "lanczos", "degenerate": "none"}},
    "c3": {"dims": (48, 32, 24), "frac": 0.10, "seed": 20260, "adjacency": "vertex", "parts": 8,
           "ref_dims": (24, 16, 12), "ref_parts": 2,
           "opts": {"method": "inverse", "degenerate": "none"}},
    "c2": {"dims": (32, 32, 16), "frac": 0.0, "adjacency": "face", "parts": 8, "ref_parts": 8,
           "opts": {"method": "lanczos", "degenerate": "resolve"}},
    "c1": {"dims": (16, 8, 4), "frac": 0.0, "adjacency": "face", "parts": 8, "ref_parts": 8,
           "opts": {"method": "lanczos", "degenerate": "resolve"}},
    "c4": {"dims": (24, 20, 16), "frac": 0.0, "adjacency": "face", "parts": 16, "ref_parts": 16,
           "opts": {"method": "lanczos", "degenerate": "resolve"}},
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        m = re.search(r"Model name:\s*(.+)", out)
        if m:
            return m.group(1).strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def build_graphs(W):
    """The workload's meshes (meshgen's seeded generators)."""
    from meshgen import batch_box_dims, box_graph, box_graph_deleted

    if W["kind"] == "box":
        return [box_graph(*W["dims"], W["adjacency"])]
    if W["kind"] == "deleted":
        return [box_graph_deleted(*W["dims"], W["frac"], W["seed"], W["adjacency"])]
    return [box_graph(*d, W["adjacency"]) for d in batch_box_dims(W["count"], W["lo"], W["hi"],
                                                                   W["seed"])]


# ----------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline), run in a child process with its
# BLAS threads set to the host's cores
# ----------------------------------------------------------------------------
_ORACLE_CHILD = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import oracle as O
from meshgen import box_graph, box_graph_deleted
S = {sample!r}
if S["frac"] > 0:
    g = box_graph_deleted(*S["dims"], S["frac"], S["seed"], S["adjacency"])
else:
    g = box_graph(*S["dims"], S["adjacency"])
P = {parts}
times = []
for _ in range({reps}):
    t = time.perf_counter()
    part = O.rsb_partition(g, P, O.Options(**S["opts"]))
    times.append(time.perf_counter() - t)
levels = (P - 1).bit_length()
print(json.dumps({{"seconds": times, "elements_bisected": g.n * levels, "n": g.n}}))
"""


def run_oracle_sample(sample, parts, threads, reps=1):
    """Times `reps` oracle partitions of the sample in one child process; returns
    {"seconds": [per rep], "elements_bisected": per rep, "n": elements}."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    code = _ORACLE_CHILD.format(root=ROOT, sample=sample, parts=parts, reps=reps)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        raise RuntimeError(p.stderr[-2000:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def _sample_text(S, parts, n):
    kind = f"{int(S['frac'] * 100)}%-deleted " if S["frac"] > 0 else ""
    return (f"FP64 oracle on a {kind}{S['dims'][0]}x{S['dims'][1]}x{S['dims'][2]} "
            f"{S['adjacency']}-adjacency box of the workload's kind ({n} elements) bisected "
            f"to {parts} parts, {S['opts']['method']}")


def reference_arm(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    S = dict(CPU_SAMPLES[args.workload])
    S["dims"] = S.get("ref_dims", S["dims"])
    P = S["ref_parts"]
    threads = os.cpu_count() or 1
    r = run_oracle_sample(S, P, threads, reps=args.warmup + args.steps)
    times = r["seconds"][args.warmup:]
    units = r["elements_bisected"] * args.steps
    n = r["n"]
    total = sum(times)
    value = units / total
    sample = _sample_text(S, P, n) + f"; host: {_cpu_model()}, {threads} cores"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["name"], "sample": sample},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu_model": _cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
                power.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_median": statistics.median(power) if power else None}


# ----------------------------------------------------------------------------
# multi-rank aggregation: independent replicas, one number for the job
# ----------------------------------------------------------------------------
def aggregate(total_ms: float, units: float, dist=None, device=None):
    """(slowest rank's time in ms, units of all ranks).

    Weak scaling: every rank runs the same workload on its own GPU; the job's
    throughput is all ranks' units over the slowest rank's time.
    """
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(total_ms), float(units)
    import torch

    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ----------------------------------------------------------------------------
# roofline of the dominant kernel family
# ----------------------------------------------------------------------------
LAUNCH_NAMES = ["kernels", "cuda_graph", "persistent_cycle", "persistent_resident"]
FAMILIES = {
    "lz_a": "k_lz_a1 (FP32 Lanczos step D1: SpMV z = L v_j of the sliced-ELL graph, v_j = w_j / nu_j)",
    "lz_a2": ("k_lz_d2 (FP32 Lanczos step D2: dots of v_j and z with the basis in one pass, the "
              "basis, v_j and z staged in shared memory by bulk copies)"),
    "lz_b": ("k_lz_d3 (FP32 Lanczos step D3: q_j = (v_j - B a) / rho and w_{j+1} = (z - B g - "
             "(q_j.z) q_j) / rho in one pass over the basis, ||w_{j+1}||)"),
    "lz_c": "k_lz_c (FP64 Lanczos step C: w -= Q c2 and ||w||)",
    "cg_ap": "k_cg_ap (CG: Ap = L p and p.Ap)",
    "cycle": ("k_lz_res (one cooperative launch per Fiedler solve: SpMV, CGS2 against the "
              "shared-memory-resident basis, Jacobi Ritz pairs, thick restart)"),
}
PROFILE_KERNEL = {"lz_a": "k_lz_a1", "lz_a2": "k_lz_d2", "lz_b": "k_lz_d3", "lz_c": "k_lz_c",
                  "cg_ap": "k_cg_ap", "cycle": "k_lz_res"}


def _source_sha():
    h = hashlib.sha256()
    for f in ("solver.cu", "rsb_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2606_14659_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_ratio(kernel, workload):
    """DRAM bytes / algorithmic bytes of `kernel` from a committed ncu summary
    (profiles/<kernel>_*_<workload>*.md with lines 'dram_over_algorithmic = x'
    and 'solver_sha = s'); None when absent or when the kernel sources changed
    since the capture."""
    pdir = os.path.join(ROOT, "profiles")
    try:
        files = sorted(os.listdir(pdir))
    except OSError:
        return None
    for fn in files:
        if not (fn.startswith(kernel + "_") and workload in fn and fn.endswith(".md")):
            continue
        txt = open(os.path.join(pdir, fn)).read()
        m = re.search(r"dram_over_algorithmic\s*=\s*([0-9.eE+-]+)", txt)
        s = re.search(r"solver_sha\s*=\s*([0-9a-f]+)", txt)
        if m and s and s.group(1) == _source_sha():
            return float(m.group(1))
    return None


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def our_arm(args):
    import numpy as np
    import torch

    import paper_2606_14659_gb300 as R

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS[args.workload]
    forms = args.forms if args.forms is not None else DEFAULT_FORMS[args.workload]
    t_gen = time.perf_counter()
    gs = build_graphs(W)
    gen_s = time.perf_counter() - t_gen
    P = W["parts"]
    Gs = [R.graph(g, device=dev) for g in gs]
    n_total = sum(g.n for g in gs)
    opts = R.options(precision=args.precision, batched=1,
                     use_graph=args.launch if args.launch is not None else 3,
                     tile_rows=args.tile_rows, **W["opts"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    outs = [torch.empty(g.n, dtype=torch.int32, device=dev) for g in gs]
    tuned = None
    if args.launch is None:  # autotuned tile rows and launch mode (before the timed region)
        opts, tune_ms = R.rsb_autotune(Gs, [P] * len(Gs), opts, outs=outs)
        tuned = {"tile_rows": opts.tile_rows, "launch": LAUNCH_NAMES[opts.use_graph],
                 "candidates_ms": {f"{t}x{LAUNCH_NAMES[l]}": round(v, 3)
                                   for (t, l), v in tune_ms.items()}}

    def step(o=opts, graphs=Gs, out=outs):
        if len(graphs) == 1:
            p, st, code = R.rsb_partition(graphs[0], P, o, out=out[0], allow_noconv=True)
            return [p], st, code
        return R.rsb_partition_batch(graphs, [P] * len(graphs), o, outs=out, allow_noconv=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # timed region: device-resident inputs, L2 flushed between steps
    clocks = Clocks(local)
    ms_steps, units, launches, codes = [], 0, 0, set()
    resid_max = 0.0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_step")  # lets a profiler select the timed steps
        e0.record()
        _, st, code = step()
        e1.record()
        e1.synchronize()
        torch.cuda.nvtx.range_pop()
        ms_steps.append(e0.elapsed_time(e1))
        units += st["elements_bisected"]
        launches += st["kernel_launches"]
        codes.add(code)
        resid_max = max(resid_max, st["resid_max"])
        lam_first = st["lambda_first"]
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    units_per_step = units / max(1, args.steps)
    med = statistics.median(ms_steps)
    total_ms, units_all = aggregate(med * args.steps, units, dist, dev)
    value = units_all / (total_ms / 1e3)

    # one more step with every kernel family bracketed by CUDA events on the
    # library's stream (kept out of the headline timing: the records add time)
    R.rsb_profile_begin("all")
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    step()
    e1.record()
    e1.synchronize()
    prof_step_ms = e0.elapsed_time(e1)
    R.rsb_profile_end()
    fam = {}
    for name in FAMILIES:
        ms, nl, by = R.rsb_profile_read(name)
        if nl:
            fam[name] = {"ms": round(ms, 3), "launches": nl, "gbs": by / (ms * 1e6) if ms else 0.0,
                         "share": ms / prof_step_ms}
    dom = max(fam, key=lambda k: fam[k]["ms"]) if fam else None

    # correctness of what was timed (outside the timed region)
    check = {}
    if W["kind"] in ("box", "batch"):
        from oracle import NotClean, box_partition_closed_form  # noqa: WPS433  (check only)

        clean, equal = 0, 0
        dims_list = [W["dims"]] if W["kind"] == "box" else [
            g.dims for g in gs]
        for d, o in zip(dims_list, outs):
            try:
                cf = box_partition_closed_form(*d, P)
            except NotClean:
                continue
            clean += 1
            equal += int(np.array_equal(o.cpu().numpy(), cf))
        check = {"closed_form_meshes": clean, "closed_form_equal": equal}
    else:
        sizes = np.bincount(outs[0].cpu().numpy(), minlength=P)
        n = gs[0].n
        expect = [(p + 1) * n // P - p * n // P for p in range(P)]
        check = {"sizes_exact": bool(np.array_equal(sizes, expect)),
                 "lambda_first": lam_first, "resid_max_over_dmax": resid_max}
    check["status_codes"] = sorted(codes)

    # end to end through the public API: pinned host CSR in, host part ids out
    Gh, outs_h, h2d, d2h = [], [], 0, 0
    for g in gs:
        rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr, dtype=np.int64)).pin_memory()
        col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).pin_memory()
        w = torch.from_numpy(np.ascontiguousarray(g.w, dtype=np.int32)).pin_memory()
        gid = torch.from_numpy(np.ascontiguousarray(g.gid, dtype=np.int64)).pin_memory()
        Gh.append(R.Graph(g.n, rp, col, w, gid, "host"))
        outs_h.append(torch.empty(g.n, dtype=torch.int32).pin_memory())
        h2d += rp.numel() * 8 + col.numel() * 4 + w.numel() * 4 + gid.numel() * 8
        d2h += g.n * 4
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    e2e_ms, e2e_units = [], 0
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st, _ = step(graphs=Gh, out=outs_h)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_units += st["elements_bisected"]
    e2e_val = e2e_units / (sum(e2e_ms) / 1e3) * (ws if ws > 1 else 1)
    del Gh, outs_h

    extra = {}
    if rank == 0:
        # FP64 forms of the same workload (the mixed batched form must beat them)
        for name, kw in (("fp64_batched", dict(precision="fp64", batched=1)),
                         ("fp64_plain", dict(precision="fp64", batched=0))):
            form = "fp64" if name == "fp64_batched" else "fp64_plain"
            if form not in forms or args.precision == "fp64" and name == "fp64_batched":
                continue
            o2 = R.options(use_graph=opts.use_graph, tile_rows=opts.tile_rows,
                           **{**W["opts"], **{k: v for k, v in kw.items()}})
            torch.cuda.synchronize()
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st2, code2 = step(o=o2)
            e1.record()
            e1.synchronize()
            ms2 = e0.elapsed_time(e1)
            v2 = st2["elements_bisected"] / (ms2 / 1e3)
            extra[name] = {"value": v2, "ms": round(ms2, 1), "status": code2, "steps": 1,
                           "mixed_speedup": (value / max(ws, 1)) / v2 if v2 else None}
        if "spmv" in forms:
            # Laplacian action bandwidth on the workload's level-0 graph (larger than L2)
            sp = {}
            for f32 in (True, False):
                ms, by = R.rsb_laplacian_bench(Gs[0], f32, 20)
                sp["f32_gbs" if f32 else "f64_gbs"] = by / (ms * 1e6)
            sp["graph"] = f"level-0 graph of the workload ({gs[0].n} rows, {gs[0].nnz} nnz)"
            peak, _ = _peaks()
            sp["f32_frac"] = sp["f32_gbs"] / peak
            extra["spmv"] = sp

    if rank == 0 and "frows" in forms:
        extra["next_rows"] = next_rows(R, gs[0], dev, flush)

    peak, peak_kind = _peaks()
    roof = None
    if dom is not None:
        ms, nl, by = R.rsb_profile_read(dom)
        achieved = by / (ms * 1e6) if ms > 0 else 0.0
        ratio = traffic_ratio(PROFILE_KERNEL[dom], args.workload)
        roof = {"bound": "hbm", "kernel": FAMILIES[dom], "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak if peak else None,
                "traffic": (ratio * by / nl) if ratio is not None and nl else None,
                "algorithmic_bytes_per_launch": by / nl if nl else None,
                "peak_kind": peak_kind, "launches_timed": nl,
                "avg_launch_us": 1e3 * ms / nl if nl else None,
                "share_of_step": fam[dom]["share"],
                "timed_in": "one extra profiled step of the same workload and options, every "
                            "kernel family bracketed by CUDA events on the library's stream",
                "families": fam}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": med,
        "ms_per_step_mean": statistics.fmean(ms_steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": W["name"], "key": args.workload, "precision": args.precision,
                   "options": {k: v for k, v in W["opts"].items()},
                   "batched": True, "launch": LAUNCH_NAMES[opts.use_graph],
                   "tile_rows": opts.tile_rows, "autotune": tuned, "elements": n_total,
                   "meshes": len(gs), "parts": P,
                   "elements_bisected_per_step": units_per_step,
                   "l2": "flushed between steps (256 MiB write); inputs larger than L2"
                         if n_total > 4_000_000 else "flushed between steps (256 MiB write)",
                   "value_from": "median step time", "input_build_s": round(gen_s, 1),
                   "check": check},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clk,
    }
    line.update(extra)
    if rank == 0 and "cpu" in forms and not args.quick:
        try:
            S = CPU_SAMPLES[args.workload]
            threads = os.cpu_count() or 1
            r = run_oracle_sample(S, S["parts"], threads)
            sec = r["seconds"][0]
            line["cpu_baseline"] = {
                "value": r["elements_bisected"] / sec, "unit": UNIT, "cores": threads,
                "kind": "oracle", "cpu_model": _cpu_model(),
                "sample": (_sample_text(S, S["parts"], r["n"]) +
                           f"; {r['elements_bisected']} elements bisected in "
                           f"{sec:.1f} s; numpy BLAS on {threads} threads (the sparse "
                           f"product runs on one)")}
        except Exception as e:  # pragma: no cover
            line["cpu_baseline"] = {"error": str(e)[-300:]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------
# the rows beyond the headline path: gather-scatter Laplacian, RCB and the RCB
# reordering, AMG-preconditioned inverse iteration, block Lanczos
# ----------------------------------------------------------------------------
def _timed(torch, fn, flush):
    flush.zero_()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1), out


def next_rows(R, g5, dev, flush):
    import torch

    from meshgen import box_graph_deleted, permute_graph

    out = {}
    peak, _ = _peaks()
    # f4: matrix-free Laplacian from the hex vertex ids of the headline mesh
    ev = torch.from_numpy(g5.hex_vertices()).to(dev)
    gs = {}
    for f32 in (True, False):
        ms, by = R.rsb.rsb_laplacian_bench_gs(ev, f32, 10)
        gs["f32_gbs" if f32 else "f64_gbs"] = by / (ms * 1e6)
        gs["f32_ms" if f32 else "f64_ms"] = ms
    gs["f32_frac"] = gs["f32_gbs"] / peak
    t0 = time.perf_counter()
    n, rp, col, w = R.rsb.rsb_dual_graph(ev)
    torch.cuda.synchronize()
    gs["dual_graph_build_s"] = time.perf_counter() - t0
    gs["dual_graph_nnz"] = int(col.numel())
    out["gather_scatter_c5"] = gs
    del ev, rp, col, w
    # f3: RCB of the headline mesh into 1024 parts
    G5 = R.graph(g5, device=dev)
    o = R.options(method="rcb")
    R.rsb_partition(G5, 1024, o)
    ms, (p, st, code) = _timed(torch, lambda: R.rsb_partition(G5, 1024, o), flush)
    out["rcb_c5_1024"] = {"ms": ms, "elements_bisected_per_s": st["elements_bisected"] / (ms / 1e3)}
    del G5
    # f3 and f2, f1 on the 2.1M-element C3 mesh (first split)
    g3 = box_graph_deleted(192, 128, 96, 0.10, 20260, "vertex")
    h3 = permute_graph(g3, 1)
    G3 = R.graph(g3, device=dev)
    H3 = R.graph(h3, device=dev)
    runs = {
        "c3_lanczos_natural_order": (G3, dict(precision="mixed", degenerate_policy="none")),
        "c3_lanczos_permuted": (H3, dict(precision="mixed", degenerate_policy="none")),
        "c3_lanczos_permuted_rcb_reorder": (H3, dict(precision="mixed", degenerate_policy="none",
                                                     reorder=1)),
        "c3_lanczos_block2": (G3, dict(precision="mixed", degenerate_policy="none", block=2)),
        "c3_inverse_cg": (G3, dict(method="inverse", precision="mixed", degenerate_policy="none",
                                   reorder=1, polish_cycles=8)),
        "c3_inverse_amg_fcg": (G3, dict(method="inverse", amg=1, precision="mixed",
                                        degenerate_policy="none", reorder=1, polish_cycles=8)),
    }
    for name, (G, kw) in runs.items():
        o = R.options(**kw)
        R.rsb_partition(G, 2, o)
        ms, (p, st, code) = _timed(torch, lambda: R.rsb_partition(G, 2, o), flush)
        out[name] = {"ms_first_split": ms, "lambda2": st["lambda_first"], "cycles": st["cycles"],
                     "cg_iterations": st["inner"], "status": code}
    return out


# ----------------------------------------------------------------------------
# small fixed cases for ncu captures
# ----------------------------------------------------------------------------
def case_main(args):
    import torch

    import paper_2606_14659_gb300 as R
    from meshgen import box_graph, box_graph_deleted

    if args.frac > 0:
        g = box_graph_deleted(*args.dims, args.frac, args.seed, args.adjacency)
    else:
        g = box_graph(*args.dims, args.adjacency)
    G = R.graph(g)
    if args.case == "lanczos":
        o = R.options(precision=args.precision, max_restarts=args.cycles, tol=1e-14,
                      mixed_tol=1e-14, use_graph=args.launch if args.launch is not None else 1,
                      polish_cycles=0)
        lam, v, res, code = R.rsb_fiedler(G, o)
        torch.cuda.synchronize()
        print(f"lanczos {args.dims} {args.adjacency} {args.precision}: {args.cycles} cycles, "
              f"lambda {lam:.6e}, resid {res:.2e}")
    elif args.case == "spmv":
        f32 = args.precision == "mixed"
        ms, by = R.rsb_laplacian_bench(G, f32, args.reps)
        print(f"spmv {args.dims} {args.adjacency} {'f32' if f32 else 'f64'}: {ms:.4f} ms, "
              f"{by / ms / 1e6:.0f} GB/s")
    else:
        # the headline's options on a smaller mesh: one warm run, one run inside
        # the NVTX range "case_step" (what a launch list selects), then one run
        # with every kernel family timed, whose shares the launch list should
        # reproduce
        o = R.options(precision=args.precision, method="lanczos", degenerate_policy="none",
                      use_graph=args.launch if args.launch is not None else 1)
        R.rsb_partition(G, args.parts, o)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("case_step")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        part, st, code = R.rsb_partition(G, args.parts, o)
        e1.record()
        e1.synchronize()
        torch.cuda.nvtx.range_pop()
        print(f"partition {args.dims} -> {args.parts}: {st['levels']} levels, "
              f"{st['kernel_launches']} launches, {e0.elapsed_time(e1):.1f} ms, code {code}")
        R.rsb_profile_begin("all")
        e0.record()
        R.rsb_partition(G, args.parts, o)
        e1.record()
        e1.synchronize()
        R.rsb_profile_end()
        step_ms = e0.elapsed_time(e1)
        for name in FAMILIES:
            ms, nl, by = R.rsb_profile_read(name)
            if nl:
                print(f"  family {name}: {nl} launches, {ms:.2f} ms, share {ms / step_ms:.3f}, "
                      f"{by / (ms * 1e6):.0f} GB/s")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--forms", nargs="*", default=None,
                    help="extras beside the headline: fp64 (FP64 batched), fp64_plain (FP64, one "
                         "segment at a time), spmv (Laplacian bandwidth), cpu (oracle baseline)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--launch", type=int, default=None, choices=[0, 1, 2, 3],
                    help="fix the Lanczos launch mode (0 kernels, 1 CUDA graph per cycle, "
                         "2 persistent kernel per cycle, 3 resident persistent kernel per "
                         "solve) instead of autotuning it with the tile rows")
    ap.add_argument("--tile-rows", type=int, default=0,
                    help="minimum rows per thread of a tile when --launch fixes the launch mode "
                         "(0: the library's default)")
    ap.add_argument("--quick", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--case", choices=["lanczos", "spmv", "partition"], default=None,
                    help="run one small fixed case (for ncu) instead of the benchmark")
    ap.add_argument("--dims", type=int, nargs=3, default=[192, 128, 96])
    ap.add_argument("--adjacency", default="face", choices=["face", "vertex"])
    ap.add_argument("--frac", type=float, default=0.0)
    ap.add_argument("--seed", type=int, default=20261)
    ap.add_argument("--cycles", type=int, default=2)
    ap.add_argument("--parts", type=int, default=64)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    if args.case:
        return case_main(args)
    if args.impl == "reference":
        return reference_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
