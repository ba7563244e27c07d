"""Benchmark: elements bisected per second of full recursive spectral bisection.

Default workload: the 64x64x32 box hex mesh (131,072 elements), face-adjacency
dual graph with unit weights, bisected to 64 parts (6 levels) by Lanczos in
mixed precision (FP32 vectors, FP64 coefficients / tridiagonal / Rayleigh
quotient), every level's subgraphs batched in one set of launches; the tile
rows and the launch mode (3: one persistent cooperative kernel per solve with
the basis in shared memory when the level fits; 1: one CUDA graph per cycle)
are picked by rsb_autotune before the timed region (--launch fixes the mode
instead).  A step is one full rsb_partition call from device-resident CSR to
part ids.  metric = (sum over levels and split segments of their element
count) / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs the same workload on its own GPU (independent
replicas, no collective on the data path); the value is all ranks' elements
bisected divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
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
    "c2": {"dims": (64, 64, 32), "adjacency": "face", "parts": 64, "method": "lanczos",
           "degenerate": "resolve"},
    "c1": {"dims": (16, 8, 4), "adjacency": "face", "parts": 8, "method": "lanczos",
           "degenerate": "resolve"},
}
# bounded sample for the CPU oracle: one level-3 segment of the 64x64x32
# recursion (a 32x32x16 box) bisected to 8 parts, i.e. levels 3-5 of the same
# workload
CPU_SAMPLE = {"dims": (32, 32, 16), "parts": 8}


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


# ----------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------
_ORACLE_CHILD = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import oracle as O
from meshgen import box_graph
g = box_graph(*{dims!r})
t = time.perf_counter()
part = O.rsb_partition(g, {parts})
dt = time.perf_counter() - t
ok = bool((part == O.box_partition_closed_form(*{dims!r}, {parts})).all())
levels = ({parts} - 1).bit_length()
print(json.dumps({{"seconds": dt, "elements_bisected": g.n * levels, "ok": ok}}))
"""


def run_oracle_sample(dims, parts, threads=1):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    code = _ORACLE_CHILD.format(root=ROOT, dims=tuple(dims), parts=parts)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        raise RuntimeError(p.stderr[-2000:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def reference_arm(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    d, P = CPU_SAMPLE["dims"], CPU_SAMPLE["parts"]
    for _ in range(args.warmup):
        run_oracle_sample(d, P)
    times, units = [], 0
    ok = True
    for _ in range(args.steps):
        r = run_oracle_sample(d, P)
        times.append(r["seconds"])
        units += r["elements_bisected"]
        ok = ok and r["ok"]
    total = sum(times)
    value = units / total
    sample = (f"oracle on one {d[0]}x{d[1]}x{d[2]} level-3 segment of the 64x64x32 recursion, "
              f"bisected to {P} parts (levels 3-5; {units // args.steps} elements bisected per step)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "sample": sample, "matches_closed_form": ok},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


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
# our arm
# ----------------------------------------------------------------------------
LAUNCH_NAMES = ["kernels", "cuda_graph", "persistent_cycle", "persistent_resident"]
KERNEL_NAMES = {
    ("cycle", 3): ("k_lz_res (one cooperative launch per Fiedler solve: SpMV, CGS2 against the "
                   "shared-memory-resident basis, Jacobi Ritz pairs, thick restart; FP32 stage "
                   "and FP64 polish)"),
    ("cycle", 2): "k_lz_cycle (one cooperative launch per Lanczos cycle)",
}
WORKLOAD_NAME = ("box 64x64x32 hex mesh, face-adjacency dual graph, unit weights, "
                 "131072 elements -> 64 parts (6 levels)")


def our_arm(args):
    import numpy as np
    import torch

    import paper_2606_14659_gb300 as R
    from meshgen import box_graph

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS[args.workload]
    g = box_graph(*W["dims"], W["adjacency"])
    P = W["parts"]
    G = R.graph(g, device=f"cuda:{local}")
    opts = R.options(method=W["method"], precision=args.precision, degenerate_policy=W["degenerate"],
                     batched=1, use_graph=args.launch if args.launch is not None else 3)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
    out = torch.empty(g.n, dtype=torch.int32, device=f"cuda:{local}")
    tuned = None
    if args.launch is None:  # autotuned tile rows and launch mode (before the timed region)
        opts, tune_ms = R.rsb_autotune([G], [P], opts, outs=[out])
        tuned = {"tile_rows": opts.tile_rows, "launch": LAUNCH_NAMES[opts.use_graph],
                 "candidates_ms": {f"{t}x{LAUNCH_NAMES[l]}": round(v, 3)
                                   for (t, l), v in tune_ms.items()}}

    def step():
        return R.rsb_partition(G, P, opts, out=out, allow_noconv=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # timed region: device-resident inputs, L2 flushed between steps
    fam = args.profile if args.profile != "auto" else ("cycle" if opts.use_graph in (2, 3)
                                                        else "lz_b")
    clocks = Clocks(local)
    ms_steps, units, launches = [], 0, 0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, st, code = step()
        e1.record()
        e1.synchronize()
        ms_steps.append(e0.elapsed_time(e1))
        units += st["elements_bisected"]
        launches += st["kernel_launches"]
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    # the same steps again with the dominant kernel family bracketed by CUDA
    # events (kept out of the headline timing: the event records add time)
    prof_ms_steps = []
    R.rsb_profile_begin(fam)
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        prof_ms_steps.append(e0.elapsed_time(e1))
    prof_ms, prof_launches, prof_bytes = R.rsb_profile_end()
    total_ms, units_all = aggregate(sum(ms_steps), units, dist, f"cuda:{local}")
    value = units_all / (total_ms / 1e3)
    # correctness of what was timed (outside the timed region)
    from oracle import box_partition_closed_form  # noqa: WPS433  (check only)

    ok = bool(np.array_equal(out.cpu().numpy(), box_partition_closed_form(*W["dims"], P)))

    # end to end through the public API with pinned host buffers
    Gh = R.Graph(g.n, torch.from_numpy(np.ascontiguousarray(g.row_ptr)).pin_memory(),
                 torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).pin_memory(),
                 torch.from_numpy(np.ascontiguousarray(g.w, dtype=np.int32)).pin_memory(),
                 torch.from_numpy(np.ascontiguousarray(g.gid)).pin_memory(), "host")
    out_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
    h2d = 8 * (g.n + 1) + 4 * g.nnz + 4 * g.nnz + 8 * g.n
    d2h = 4 * g.n
    R.rsb_partition(Gh, P, opts, out=out_h)
    e2e_ms = []
    e2e_units = 0
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st, _ = R.rsb_partition(Gh, P, opts, out=out_h)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_units += st["elements_bisected"]
    e2e_val = e2e_units / (sum(e2e_ms) / 1e3) * (ws if ws > 1 else 1)

    extra = {}
    if rank == 0 and not args.quick:
        # FP64 forms of the same workload (the mixed batched form must beat them)
        for name, kw in (("fp64_batched", dict(precision="fp64", batched=1)),
                         ("fp64_plain", dict(precision="fp64", batched=0))):
            o2 = R.options(method=W["method"], degenerate_policy=W["degenerate"],
                           use_graph=opts.use_graph, tile_rows=opts.tile_rows, **kw)
            R.rsb_partition(G, P, o2, out=out)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            flush.zero_()
            e0.record()
            _, st2, _ = R.rsb_partition(G, P, o2, out=out)
            e1.record()
            e1.synchronize()
            extra[name] = st2["elements_bisected"] / (e0.elapsed_time(e1) / 1e3)
        # Laplacian action bandwidth on a graph larger than L2
        gs = box_graph(192, 128, 96, "vertex")
        Gs = R.graph(gs, device=f"cuda:{local}")
        sp = {}
        for f32 in (True, False):
            ms, by = R.rsb_laplacian_bench(Gs, f32, 20)
            sp["f32_gbs" if f32 else "f64_gbs"] = by / (ms * 1e6)
        sp["graph"] = "192x128x96 vertex adjacency, 4/2/1 weights, %d nnz" % gs.nnz
        extra["spmv"] = sp
        del Gs

    peak, peak_kind = _peaks()
    achieved = (prof_bytes / (prof_ms * 1e6)) if prof_ms > 0 else 0.0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "method": W["method"], "precision": args.precision,
                   "batched": True, "launch": LAUNCH_NAMES[opts.use_graph],
                   "tile_rows": opts.tile_rows, "autotune": tuned, "elements": g.n, "parts": P,
                   "l2": "flushed between steps (256 MiB write)", "matches_closed_form": ok},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm",
                     "kernel": KERNEL_NAMES.get((fam, opts.use_graph),
                                                f"lanczos kernel family '{fam}'"),
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None, "traffic": None,
                     "peak_kind": peak_kind, "launches_timed": prof_launches,
                     "avg_launch_us": 1e3 * prof_ms / prof_launches if prof_launches else None,
                     "share_of_step": prof_ms / sum(prof_ms_steps) if prof_ms_steps else None,
                     "timed_in": "profiled repeat of the timed steps (same workload and options)"},
        "clocks": clk,
    }
    line.update(extra)
    if rank == 0 and not args.quick:
        try:
            d, Pc = CPU_SAMPLE["dims"], CPU_SAMPLE["parts"]
            r = run_oracle_sample(d, Pc)
            line["cpu_baseline"] = {
                "value": r["elements_bisected"] / r["seconds"], "unit": UNIT, "cores": 1,
                "kind": "oracle",
                "sample": (f"oracle on one {d[0]}x{d[1]}x{d[2]} level-3 segment of the 64x64x32 "
                           f"recursion bisected to {Pc} parts ({r['elements_bisected']} "
                           f"elements bisected, {r['seconds']:.1f} s)")}
        except Exception as e:  # pragma: no cover
            line["cpu_baseline"] = {"error": str(e)[-300:]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--profile", default="auto",
                    choices=["auto", "cycle", "lz_a", "lz_b", "lz_c", "cg_ap"])
    ap.add_argument("--launch", type=int, default=None, choices=[0, 1, 2, 3],
                    help="fix the Lanczos launch mode (0 kernels, 1 CUDA graph per cycle, "
                         "2 persistent kernel per cycle, 3 resident persistent kernel per "
                         "solve) instead of autotuning it with the tile rows")
    ap.add_argument("--quick", action="store_true", help="skip the FP64/SpMV/CPU extras")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
