"""Elements bisected per second on the five workload shapes, mixed and FP64.

    python -m paper_2606_14659_gb300.bench_configs [--configs c1 c3 c4 c5] [--forms mixed fp64]

c1: 16x8x4 face box -> 8 parts, Lanczos.
c3: 192x128x96 box, 10% seeded deletion, largest component, vertex adjacency
    (4/2/1), inverse iteration with CG -> 256 parts (mixed: 8 FP64 polish
    cycles, as in the tests).
c4: 512 boxes with sides drawn from [8, 96], face adjacency, 16 parts each,
    one batched call.
c5: 256^3 box, 5% seeded deletion, vertex adjacency, Lanczos -> 1024 parts
    (mixed: 8 FP64 polish cycles).
Each form is timed once with CUDA events after a one-level warm-up of the same
inputs (so the workspace is already allocated); inputs are device-resident.
One JSON line per (config, form).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _workloads(which):
    from meshgen import batch_box_dims, box_graph, box_graph_deleted

    if which == "c1":
        return [box_graph(16, 8, 4)], 8, dict(method="lanczos")
    if which == "c3":
        return ([box_graph_deleted(192, 128, 96, 0.10, 20260, "vertex")], 256,
                dict(method="inverse", degenerate_policy="none", polish_cycles=8))
    if which == "c4":
        return [box_graph(*d) for d in batch_box_dims(512, 8, 96, 2026)], 16, dict(method="lanczos")
    if which == "c5":
        return ([box_graph_deleted(256, 256, 256, 0.05, 20261, "vertex")], 1024,
                dict(method="lanczos", degenerate_policy="none", polish_cycles=8))
    raise ValueError(which)


def main(argv=None):
    import torch

    import paper_2606_14659_gb300 as R

    ap = argparse.ArgumentParser()
    ap.add_argument("--configs", nargs="+", default=["c1", "c3", "c4", "c5"])
    ap.add_argument("--forms", nargs="+", default=["mixed", "fp64"])
    a = ap.parse_args(argv)
    for cfg in a.configs:
        t0 = time.perf_counter()
        gs, P, kw = _workloads(cfg)
        G = [R.graph(g) for g in gs]
        gen_s = time.perf_counter() - t0
        for form in a.forms:
            kw2 = dict(kw)
            if form == "fp64":
                kw2.pop("polish_cycles", None)
            o = R.options(precision=form, **kw2)
            R.rsb_partition_batch(G, [min(P, 2)] * len(G), o)  # workspace warm-up
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st, code = R.rsb_partition_batch(G, [P] * len(G), o)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            print(json.dumps({
                "config": cfg, "form": form, "meshes": len(G), "elements": sum(g.n for g in gs),
                "parts": P, "ms": round(ms, 2),
                "elements_bisected_per_s": st["elements_bisected"] / (ms / 1e3),
                "levels": st["levels"], "solves": st["solves"], "cycles": st["cycles"],
                "resid_max": st["resid_max"], "code": code, "input_build_s": round(gen_s, 1)}),
                flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
