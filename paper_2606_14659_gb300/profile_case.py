"""Small, fixed workloads for kernel profiling (ncu) of librsb.

    python -m paper_2606_14659_gb300.profile_case lanczos --dims 192 128 96 --cycles 2
    python -m paper_2606_14659_gb300.profile_case spmv --dims 192 128 96 --adjacency vertex
    python -m paper_2606_14659_gb300.profile_case partition --dims 64 64 32 --parts 64

`lanczos` runs one Fiedler solve capped at --cycles Lanczos cycles (vectors of
the 192x128x96 face box exceed L2, so DRAM counters mean something); `spmv`
applies the Laplacian --reps times; `partition` runs one rsb_partition.  Each
prints one line of what it ran.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import torch

    import paper_2606_14659_gb300 as R
    from meshgen import box_graph

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["lanczos", "spmv", "partition"])
    ap.add_argument("--dims", type=int, nargs=3, default=[192, 128, 96])
    ap.add_argument("--adjacency", default="face", choices=["face", "vertex"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cycles", type=int, default=2)
    ap.add_argument("--parts", type=int, default=64)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--launch", type=int, default=1)
    a = ap.parse_args(argv)
    g = box_graph(*a.dims, a.adjacency)
    G = R.graph(g)
    if a.case == "lanczos":
        o = R.options(precision=a.precision, max_restarts=a.cycles, tol=1e-14, mixed_tol=1e-14,
                      use_graph=a.launch)
        lam, v, res, code = R.rsb_fiedler(G, o)
        torch.cuda.synchronize()
        print(f"lanczos {a.dims} {a.precision}: {a.cycles} cycles, lambda {lam:.6e}, resid {res:.2e}")
    elif a.case == "spmv":
        f32 = a.precision == "mixed"
        ms, by = R.rsb_laplacian_bench(G, f32, a.reps)
        print(f"spmv {a.dims} {a.adjacency} {'f32' if f32 else 'f64'}: {ms:.4f} ms, "
              f"{by / ms / 1e6:.0f} GB/s")
    else:
        part, st, code = R.rsb_partition(G, a.parts, R.options(precision=a.precision,
                                                               use_graph=a.launch))
        torch.cuda.synchronize()
        print(f"partition {a.dims} -> {a.parts}: {st['levels']} levels, "
              f"{st['kernel_launches']} launches, code {code}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
