"""Writes the stored expected values of the irregular-mesh parity tests.

Every value comes from the FP64 oracle (``oracle/``) on inputs from the seeded
generators (``meshgen/``); nothing here touches the CUDA library.

    python tests/golden/make_golden.py medium      # irregular_medium.json (about 2 min)
    python tests/golden/make_golden.py c3          # c3_levels01.json (about an hour)
    python tests/golden/make_golden.py c5          # c5_level0.json (hours)

medium: two 26-neighbour meshes with a seeded 10 % deletion (vertex adjacency,
weights 4/2/1 shared vertices, §2), partitioned into 16 parts by both Fiedler
solvers (§6 Lanczos, §7 inverse iteration) under both degeneracy policies; the
first split's lambda_2, residual, weighted cut and cluster size, lambda_3 (a
solve deflated against the Fiedler vector, for the Davis-Kahan bound on the
vector error), the oriented Fiedler vector at 64 sampled rows, and the quality
metrics of the 16-part partition (§8).
c3: the 192x128x96 mesh with 10 % deleted, first two bisection levels by inverse
iteration (its configured solver): lambda_2, residual and cut of each split and
the weighted cut of the 2- and 4-part partitions.
c5: the 256^3 mesh with 5 % deleted, first split by Lanczos.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from meshgen import box_graph_deleted  # noqa: E402

MEDIUM = [
    # (nx, ny, nz, deleted fraction, seed): a simple lambda_2 (longest axis 40)
    (40, 32, 24, 0.10, 20262),
    # x and y of equal length: lambda_2 and lambda_3 nearly repeated, so the
    # degeneracy policy decides the first split
    (32, 32, 20, 0.10, 20263),
]
SAMPLES = 64


def _sample_rows(n: int) -> list[int]:
    return sorted(set(int(r) for r in np.linspace(0, n - 1, SAMPLES)))


def medium() -> dict:
    out = {"source": "tests/golden/make_golden.py medium (FP64 oracle)", "meshes": []}
    for (nx, ny, nz, frac, seed) in MEDIUM:
        g = box_graph_deleted(nx, ny, nz, frac, seed, "vertex")
        dmax = float(O.degree(g).max())
        opts = O.Options(method="lanczos")
        lam, v, r = O.fiedler_of_graph(g, opts)
        r3 = O.fiedler(g, opts, deflate=[r.v])
        rows = _sample_rows(g.n)
        mesh = {"dims": [nx, ny, nz], "frac": frac, "seed": seed, "adjacency": "vertex",
                "n": g.n, "nnz": g.nnz, "dmax": dmax, "lambda2": lam, "resid": r.resid,
                "lambda3": r3.lam, "sample_rows": rows,
                "v_samples": [float(v[i]) for i in rows], "parts": 16, "runs": {}}
        for method in ("lanczos", "inverse"):
            for policy in ("none", "resolve"):
                t = time.perf_counter()
                rec = []
                part = O.rsb_partition(g, 16, O.Options(method=method, degenerate=policy),
                                       record=rec)
                m = O.partition_metrics(g, part, 16)
                first = rec[0]
                part2 = O.rsb_partition(g, 2, O.Options(method=method, degenerate=policy))
                mesh["runs"][f"{method}/{policy}"] = {
                    "lambda2_first": first["lam"], "resid_first": first["resid"],
                    "cluster_first": first["cluster"],
                    "cut_2": O.partition_metrics(g, part2, 2)["weighted_cut"],
                    "weighted_cut_16": m["weighted_cut"], "edge_cut_16": m["edge_cut"],
                    "max_neighbours_16": m["max_neighbours"],
                    "avg_neighbours_16": m["avg_neighbours"],
                    "all_converged": bool(all(x["resid"] <= 1e-10 * dmax for x in rec)),
                    "seconds": round(time.perf_counter() - t, 1)}
                print(nx, ny, nz, method, policy, mesh["runs"][f"{method}/{policy}"], flush=True)
        out["meshes"].append(mesh)
    return out


def c3() -> dict:
    g = box_graph_deleted(192, 128, 96, 0.10, 20260, "vertex")
    dmax = float(O.degree(g).max())
    opts = O.Options(method="inverse", degenerate="none")
    t = time.perf_counter()
    rec = []
    part = O.rsb_partition(g, 4, opts, record=rec)
    m4 = O.partition_metrics(g, part, 4)
    # the 2-part partition is the first split alone
    left = part < 2
    out = {"source": "tests/golden/make_golden.py c3 (FP64 oracle)",
           "mesh": {"dims": [192, 128, 96], "frac": 0.10, "seed": 20260, "adjacency": "vertex",
                    "n": g.n, "nnz": g.nnz, "dmax": dmax},
           "method": "inverse", "degenerate": "none",
           "splits": [{"n": x["n"], "k": x["k"], "lambda2": x["lam"], "resid": x["resid"],
                       "outer": x["iters"], "cut": x["cut"]} for x in rec],
           "weighted_cut_2": O.weighted_cut(g, left),
           "weighted_cut_4": m4["weighted_cut"], "sizes_4": m4["sizes"].tolist(),
           "seconds": round(time.perf_counter() - t, 1)}
    return out


def c5() -> dict:
    g = box_graph_deleted(256, 256, 256, 0.05, 20261, "vertex")
    dmax = float(O.degree(g).max())
    opts = O.Options(method="lanczos", degenerate="none")
    t = time.perf_counter()
    rec = []
    part = O.rsb_partition(g, 2, opts, record=rec)
    return {"source": "tests/golden/make_golden.py c5 (FP64 oracle)",
            "mesh": {"dims": [256, 256, 256], "frac": 0.05, "seed": 20261, "adjacency": "vertex",
                     "n": g.n, "nnz": g.nnz, "dmax": dmax},
            "method": "lanczos", "degenerate": "none",
            "splits": [{"n": x["n"], "k": x["k"], "lambda2": x["lam"], "resid": x["resid"],
                        "cycles": x["iters"], "cut": x["cut"]} for x in rec],
            "weighted_cut_2": O.partition_metrics(g, part, 2)["weighted_cut"],
            "seconds": round(time.perf_counter() - t, 1)}


def main(argv):
    which = argv[1:] or ["medium"]
    for w in which:
        data = {"medium": medium, "c3": c3, "c5": c5}[w]()
        name = {"medium": "irregular_medium.json", "c3": "c3_levels01.json",
                "c5": "c5_level0.json"}[w]
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(data, f, indent=1)
            f.write("\n")
        print("wrote", name, flush=True)


if __name__ == "__main__":
    main(sys.argv)
