"""Parity of every workload and form against the ground truth, as numbers.

For each workload (Robertson, mech22, mech54, the mixed batch's two kinds,
the adjoint workload's forward map) and each GPU form (plain: FP64 Newton
matrix, 32 lanes per cell, static assignment; chosen: FP32 Newton matrix,
device queue, the benchmark's mapping), at rtol 1e-6 and 1e-8 (atol 1e-10
and 1e-12): the GPU's final states on a sample of cells -- the first cells
plus the ones with the most GPU steps -- against the oracle at rtol 1e-12
(atol 1e-4 times the run's), in tolerance units |y - y_ref| / (rtol |y_ref| + atol)
(each cell's worst component: median, 99th percentile, maximum), with the
oracle's own run at the same rtol beside it (bench.parity_check).

Run on a GPU:  python tests/parity_report.py [--out FILE.json]
Prints a markdown table.  The GPU runs integrate whole batches (full size,
or a stated prefix for mech54) in the launch form the benchmark times; the
samples are taken from those batches.
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
import synth  # noqa: E402


def gpu_run(w, form, rtol, atol):
    import torch
    import paper_2405_01713_b300 as sb
    Y, P, C = bench.flat_inputs(w)
    kw = dict(bench.FORMS[form])
    prec = kw["precision"] if w["kind"] in ("mechanism", "mixed") else 0
    it = sb.from_workload(w, precision=prec, lanes_per_cell=kw["lanes_per_cell"], schedule=kw["schedule"])
    n_tol = (w["mech"].n_vars + 1) if w["kind"] == "mixed" else w.get("n_vars", 1)
    it.set_tolerances(rtol, np.full(n_tol, atol))
    it.set_params(torch.tensor(P, device="cuda"))
    y = torch.tensor(Y, device="cuda")
    it.integrate(y, w["t0"], w["tout"])
    tot = it.totals()
    nst = it.cell_stats()[:, 0].cpu().numpy()
    out = y.cpu().numpy()
    mapping = it.mapping()[:3] if w["kind"] in ("mechanism", "mixed") else None
    it.close()
    return out, nst, tot, mapping


WORKLOADS = [
    ("robertson", lambda: synth.workloads.robertson(1024), 1024, 0, "all 1024 cells"),
    ("mech22", lambda: synth.workloads.mech22(), 4096, 256, "2^18 cells"),
    ("mech54", lambda: synth.workloads.mech54(2 ** 16), 1024, 64, "first 2^16 of the 2^20 cells"),
    ("mixed", lambda: synth.workloads.mixed(), 4096, 256, "2^24 + 2^16 cells"),
    ("adjoint", lambda: synth.workloads.adjoint(), 1024, 128, "2^16 cells, forward map"),
]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--only", default=None, help="comma-separated workload names")
    args = ap.parse_args()
    nth = oracle.num_threads()
    rows = []
    for name, make, n_first, n_hard, batch in WORKLOADS:
        if args.only and name not in args.only.split(","):
            continue
        w = make()
        w.setdefault("name", name)
        forms = ["plain", "chosen"] if w["kind"] in ("mechanism", "mixed") else ["chosen"]
        for rtol, atol in ((1e-6, 1e-10), (1e-8, 1e-12)):
            res = {}
            for form in forms:
                y, nst, tot, mapping = gpu_run(w, form, rtol, atol)
                res[form] = (y, nst, tot, mapping)
            # the sample: the first cells plus the ones the chosen form found hardest
            y_c, nst_c = res["chosen"][0], res["chosen"][1]
            for form in forms:
                y, nst, tot, mapping = res[form]
                cells_out = []
                par = bench.parity_check(w, y, nst_c, rtol=rtol, atol=atol, n_first=n_first, n_hard=n_hard,
                                         nthreads=nth, per_cell=cells_out)
                for p, pc in zip(par, cells_out):
                    rows.append(dict(workload=name, batch=batch, kind=p["kind"], form=form, rtol=rtol,
                                     cells=p["cells"], gpu=p["gpu"], oracle=p["oracle"],
                                     beyond_10rtol=p["beyond_10rtol"],
                                     worst_status=tot["worst_status"], mapping=mapping))
                    print(json.dumps(rows[-1]), flush=True)
                    rows[-1]["per_cell"] = {k: np.asarray(v).tolist() for k, v in pc.items() if k != "kind"}
    print()
    print("| workload | kind | form | rtol | GPU median / p99 / max | oracle median / p99 / max "
          "| cells within 10 rtol (GPU / oracle) | GPU cells beyond: oracle also beyond, median GPU/oracle |")
    print("|---|---|---|---|---|---|---|---|")
    for r in rows:
        g, o, b = r["gpu"], r["oracle"], r["beyond_10rtol"]
        bb = "-" if not b["cells"] else f"{b['cells']}: {100 * b['oracle_also_beyond']:.0f} %, {b['median_gpu_over_oracle']:.2g}"
        print(f"| {r['workload']} ({r['batch']}) | {r['kind']} | {r['form']} | {r['rtol']:g} | "
              f"{g['median']:.3g} / {g['p99']:.3g} / {g['max']:.3g} | "
              f"{o['median']:.3g} / {o['p99']:.3g} / {o['max']:.3g} | "
              f"{100 * g['within_10rtol']:.1f} / {100 * o['within_10rtol']:.1f} % | {bb} |")
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(rows, fh, indent=1)


if __name__ == "__main__":
    main()
