"""Run LR-PD-SDP iterations of a synthetic workload with direct kernel
launches (no CUDA graph), so that a profiler sees every kernel launch
individually, and summarise an ncu launch list:

    python -m paper_1810_05231_gb300.profile_run --solve
    python -m paper_1810_05231_gb300.profile_run --iters 150 --rank 32
    python -m paper_1810_05231_gb300.profile_run --instance maxcut_16384 --iters 12 --rank 32
    python -m paper_1810_05231_gb300.profile_run --summarize launches.csv

Workloads: the MaxCut SDP relaxation (Sec. 5.1) of the seeded weighted
Erdos-Renyi graph G(2000, 0.01) with integer weights 1..5 (seed 1; the bench
workload); the graph equipartition relaxation of G(5000, 0.002) (unit
weights, seed 3, the structured row tr(11^T X) = 0); the MaxCut relaxation of
G(16384, 0.001) (unit weights, seed 5; S^k is 1 GiB).  ``--solve`` runs the
bench's own solve (initial rank 8, tolerance 1e-4, the rank rule on) to
convergence; otherwise ``--iters`` iterations run from X = 0 at initial rank
``--rank``.  Prints the solver's info record as one line.  ``--operator
factored`` applies S^k from the factors of X^k instead of forming it.
``--summarize`` reads the CSV that ``ncu --metrics gpu__time_duration.sum
--csv`` wrote and prints per kernel its launches, total and average time and
share of the device time, as a Markdown table.
"""
from __future__ import annotations

import argparse
import csv
import json
import os
import sys
from collections import defaultdict


def summarize(path: str) -> str:
    tot = defaultdict(float)
    cnt = defaultdict(int)
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for row in csv.DictReader(lines):
        if row.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = row["Kernel Name"].split("(")[0].replace("void ", "").replace("psdp::", "")
        unit = row.get("Metric Unit", "nsecond")
        val = float(row["Metric Value"].replace(",", ""))
        scale = {"nsecond": 1e-3, "usecond": 1.0, "msecond": 1e3, "second": 1e6}.get(unit, 1e-3)
        tot[name] += val * scale
        cnt[name] += 1
    total = sum(tot.values())
    out = [f"Total {total / 1e3:.1f} ms over {sum(cnt.values())} launches.", "",
           "| kernel | launches | total ms | avg us | share |", "|---|---:|---:|---:|---:|"]
    for name in sorted(tot, key=lambda k: -tot[k]):
        out.append(f"| `{name}` | {cnt[name]} | {tot[name] / 1e3:.2f} | {tot[name] / cnt[name]:.1f} | "
                   f"{100.0 * tot[name] / total:.1f}% |")
    return "\n".join(out)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=150)
    ap.add_argument("--rank", type=int, default=32)
    ap.add_argument("--solve", action="store_true", help="the bench's solve: rank 8 to 1e-4, rank rule on")
    ap.add_argument("--graphs", action="store_true", help="use the graph-captured loop instead")
    ap.add_argument("--operator", choices=["explicit", "factored", "auto"], default="explicit")
    ap.add_argument("--instance", choices=["maxcut_2000", "equipartition_5000", "maxcut_16384"],
                    default="maxcut_2000")
    ap.add_argument("--summarize", default="", help="ncu launch-list CSV to summarise (no GPU work)")
    args = ap.parse_args(argv)
    if args.summarize:
        print(summarize(args.summarize))
        return 0
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import sdp_instances as si

    import paper_1810_05231_gb300 as pkg

    if args.instance == "maxcut_2000":
        inst = si.config_maxcut_2000()
    elif args.instance == "equipartition_5000":
        inst = si.config_equipartition_5000()
    else:
        inst = si.maxcut_er_streaming(16384)
    form = {"explicit": pkg.OP_EXPLICIT, "factored": pkg.OP_FACTORED, "auto": pkg.OP_AUTO}[args.operator]
    if args.solve:
        slv = pkg.Solver(tol=1e-4, rank_init=8, block_size=16, use_graphs=1 if args.graphs else 0, check_every=50,
                         operator_form=form)
        slv.set_instance(inst)
        info = slv.solve()
    else:
        slv = pkg.Solver(tol=1e-4, rank_init=args.rank, max_rank=max(args.rank, 60), block_size=16,
                         use_graphs=1 if args.graphs else 0, check_every=1000, operator_form=form)
        slv.set_instance(inst)
        info = slv.iterate(args.iters)
    print(json.dumps(info.as_dict()))
    slv.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
