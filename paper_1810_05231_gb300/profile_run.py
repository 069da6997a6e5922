"""Run a fixed number of LR-PD-SDP iterations of a synthetic workload with
direct kernel launches (no CUDA graph), so that a profiler sees every kernel
launch individually:

    python -m paper_1810_05231_gb300.profile_run --iters 150 --rank 32

The workload is the MaxCut SDP relaxation (Sec. 5.1) of the seeded weighted
Erdos-Renyi graph G(2000, 0.01) with integer weights 1..5 (seed 1); ``--rank``
sets the initial target rank r (the block width follows from it).  Prints the
solver's info record as one line.  ``--operator factored`` applies S^k from
the factors of X^k instead of forming it; ``--instance equipartition_5000``
runs the graph equipartition relaxation of G(5000, 0.002) (unit weights,
seed 3, the structured row tr(11^T X) = 0) instead.
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=150)
    ap.add_argument("--rank", type=int, default=32)
    ap.add_argument("--graphs", action="store_true", help="use the graph-captured loop instead")
    ap.add_argument("--operator", choices=["explicit", "factored", "auto"], default="explicit")
    ap.add_argument("--instance", choices=["maxcut_2000", "equipartition_5000"], default="maxcut_2000")
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import sdp_instances as si

    import paper_1810_05231_gb300 as pkg

    inst = si.config_maxcut_2000() if args.instance == "maxcut_2000" else si.config_equipartition_5000()
    form = {"explicit": pkg.OP_EXPLICIT, "factored": pkg.OP_FACTORED, "auto": pkg.OP_AUTO}[args.operator]
    slv = pkg.Solver(tol=1e-4, rank_init=args.rank, block_size=16, use_graphs=1 if args.graphs else 0,
                     check_every=1000, operator_form=form)
    slv.set_instance(inst)
    info = slv.iterate(args.iters)
    print(json.dumps(info.as_dict()))
    slv.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
