"""Write ``c2_oracle.json``: the FP64 oracle's converged solve of the n = 2000 MaxCut workload.

The workload is the MaxCut relaxation (Sec. 1.4, ``min -1/4 tr(L X)``,
``diag(X) = 1``) of the seeded G(2000, 0.01) graph with integer weights 1..5
(``sdp_instances.config_maxcut_2000``).  The values come from
``oracle.solve`` (Alg. 2 with the exact truncated projection of Eq. trunc_eig)
run to a tolerance ten times tighter than the 1e-4 target, and from
``oracle.certificates`` of the result; nothing here calls the CUDA library.

Run from the repository root (about an hour on eight host cores)::

    python tests/golden/make_c2_oracle.py
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import sdp_instances as gen  # noqa: E402
from oracle.sdp import Problem  # noqa: E402

TOL = 1e-5


def main():
    inst = gen.config_maxcut_2000()
    prob = Problem.from_instance(inst)
    t0 = time.time()
    res = oracle.solve(prob, mode="lr", tol=TOL, max_iter=20000, rank_init=8, record_history=True)
    secs = time.time() - t0
    cert = oracle.certificates(prob, res.X, res.y)
    first = {}
    for h in res.history:
        worst = max(h["rel_p"], h["rel_d"], h["rel_gap"])
        for t in (1e-3, 1e-4, 1e-5):
            if worst <= t and str(t) not in first:
                first[str(t)] = dict(it=h["it"], pobj=h["pobj"], r=h["r"])
    out = dict(
        source="oracle.solve(mode='lr') on sdp_instances.config_maxcut_2000(), then oracle.certificates",
        workload="maxcut_er_n2000_p0.01_w1-5_seed1",
        n=inst.n,
        tol=TOL,
        status=int(res.status),
        iters=int(res.iters),
        rank=int(res.rank),
        rank_path_changes=[int(i + 1) for i in range(1, len(res.rank_path))
                           if res.rank_path[i] != res.rank_path[i - 1]],
        pobj=res.pobj,
        dobj=res.dobj,
        rel_primal=res.rel_primal,
        rel_dual=res.rel_dual,
        rel_gap=res.rel_gap,
        certificates=cert,
        first_iteration_within=first,
        seconds=secs,
        host_threads=os.cpu_count(),
        numpy=np.__version__,
    )
    path = os.path.join(HERE, "c2_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(json.dumps(out, sort_keys=True))


if __name__ == "__main__":
    main()
