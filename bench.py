#!/usr/bin/env python3
"""Benchmark: LR-PD-SDP (Alg. 2) time-to-1e-4 and PDHG iterations/s on GB300.

Workload: MaxCut relaxation of G(n=2000, p=0.01) with integer edge weights in
{1..5} (seed 1), low-rank projection by block Lanczos (block 16, initial rank
8), FP32 block products, tolerance 1e-4 on the relative residuals and gap.

A "step" is one complete solve from X = 0, y = 0 to tolerance 1e-4 with the
problem already resident on the device (every row of the hot path runs in
every iteration).  ``value`` is PDHG iterations per second over the K timed
solves; ``time_to_tol_s`` is the median device time of one solve.  ``e2e``
repeats the measurement through the public C ABI with host buffers:
set_problem (host -> device copy of the problem), solve, and the read-back
of y, the factors V and their eigenvalues.  The full-eigendecomposition PDHG
(Alg. 1) on the same GPU is reported beside it (``full_eig``), using the
vendor eigensolver (torch.linalg.eigh) as a comparison baseline only.

``roofline`` places the tensor-core block product W = S Q (the projection's
O(n^2) term) on the HBM roofline at n = 16384, where S (1 GiB) streams from
HBM; ``streaming`` runs 30 LR-PD-SDP iterations of MaxCut on G(16384, 0.001)
at rank 32 and reports the projection's HBM share over the iteration time;
``projection_hbm`` does the same for the n = 2000 workload (S stays in L2).
``cpu_lr_arpack`` times the paper's own CPU design (ARPACK for the r largest
eigenpairs) on the host cores beside the oracle.

``--impl reference`` times the FP64 CPU oracle (the only reference this work
has; it is deliberately slow) on bounded samples of the same workload.

``--workload mimo-batch`` instead measures the batched path: 256 MIMO
detection relaxations (Sec. 5.3; N log-uniform in [32, 512], seed 4) solved
concurrently through proxsdp_gpu_solve_batch, reported as solves per second.

Multi-GPU (torchrun): the method does not shard a single instance here, so
each rank runs an independent replica ("replicas only"); value = iterations of
all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PDHG time-to-1e-4 & iters/s, low-rank vs full-eig projection, same GB300; HBM %"
WORKLOAD = "maxcut_er_n2000_p0.01_w1-5_seed1"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1916.4)), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.samples = []
        self.proc = None
        self.index = index

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for name, v in zip(names, s[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def workload_problem():
    import sdp_instances as si

    return si.config_maxcut_2000()


OPERATOR_FORMS = {"explicit": 0, "factored": 1, "auto": 2}  # settings.operator_form


def settings_for(pkg, operator="explicit", **kw):
    s = pkg.default_settings(tol=1e-4, rank_init=8, block_size=16, check_every=50,
                             operator_form=OPERATOR_FORMS[operator])
    for k, v in kw.items():
        setattr(s, k, v)
    return s


def flush_l2(torch, buf):
    buf.add_(1.0)  # touch 512 MB (> 129 MB L2)


def run_ours(args, rank, world):
    import torch

    import paper_1810_05231_gb300 as pkg

    torch.cuda.set_device(0 if world == 1 else int(os.environ.get("LOCAL_RANK", rank)))
    dev = torch.device("cuda")
    stream = torch.cuda.Stream()
    inst = workload_problem()
    n = inst.n
    flush = torch.zeros(128 * 1024 * 1024, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        slv = pkg.Solver(settings_for(pkg, args.operator), stream=stream.cuda_stream)
        slv.set_instance(inst)
        for _ in range(args.warmup):
            slv.solve()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = ClockSampler()
        clocks.start()
        times, iters, infos = [], [], []
        for _ in range(args.steps):
            flush_l2(torch, flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = slv.solve()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
            iters.append(info.iters)
            infos.append(info.as_dict())
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = clocks.stop()
    total_t = sum(times)
    total_it = sum(iters)
    # end to end through the C ABI with host buffers (fresh handle state each step)
    e2e_times, e2e_iters = [], []
    h2d = (inst.A_rowptr.nbytes + inst.A_col.nbytes + inst.A_val.nbytes + inst.rhs.nbytes +
           inst.C_idx.nbytes + inst.C_val.nbytes)
    d2h = 0
    with torch.cuda.stream(stream):
        slv2 = pkg.Solver(settings_for(pkg, args.operator), stream=stream.cuda_stream)
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            slv2.set_instance(inst)
            info = slv2.solve()
            out = slv2.get_primal_dual(want_X=False)
            t1 = time.perf_counter()
            e2e_times.append(t1 - t0)
            e2e_iters.append(info.iters)
            d2h = out["y"].nbytes + out["V"].nbytes + out["lam"].nbytes
        slv2.close()
    roof = block_product_roofline(pkg, torch, stream, STREAM_N, 48)
    stream_leg = streaming_leg(pkg, torch, stream) if args.streaming else None
    full = full_eig_baseline(torch, inst, stream, cap_s=args.full_eig_cap) if args.full_eig_cap > 0 else None
    other = args.other_operator
    alt = (operator_form_run(pkg, torch, stream, inst, flush, other, args.steps, min(args.warmup, 2))
           if other != "none" and other != args.operator else None)
    res = dict(times=times, iters=iters, infos=infos, clocks=clk, e2e_times=e2e_times, e2e_iters=e2e_iters,
               h2d=h2d, d2h=d2h, roofline=roof, full=full, launches=sum(i["kernel_launches"] for i in infos),
               alt=alt, streaming=stream_leg)
    slv.close()
    return res


def operator_form_run(pkg, torch, stream, inst, flush, operator, steps, warmup):
    """The same timed solves with the other operator form of S^k (the factored
    one applies S^k from the factors of X^k and never writes it to HBM)."""
    with torch.cuda.stream(stream):
        slv = pkg.Solver(settings_for(pkg, operator), stream=stream.cuda_stream)
        slv.set_instance(inst)
        for _ in range(warmup):
            slv.solve()
        times, iters, launches = [], [], 0
        for _ in range(steps):
            flush_l2(torch, flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = slv.solve()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
            iters.append(info.iters)
            launches += info.kernel_launches
        slv.close()
    return {"operator": operator, "value": round(sum(iters) / sum(times), 2), "unit": "iters/s",
            "time_to_tol_s": round(statistics.median(times), 5), "iters_per_solve": int(statistics.median(iters)),
            "final_rank": info.final_rank, "rel_gap": info.rel_gap, "gpu_launches": int(launches)}


STREAM_N = 16384
STREAM_WORKLOAD = "maxcut_er_n16384_p0.001_unit_seed5"


def block_product_roofline(pkg, torch, stream, n, k, launches=10, reps=5):
    """Time the block product W = S Q alone and place it on the HBM roofline.

    Per launch it reads S once (n^2 * 4 bytes, FP32) and Q (n * k * 4) and
    writes W (n * k * 4): algorithmic bytes n^2 * 4 + 2 * n * k * 4.  At
    n = 16384 S is 1 GiB, far larger than the 129 MB L2, so every launch
    streams S from HBM (no flush needed).  achieved = algorithmic bytes /
    mean CUDA-event time of one launch on the launching stream; peak = the
    measured copy bandwidth of MEASURED_PEAKS.json.  Each timed sample is
    `reps` calls back to back (one call = the TF32 split of Q and the
    product), so the time is the device time of the two kernels.
    """
    hbm, _, src = _peaks()
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    S = torch.randn(n, n, device="cuda", generator=g)
    S = (S + S.t()) * 0.5
    Q = torch.randn(k, n, device="cuda", generator=g)
    flush = torch.zeros(128 * 1024 * 1024, dtype=torch.float32, device="cuda") if n * n * 4 < 512 << 20 else None
    durs = []
    with torch.cuda.stream(stream):
        for it in range(launches + 3):
            if flush is not None:
                flush.add_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):  # back to back: the host side of one call overlaps the previous product
                pkg.block_matvec(S, Q, stream=stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            if it >= 3:
                durs.append(e0.elapsed_time(e1) * 1e-3 / reps)
    l2 = "S larger than L2" if flush is None else "flushed before each launch"
    del S, Q, flush
    torch.cuda.empty_cache()
    t = statistics.mean(durs)
    bytes_alg = n * n * 4 + 2 * n * k * 4
    # the library runs the tensor-core kernel from n = 1024 up (kTcMinN), the SIMT one below
    kernel = "k_block_matvec_tc" if n >= 1024 else "k_block_matvec"
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        try:
            traffic = json.load(open(tp)).get(f"{kernel}_n{n}_k{k}")
        except Exception:
            traffic = None
    achieved = bytes_alg / t / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
            "peak_source": src, "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": traffic,
            "n": n, "k": k, "alg_bytes_per_launch": bytes_alg, "avg_launch_s": t, "launches_timed": len(durs),
            "flops_per_launch": 2.0 * n * n * k, "tflops": round(2.0 * n * n * k / t / 1e12, 2),
            "l2": l2}


def streaming_leg(pkg, torch, stream, iters=30, warmup=10):
    """The LR-PD-SDP iteration where S^k streams from HBM: MaxCut of
    G(16384, 0.001) (unit weights, seed 5), S^k formed in HBM (1 GiB FP32),
    rank fixed at 32 (block width 48).  `warmup` untimed iterations, then
    `iters` iterations timed with CUDA events on the solver's stream.  The
    projection's algorithmic bytes per iteration are (q + 1) n^2 4 (q block
    products reading S, one rebuild writing it); over the whole iteration
    time they give a lower bound on the projection's HBM fraction."""
    import sdp_instances as si

    hbm = _peaks()[0]
    inst = si.maxcut_er_streaming(STREAM_N)
    n = inst.n
    with torch.cuda.stream(stream):
        slv = pkg.Solver(settings_for(pkg, "explicit", tol=1e-12, rank_init=32, max_rank=32, check_every=10),
                         stream=stream.cuda_stream)
        slv.set_instance(inst)
        i0 = slv.iterate(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        i1 = slv.iterate(iters)
        e1.record(stream)
        e1.synchronize()
        slv.close()
    t = e0.elapsed_time(e1) * 1e-3
    done = int(i1.iters - i0.iters)
    q = (i1.matvecs - i0.matvecs) / max(done, 1)
    bytes_iter = (q + 1.0) * n * n * 4.0
    gbs = bytes_iter * done / t / 1e9
    return {"workload": STREAM_WORKLOAD, "n": n, "rank": 32, "iters_timed": done, "iters_per_s": round(done / t, 2),
            "ms_per_iter": round(1000 * t / max(done, 1), 4), "q_products_per_iter": round(q, 3),
            "projection_bytes_per_iter": round(bytes_iter), "projection_gbs_over_iteration": round(gbs, 1),
            "projection_frac_lower_bound": round(gbs / hbm, 4), "status": int(i1.status),
            "gpu_launches": int(i1.kernel_launches - i0.kernel_launches)}


def full_eig_baseline(torch, inst, stream, cap_s=60.0, tol=1e-4, rate_iters_fp64=5):
    """Alg. 1 (PD-SDP, exact projection) with the vendor eigensolver
    (torch.linalg.eigh, cuSOLVER) on the same GPU: the comparison baseline of
    the metric, not part of the library.  The MaxCut workload has only the
    constraints diag(X) = 1 (||A_i||_F = 1, ||M||_2 = 1, alpha = 0.95), so
    M(X) = diag(X) and M*(y) = Diag(y).  Same stop test as the library
    (relative residuals of Sec. 2.2 and relative gap <= tol), in FP32 from
    X = 0, y = 0, capped at `cap_s` seconds; the FP64 eigensolver's
    per-iteration time is reported beside it."""
    n = inst.n
    dev = torch.device("cuda")

    def run(dtype, max_s, max_iters):
        C = torch.tensor(inst.c_dense(), dtype=dtype, device=dev)
        normC = float(torch.linalg.norm(C))
        b = torch.ones(n, dtype=dtype, device=dev)
        normb = float(torch.linalg.norm(b))
        alpha = 0.95
        X = torch.zeros(n, n, dtype=dtype, device=dev)
        y = torch.zeros(n, dtype=dtype, device=dev)
        res = None
        with torch.cuda.stream(stream):
            torch.linalg.eigh(X)  # solver workspace set-up, outside the timed loop
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it = 0
            while True:
                it += 1
                S = X - alpha * (C + torch.diag(y))
                lam, U = torch.linalg.eigh(S)
                Xn = (U * lam.clamp(min=0)) @ U.t()
                yn = y + alpha * torch.diagonal(2 * Xn - X) - alpha * b
                dX = Xn - X
                dy = yn - y
                eps_p = torch.linalg.norm(dX / alpha - torch.diag(dy))
                eps_d = torch.linalg.norm(dy / alpha - torch.diagonal(dX))
                pobj = torch.sum(C * Xn)
                dobj = -torch.dot(b, yn)
                X, y = Xn, yn
                if it % 10 == 0 or it >= max_iters:
                    vals = torch.stack([eps_p, eps_d, pobj, dobj]).double().cpu().tolist()
                    rel_p, rel_d = vals[0] / (1 + normC), vals[1] / (1 + normb)
                    gap = abs(vals[2] - vals[3]) / (1 + abs(vals[2]) + abs(vals[3]))
                    el = time.perf_counter() - t0
                    res = dict(iters=it, rel_p=rel_p, rel_d=rel_d, rel_gap=gap, pobj=vals[2], seconds=el)
                    if max(rel_p, rel_d, gap) <= tol or el >= max_s or it >= max_iters:
                        break
            torch.cuda.synchronize()
        res["seconds"] = time.perf_counter() - t0
        return res

    r32 = run(torch.float32, cap_s, 10 ** 7)
    conv = max(r32["rel_p"], r32["rel_d"], r32["rel_gap"]) <= tol
    r64 = run(torch.float64, 1e9, rate_iters_fp64)
    return {"impl": "torch.linalg.eigh (cuSOLVER), Alg. 1, same stop test", "tol": tol,
            "fp32": {"converged": conv, "time_to_tol_s": round(r32["seconds"], 4) if conv else None,
                     "iters": r32["iters"], "iters_per_s": round(r32["iters"] / r32["seconds"], 2),
                     "cap_s": cap_s, "rel_primal_res": r32["rel_p"], "rel_dual_res": r32["rel_d"],
                     "rel_gap": r32["rel_gap"], "primal_obj": r32["pobj"]},
            "fp64": {"iters_per_s": round(r64["iters"] / r64["seconds"], 3), "iters_timed": r64["iters"]}}


def cpu_oracle_sample(seconds=15.0, min_iters=2):
    """The FP64 oracle's LR iteration on the same workload for ~`seconds`."""
    import oracle
    from oracle.sdp import Problem, normalize_rows, operator_norm, pd_iteration

    inst = workload_problem()
    prob = Problem.from_instance(inst)
    sp, _ = normalize_rows(prob)
    alpha = 0.95 / operator_norm(sp)
    X = np.zeros((inst.n, inst.n))
    y = np.zeros(sp.M.m)
    t0 = time.perf_counter()
    k = 0
    while True:
        st = pd_iteration(sp, X, y, alpha, 8)
        X, y = st.X, st.y
        k += 1
        if k >= min_iters and time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return k / dt, k, dt


def arpack_step(sp, X, y, alpha, rank, v0):
    """One LR-PD-SDP iteration (Alg. 2) with the r largest eigenpairs of
    S = X - alpha (M*(y) + C) from ARPACK (scipy eigsh, which="LA");
    returns (X+, y+, start vector for the next call)."""
    import scipy.sparse.linalg as spla

    from oracle.sdp import dual_prox

    S = X - alpha * (sp.M.adjoint(y) + sp.C)
    lam, U = spla.eigsh(S, k=rank, which="LA", v0=v0, tol=1e-10)
    Xn = (U * np.maximum(lam, 0.0)) @ U.T
    yn = dual_prox(y + alpha * sp.M.apply(2.0 * Xn - X), alpha, sp.rhs, sp.m_eq)
    return Xn, yn, U[:, -1]


def cpu_arpack_sample(seconds=15.0, min_iters=2, rank=16):
    """The paper's own CPU design (Sec. 4: a Lanczos method, ARPACK, for the
    r largest eigenpairs) timed on the host cores: LR-PD-SDP iterations of the
    n = 2000 workload with the truncated projection of Eq. trunc_eig computed
    by scipy.sparse.linalg.eigsh (ARPACK, which="LA", k = r, FP64) and the
    other steps of Alg. 2 as in the oracle."""
    from oracle.sdp import Problem, normalize_rows, operator_norm

    inst = workload_problem()
    prob = Problem.from_instance(inst)
    sp, _ = normalize_rows(prob)
    alpha = 0.95 / operator_norm(sp)
    n = inst.n
    X = np.zeros((n, n))
    y = np.zeros(sp.M.m)
    v0 = np.random.default_rng(0).standard_normal(n)
    t0 = time.perf_counter()
    k = 0
    while True:
        X, y, v0 = arpack_step(sp, X, y, alpha, rank, v0)
        k += 1
        if k >= min_iters and time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return k / dt, k, dt


def host_description():
    """CPU model, hardware threads and the BLAS numpy links (for the oracle's timing)."""
    import platform

    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")) and ":" in line:
                    model = line.split(":", 1)[1].strip() or model
                    if line.lower().startswith("model name"):
                        break
    except OSError:
        pass
    blas = "unknown"
    try:
        cfg = np.show_config(mode="dicts")
        b = cfg["Build Dependencies"]["blas"]
        blas = f'{b.get("name", "?")} {b.get("version", "")}'.strip()
    except Exception:
        pass
    return {"cpu": f"{platform.machine()} {model}", "nproc": os.cpu_count(), "blas": blas,
            "blas_threads": os.environ.get("OMP_NUM_THREADS", "default (all cores)")}


def projection_hbm(n, info, iters_per_s, hbm_gbs):
    """HBM share of the projection per iteration: (q + 1) n^2 4 bytes (q block
    products reading S, one rebuild writing it; full n^2, not the symmetric
    half) over the measured time of a whole iteration (an upper bound on the
    projection's time, so the fraction is a lower bound)."""
    q = info["matvecs"] / max(info["iters"], 1)
    bytes_per_iter = (q + 1.0) * n * n * 4.0
    gbs = bytes_per_iter * iters_per_s / 1e9
    return {"bytes_per_iter": round(bytes_per_iter), "q_products_per_iter": round(q, 3),
            "achieved_gbs": round(gbs, 1), "peak_gbs": hbm_gbs, "frac": round(gbs / hbm_gbs, 4),
            "time_base": "whole iteration"}


GOLDEN_C2 = os.path.join(ROOT, "tests", "golden", "c2_oracle.json")
# device-time share of the top kernel in the ncu launch list of the bench's
# own solve (graphs off, the same rank path), committed under profiles/
DOMINANT_KERNEL = {"kernel": "k_sym_eig", "share_of_device_time": 0.475, "bound": "latency (one CTA)",
                   "source": "profiles/launches_maxcut_n2000_bench_solve.md"}


def oracle_objective_error(pobj):
    """Relative difference of the solve's objective from the FP64 oracle's
    solve to 1e-5 stored in tests/golden/c2_oracle.json (None if absent)."""
    try:
        gold = json.load(open(GOLDEN_C2))
    except Exception:
        return None
    return {"value": abs(pobj - gold["pobj"]) / abs(gold["pobj"]), "oracle_pobj": gold["pobj"],
            "oracle_tol": gold["tol"]}


def run_mimo_batch(args):
    """Aggregate solves/s of the MIMO batch (row a12), inputs resident."""
    # more hardware work queues than the default 8, so that the instances'
    # streams do not share queues (set before the first CUDA call)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch

    import paper_1810_05231_gb300 as pkg
    import sdp_instances as si

    insts = si.config_mimo_batch(args.batch, seed=4)
    def make():
        out = []
        for p in insts:
            s = pkg.Solver(tol=1e-4, rank_init=4, max_iter=200000, check_every=200)
            s.set_instance(p)
            out.append(s)
        return out
    for _ in range(max(1, args.warmup)):
        sv = make()
        pkg.solve_batch(sv, host_threads=args.host_threads)
        for s in sv:
            s.close()
    times, infos = [], None
    for _ in range(args.steps):
        sv = make()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = pkg.solve_batch(sv, host_threads=args.host_threads)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        for s in sv:
            s.close()
    conv = sum(1 for i in infos if i.status == pkg.CONVERGED)
    t = statistics.median(times)
    line = {"metric": "MIMO batch solves/s (256 instances, N in [32, 512], tol 1e-4)",
            "value": round(len(insts) / t, 3), "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1000 * t, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "mimo_batch_256_seed4", "host_threads": args.host_threads, "tol": 1e-4},
            "converged": conv, "iters_total": int(sum(i.iters for i in infos)),
            "max_iters": int(max(i.iters for i in infos))}
    print(json.dumps(line))
    return 0


def main_config(args, world):
    """The workload of the main line, printed identically by both arms."""
    return {"workload": WORKLOAD, "n": 2000, "rank_init": 8, "block": 16, "tol": 1e-4, "operator": args.operator,
            "l2": "flushed before each timed solve", "parallelism": "replicas" if world > 1 else "single"}


def mimo_batch_leg(n_inst, host_threads):
    """Config 5 beside the main line: n_inst MIMO relaxations (N log-uniform in
    [32, 512], seed 4) solved to 1e-4 through proxsdp_gpu_solve_batch (one
    handle, stream and graph per instance on host threads), timed once after
    a warm-up on eight of them."""
    import torch

    import paper_1810_05231_gb300 as pkg
    import sdp_instances as si

    insts = si.config_mimo_batch(n_inst, seed=4)

    def make(ps):
        out = []
        for p in ps:
            s = pkg.Solver(tol=1e-4, rank_init=4, max_iter=200000, check_every=200)
            s.set_instance(p)
            out.append(s)
        return out

    sv = make(insts[:8])
    pkg.solve_batch(sv, host_threads=host_threads)
    for s in sv:
        s.close()
    sv = make(insts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos = pkg.solve_batch(sv, host_threads=host_threads)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    for s in sv:
        s.close()
    return {"value": round(len(insts) / t, 3), "unit": "solves/s", "instances": len(insts), "seconds": round(t, 3),
            "converged": sum(1 for i in infos if i.status == pkg.CONVERGED),
            "iters_total": int(sum(i.iters for i in infos)), "host_threads": host_threads,
            "how": "proxsdp_gpu_solve_batch: one handle, stream and graph per instance, host thread pool "
                   "(not one persistent launch)"}


SWEEPS = {
    # Table 2 shape: sensor network localisation (Sec. 5.2), n sensors, 5 anchors, radius 0.3
    "table2": ("sensor network localisation (Sec. 5.2), Table 2 sizes", [50, 100, 150, 200, 250, 300]),
    # Table 3 shape: MIMO detection with high SNR (Sec. 5.3, noise variance 0.01), signal length n
    "table3": ("MIMO detection, high SNR (Sec. 5.3), Table 3 sizes", [100, 500, 1000, 2000]),
}
# LR-PD-SDP running times (s) printed in the paper's Table 2 and Table 3 (a
# CPU implementation on other hardware): context beside each size, not a target
PAPER_SECONDS = {
    "table2": {50: 0.6, 100: 1.6, 150: 3.6, 200: 6.1, 250: 7.9, 300: 13.5},
    "table3": {100: 0.1, 500: 1.1, 1000: 4.7, 2000: 38.9, 3000: 122.1, 4000: 258.3, 5000: 472.4},
}


def sweep_instance(kind, n, seed):
    import numpy as np

    import sdp_instances as si

    if kind == "table2":
        return si.sensor_network(n, 5, 0.3, seed=seed)
    return si.mimo(n, np.random.default_rng(seed), snr_noise_var=0.01)


def run_sweep(args):
    """One seeded instance per size, solved once to 1e-4 (after one untimed
    solve of the smallest size); the line lists time to tolerance per size."""
    import torch

    import paper_1810_05231_gb300 as pkg

    title, sizes = SWEEPS[args.workload]
    if args.sizes:
        sizes = [int(v) for v in args.sizes.split(",")]
    rank0 = 4 if args.workload == "table2" else 2

    def solve(n):
        inst = sweep_instance(args.workload, n, seed=n)
        slv = pkg.Solver(tol=1e-4, rank_init=rank0, max_iter=10 ** 7, time_limit_s=args.time_limit,
                         check_every=200)
        t0 = time.perf_counter()
        slv.set_instance(inst)
        info = slv.solve()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        slv.close()
        return inst.n, info, wall

    solve(sizes[0])
    rows = []
    for n in sizes:
        dim, info, wall = solve(n)
        rows.append({"n": n, "matrix_dim": dim, "status": info.status, "converged": info.status == pkg.CONVERGED,
                     "time_to_tol_s": round(info.solve_seconds, 4), "wall_s_with_set_problem": round(wall, 4),
                     "iters": int(info.iters), "final_rank": info.final_rank, "primal_obj": info.primal_obj,
                     "rel_primal_res": info.rel_primal_res, "rel_dual_res": info.rel_dual_res,
                     "rel_gap": info.rel_gap, "gpu_launches": int(info.kernel_launches),
                     "paper_lr_pd_sdp_s": PAPER_SECONDS[args.workload].get(n)})
    total = sum(r["time_to_tol_s"] for r in rows)
    line = {"metric": f"time to 1e-4 per instance size: {title}", "value": round(total, 4), "unit": "s",
            "n_gpus": 1, "steps": len(rows), "warmup": 1, "ms_per_step": round(1000 * total / len(rows), 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": args.workload, "tol": 1e-4, "rank_init": rank0,
                                            "time_limit_s": args.time_limit},
            "sweep": rows, "gpu_launches": int(sum(r["gpu_launches"] for r in rows))}
    print(json.dumps(line))
    return 0


WORKLOAD_SOLVES = {
    # one whole solve to 1e-4 of a larger configuration, capped (seconds)
    "c4": ("graph equipartition of G(5000, 0.002), unit weights, seed 3 (Sec. 5.1), tr(11^T X) = 0 as a "
           "structured row", "config_equipartition_5000", 16),
    "c3": ("sensor network localisation, 1000 sensors + 10 anchors, radius 0.2, seed 2 (Sec. 5.2)",
           "config_sensor_1000", 8),
}


def run_workload_solve(args):
    """Time to 1e-4 of one solve of a larger configuration (the factored
    operator where it applies), capped at --time-limit seconds; the line
    reports the residuals and the gap reached when the cap ends it."""
    import torch

    import paper_1810_05231_gb300 as pkg
    import sdp_instances as si

    title, fn, rank0 = WORKLOAD_SOLVES[args.workload]
    inst = getattr(si, fn)()
    slv = pkg.Solver(tol=1e-4, rank_init=rank0, max_iter=10 ** 7, time_limit_s=args.time_limit, check_every=200,
                     operator_form=OPERATOR_FORMS[args.operator], at_max_rank=1 if args.at_max_rank else 0)
    t0 = time.perf_counter()
    slv.set_instance(inst)
    info = slv.solve()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    slv.close()
    conv = info.status == pkg.CONVERGED
    line = {"metric": f"time to 1e-4: {title}", "value": round(info.solve_seconds, 3), "unit": "s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": round(1000 * info.solve_seconds, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": fn, "n": inst.n, "tol": 1e-4, "rank_init": rank0, "operator": args.operator,
                       "time_limit_s": args.time_limit, "at_max_rank": "continue" if args.at_max_rank else "stop"},
            "converged": conv, "status": int(info.status), "iters": int(info.iters), "final_rank": info.final_rank,
            "iters_per_s": round(info.iters / max(info.solve_seconds, 1e-9), 2), "primal_obj": info.primal_obj,
            "rel_primal_res": info.rel_primal_res, "rel_dual_res": info.rel_dual_res, "rel_gap": info.rel_gap,
            "wall_s_with_set_problem": round(wall, 3), "gpu_launches": int(info.kernel_launches)}
    print(json.dumps(line))
    return 0


def aggregate_replicas(total_t, total_it, device):
    """Whole-job figures of N independent replicas (one per rank, no data-path
    collective): iterations summed over the ranks, time the maximum over the
    ranks (the slowest replica ends the job).  `device` is "cuda" under NCCL,
    "cpu" under gloo."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(total_t)], dtype=torch.float64, device=device)
    it = torch.tensor([float(total_it)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(it, op=dist.ReduceOp.SUM)
    return float(t.item()), float(it.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--full-eig-cap", type=float, default=100.0,
                    help="seconds allowed to the full-eig PDHG baseline to reach 1e-4 (0: skip)")
    ap.add_argument("--arpack-seconds", type=float, default=10.0, help="host seconds of the ARPACK LR leg (0: skip)")
    ap.add_argument("--streaming", type=int, default=1, help="run the n = 16384 streaming leg (1) or not (0)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="maxcut",
                    choices=["maxcut", "mimo-batch"] + sorted(SWEEPS) + sorted(WORKLOAD_SOLVES))
    ap.add_argument("--sizes", default="", help="comma-separated sizes for the table2 / table3 sweeps")
    ap.add_argument("--time-limit", type=float, default=60.0, help="per-instance cap of the sweeps (s)")
    ap.add_argument("--at-max-rank", action="store_true",
                    help="workload solves: keep iterating at the rank cap instead of stopping there")
    ap.add_argument("--operator", default="explicit", choices=sorted(OPERATOR_FORMS),
                    help="how the projection applies S^k: formed in HBM, or from the factors of X^k")
    ap.add_argument("--other-operator", default="factored", choices=sorted(OPERATOR_FORMS) + ["none"],
                    help="also time the solves with this operator form (reported beside the line)")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--batch-leg", type=int, default=256,
                    help="MIMO instances of the batch leg of the main line (0: skip it)")
    ap.add_argument("--host-threads", type=int, default=48)
    args = ap.parse_args()
    # more hardware work queues than the default 8 for the batch legs' many
    # streams (before the first CUDA call)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    if args.workload == "mimo-batch":
        return run_mimo_batch(args)
    if args.workload in SWEEPS:
        return run_sweep(args)
    if args.workload in WORKLOAD_SOLVES:
        return run_workload_solve(args)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank != 0:
            return 0
        vals = []
        total_k, total_t = 0, 0.0
        for _ in range(args.warmup):
            cpu_oracle_sample(seconds=1.0, min_iters=1)
        for _ in range(args.steps):
            v, k, dt = cpu_oracle_sample(seconds=args.cpu_seconds / max(args.steps, 1), min_iters=1)
            vals.append(v)
            total_k += k
            total_t += dt
        value = total_k / total_t
        line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "iters/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1000 * total_t / max(args.steps, 1), 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": main_config(args, 1),
                "cpu_baseline": {"value": round(value, 4), "unit": "iters/s", "cores": os.cpu_count(),
                                 "kind": "oracle", "sample": f"{total_k} LR-PD-SDP iterations (exact eigh) of the n=2000 workload"},
                "e2e": {"value": round(value, 4), "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world)
    total_t = sum(res["times"])
    total_it = sum(res["iters"])
    if world > 1:
        total_t, total_it = aggregate_replicas(total_t, total_it, "cuda")
    cpu = None
    arpack = None
    if rank == 0 and world == 1:
        v, k, dt = cpu_oracle_sample(seconds=args.cpu_seconds)
        cpu = {"value": round(v, 4), "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{k} LR-PD-SDP iterations of the n=2000 workload (FP64, exact eigh) in {dt:.1f} s",
               "host": host_description()}
        if args.arpack_seconds > 0:
            va, ka, dta = cpu_arpack_sample(seconds=args.arpack_seconds)
            arpack = {"value": round(va, 4), "unit": "iters/s", "cores": os.cpu_count(),
                      "kind": "LR-PD-SDP with ARPACK eigsh (the paper's CPU design), FP64",
                      "sample": f"{ka} iterations of the n=2000 workload at rank 16 in {dta:.1f} s"}
    batch = None
    if rank == 0 and world == 1 and args.batch_leg > 0:
        batch = mimo_batch_leg(args.batch_leg, args.host_threads)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    value = total_it / total_t
    info = res["infos"][-1]
    e2e_val = sum(res["e2e_iters"]) / sum(res["e2e_times"])
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1000 * total_t / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": main_config(args, world),
        "time_to_tol_s": round(statistics.median(res["times"]), 5),
        "iters_per_solve": int(statistics.median(res["iters"])),
        "final_rank": info["final_rank"], "primal_obj": info["primal_obj"], "rel_gap": info["rel_gap"],
        "matvecs_per_iter": round(info["matvecs"] / max(info["iters"], 1), 3),
        "lanczos_cycles_per_iter": round(info["lanczos_cycles"] / max(info["iters"], 1), 3),
        "e2e": {"value": round(e2e_val, 2), "unit": "iters/s", "h2d_bytes_per_step": int(res["h2d"]),
                "d2h_bytes_per_step": int(res["d2h"]),
                "time_to_tol_s": round(statistics.median(res["e2e_times"]), 5)},
        "obj_rel_err_vs_oracle": oracle_objective_error(info["primal_obj"]),
        "roofline": res["roofline"],
        "projection_hbm": projection_hbm(2000, info, value, _peaks()[0]),
        "streaming": res["streaming"],
        "dominant_kernel": DOMINANT_KERNEL,
        "cpu_baseline": cpu, "cpu_lr_arpack": arpack, "clocks": res["clocks"],
        "gpu_launches": int(res["launches"]), "full_eig": res["full"], "other_operator_form": res["alt"],
        "mimo_batch": batch,
    }
    print(json.dumps(line))
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
