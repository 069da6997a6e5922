"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (float comparisons):
* block product S Q (FP32 data, FP32 accumulation): relative Frobenius error
  <= 2e-6 * sqrt(n)/sqrt(2000) + 1e-6 against the FP64 product;
* small Jacobi eigensolver (FP32 rotations): eigenvalues within 2e-6 ||T||,
  residual ||T y - theta y|| <= 1e-5 ||T||;
* truncated projection aproj(S, r): ||P_gpu - P_ref||_F / ||P_ref||_F <= 1e-5;
* one iteration of Alg. 2 from a shared iterate: X and y within 1e-4
  relative, residuals within 1e-3 relative (they are differences of nearby
  iterates);
* converged solves: objective within 1e-4 relative of the closed form or of
  the oracle, certificates (primal infeasibility, relative gap, dual
  infeasibility) within 1e-4.
"""
import json
import os
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import sdp_instances as si
from oracle.sdp import Problem, normalize_rows, pd_iteration

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_05231_gb300 as p

    return p


DEV = "cuda:0"


# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,k", [(1, 1), (17, 3), (300, 16), (1000, 48), (2000, 16), (2049, 7), (2000, 80),
                                 (2000, 128), (1536, 256), (1537, 130), (5000, 64), (16384, 48), (100, 40)])
def test_block_matvec(pkg, n, k):
    """n a multiple of 4 takes the tensor-core kernel (TMA needs 16-byte row
    strides), other n the SIMT kernel."""
    rng = np.random.default_rng(n + k)
    A = rng.standard_normal((n, n))
    S = (A + A.T) / 2
    Q = rng.standard_normal((n, k))
    W = pkg.block_matvec(torch.tensor(S, dtype=torch.float32, device=DEV),
                         torch.tensor(Q.T.copy(), dtype=torch.float32, device=DEV))
    torch.cuda.synchronize()
    Wg = W.double().cpu().numpy().T
    ref = S.astype(np.float32).astype(np.float64) @ Q.astype(np.float32).astype(np.float64)
    err = np.linalg.norm(Wg - ref) / max(np.linalg.norm(ref), 1e-30)
    assert err <= 2e-6 * math.sqrt(n / 2000.0) + 1e-6


@pytest.mark.parametrize("K", [2, 8, 33, 48, 64, 96, 128])
def test_sym_eig(pkg, K):
    rng = np.random.default_rng(K)
    A = rng.standard_normal((K, K))
    T = (A + A.T) / 2
    theta, Y = pkg.sym_eig(torch.tensor(T, device=DEV))
    torch.cuda.synchronize()
    th = theta.cpu().numpy()
    Yn = Y.double().cpu().numpy()
    ref = np.sort(np.linalg.eigvalsh(T))[::-1]
    nT = np.linalg.norm(T, 2)
    assert np.max(np.abs(th - ref)) <= 2e-6 * nT
    assert np.linalg.norm(T @ Yn - Yn * th) <= 1e-5 * nT * math.sqrt(K)
    assert np.linalg.norm(Yn.T @ Yn - np.eye(K)) <= 1e-5 * math.sqrt(K)


@pytest.mark.parametrize("K", [32, 96, 128])
def test_sym_eig_ritz_values_fp64_grade(pkg, K):
    """The Rayleigh-Ritz eigensolve runs in FP32 with the FP32-pair refinement
    (Ogita-Aishima step, T y accumulated in FP32 pairs against the FP64 T,
    Rayleigh quotients in FP64): on a separated spectrum the Ritz values
    reach FP64 grade (<= 1e-11 ||T||) while the vectors stay FP32 grade."""
    rng = np.random.default_rng(100 + K)
    lam = np.sort(np.linspace(-1.0, 1.0, K) + rng.uniform(-0.2, 0.2, K) / K)[::-1] * 7.0
    Q, _ = np.linalg.qr(rng.standard_normal((K, K)))
    T = (Q * lam) @ Q.T
    T = (T + T.T) / 2
    theta, Y = pkg.sym_eig(torch.tensor(T, device=DEV))
    torch.cuda.synchronize()
    th = theta.cpu().numpy()
    Yn = Y.double().cpu().numpy()
    nT = np.abs(lam).max()
    assert np.max(np.abs(th - lam)) <= 1e-11 * nT, np.max(np.abs(th - lam)) / nT
    assert np.linalg.norm(T @ Yn - Yn * th, axis=0).max() <= 2e-6 * nT


def _spectrum(n, npos, seed, gap=0.3):
    rng = np.random.default_rng(seed)
    pos = np.sort(rng.uniform(1.0, 10.0, npos))[::-1]
    neg = -np.sort(rng.uniform(0.1, 40.0, n - npos))
    lam = np.concatenate([pos, neg])
    return lam


@pytest.mark.parametrize("n,r,npos", [(50, 5, 10), (127, 8, 8), (129, 8, 20), (300, 8, 30), (777, 16, 24),
                                      (1000, 32, 40), (2000, 8, 12), (2000, 16, 64), (2000, 60, 70),
                                      (5000, 16, 24), (2000, 64, 80), (3000, 64, 80)])
def test_aproj_known_spectrum(pkg, n, r, npos):
    lam = _spectrum(n, npos, seed=n + r)
    # separate lambda_r from lambda_{r+1} by a relative gap so the truncation is unique
    lam[:r] += 0.5
    S, Q, lam = si.random_symmetric_with_spectrum(n, lam, seed=n)
    order = np.argsort(-lam)
    Pref = (Q[:, order[:r]] * np.maximum(lam[order[:r]], 0)) @ Q[:, order[:r]].T
    P, V, lg, info = pkg.aproj(torch.tensor(S, dtype=torch.float32, device=DEV), r)
    torch.cuda.synchronize()
    err = np.linalg.norm(P.double().cpu().numpy() - Pref) / np.linalg.norm(Pref)
    assert err <= 1e-5, (err, info.as_dict())
    np.testing.assert_allclose(lg.cpu().numpy(), np.sort(lam)[::-1][:r], rtol=1e-5, atol=1e-5 * np.abs(lam).max())


def test_aproj_negative_definite_gives_zero(pkg):
    n = 300
    lam = -np.linspace(0.5, 10, n)
    S, _, _ = si.random_symmetric_with_spectrum(n, lam, seed=1)
    P, V, lg, info = pkg.aproj(torch.tensor(S, dtype=torch.float32, device=DEV), 4)
    torch.cuda.synchronize()
    assert float(P.abs().max()) == 0.0
    assert np.all(lg.cpu().numpy() < 0)


# ---------------------------------------------------------------------------
# one iteration of Alg. 2 from a shared iterate
# ---------------------------------------------------------------------------

def _shared_iterate(inst, r, iters):
    prob = Problem.from_instance(inst)
    res = oracle.solve(prob, mode="lr", tol=1e-12, rank_init=r, max_iter=iters, max_rank=r)
    lam_x, U = np.linalg.eigh(res.X)
    return prob, U[:, ::-1][:, :r].copy(), lam_x[::-1][:r].copy(), res.y_paper


@pytest.mark.parametrize("form", [0, 1], ids=["explicit", "factored"])
@pytest.mark.parametrize("kind,n,r", [("maxcut", 200, 4), ("maxcut", 90, 6), ("equi", 160, 8), ("sensor", 0, 8),
                                      ("workload", 2000, 16), ("maxcut", 400, 64)])
def test_one_iteration_matches_oracle(pkg, kind, n, r, form):
    """form 1 applies S^k from the factors of X^k (n > 128; n = 90 takes the
    dense eigensolver, which always forms S)."""
    if kind == "maxcut":
        inst = si.maxcut_er(n, 0.05, 3)
    elif kind == "equi":
        rng = np.random.default_rng(7)
        ei, ej = si.erdos_renyi(n, 0.05, rng)
        inst = si.equipartition(n, ei, ej, np.ones(ei.shape[0]))
    elif kind == "workload":  # the n = 2000 MaxCut workload (weights 1..5, seed 1)
        inst = si.config_maxcut_2000()
    else:
        inst = si.sensor_network(140, 6, 0.3, seed=5)
    prob, Vx, lx, yp = _shared_iterate(inst, r, 25)
    sp, scale = normalize_rows(prob)
    slv = pkg.Solver(rank_init=r, max_rank=r, lanczos_tol=1e-6, lanczos_max_cycles=30, operator_form=form)
    slv.set_instance(inst)
    if form == 1 and r > 60:
        # the factored operator holds at most 60 factors: rejected, not run
        with pytest.raises(pkg.ProxSDPError) as e:
            slv.set_iterate(Vx, lx, yp)
        assert e.value.code == pkg.ERR_UNSUPPORTED
        slv.close()
        return
    slv.set_iterate(Vx, lx, yp)
    info = slv.iterate(1)
    got = slv.get_primal_dual()
    X0 = (Vx * np.maximum(lx, 0)) @ Vx.T
    st = pd_iteration(sp, X0, -yp / scale, info.alpha, r)
    ex = np.linalg.norm(got["X"] - st.X) / np.linalg.norm(st.X)
    assert ex <= 1e-4, ex
    y_ref = -st.y * scale
    ey = np.linalg.norm(got["y"] - y_ref) / max(np.linalg.norm(y_ref), 1e-12)
    assert ey <= 1e-4, ey
    assert abs(info.eps_primal - st.eps_primal) <= 1e-3 * st.eps_primal + 1e-6
    assert abs(info.eps_dual - st.eps_dual) <= 1e-3 * st.eps_dual + 1e-6
    assert abs(info.lambda_r - st.lam_desc[r - 1]) <= 1e-4 * abs(st.lam_desc[0])
    slv.close()


# ---------------------------------------------------------------------------
# full solves
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,graph,tol", [(5, "K", 1e-6), (6, "K", 1e-6), (7, "C", 1e-6), (64, "C", 1e-6),
                                         (16, "K", 1e-6), (100, "K", 1e-6), (101, "C", 5e-5)])
def test_maxcut_closed_forms_small(pkg, n, graph, tol):
    """Dense projection path (n <= 128).  The 101-cycle converges slowly under
    PDHG (the FP64 oracle needs 35 649 iterations to 1e-4 and 164 457 to
    1e-5), so it runs at 5e-5: a relative gap tol bounds the objective error
    by about 2 tol (reading A21)."""
    ei, ej, w = si.complete_graph(n) if graph == "K" else si.cycle_graph(n)
    inst = si.maxcut(n, ei, ej, w)
    slv = pkg.Solver(tol=tol, rank_init=1, max_iter=400000)
    slv.set_instance(inst)
    info = slv.solve()
    if graph == "K":
        want = -n * n / 4.0
    else:
        want = -(n / 2.0) * (1 + math.cos(math.pi / n)) if n % 2 else -float(n)
    assert info.status == pkg.CONVERGED, info.as_dict()
    assert abs(info.primal_obj - want) <= 1e-4 * abs(want)
    slv.close()


@pytest.mark.parametrize("n", [201])
def test_maxcut_cycle_closed_form_lanczos_path(pkg, n):
    """An odd cycle with n > 128 (block Krylov path): the MaxCut SDR (Sec. 1.4)
    of C_n has the value -(n/2)(1 + cos(pi/n)) for odd n.  Solved to 5e-5 so
    that the objective is within 1e-4 (reading A21)."""
    ei, ej, w = si.cycle_graph(n)
    inst = si.maxcut(n, ei, ej, w)
    slv = pkg.Solver(tol=5e-5, rank_init=2, max_iter=400000)
    slv.set_instance(inst)
    info = slv.solve()
    want = -(n / 2.0) * (1 + math.cos(math.pi / n)) if n % 2 else -float(n)
    assert info.status == pkg.CONVERGED, info.as_dict()
    assert abs(info.primal_obj - want) <= 1e-4 * abs(want), (info.primal_obj, want)
    slv.close()


def test_c1_full_projection_against_oracle(pkg):
    """PD-SDP (Alg. 1, exact projection every iteration) on the n = 100
    MaxCut instance (G(100, 0.1), seed 0) against the oracle's Alg. 1 at a
    tolerance ten times tighter, with the certificates of the GPU pair."""
    inst = si.config_maxcut_small()
    prob = Problem.from_instance(inst)
    ref = oracle.solve(prob, mode="full", tol=1e-7)
    assert ref.status == 0
    slv = pkg.Solver(tol=1e-6, full_eig=1, max_iter=200000)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    assert abs(info.primal_obj - ref.pobj) <= 1e-4 * abs(ref.pobj), (info.primal_obj, ref.pobj)
    got = slv.get_primal_dual()
    cert = oracle.certificates(prob, got["X"], -got["y"])
    assert cert["primal_eq"] <= 1e-4 and cert["rel_gap"] <= 1e-4 and cert["dual_min_eig_rel"] >= -1e-4, cert
    assert cert["x_min_eig_rel"] >= -1e-6
    slv.close()


@pytest.mark.parametrize("a,b,seed", [(70, 70, 3)])
def test_maxcut_bipartite_closed_form_lanczos_path(pkg, a, b, seed):
    """n = a + b > 128 (block Lanczos path).  On a bipartite graph the cut of
    the two sides takes every edge, and every term (1 - X_ij)/2 of the SDP
    objective is at most 1, so the SDP value is minus the number of edges
    (unit weights)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((a, b)) < 0.1
    ei, ej = np.nonzero(mask)
    ej = ej + a
    inst = si.maxcut(a + b, ei, ej, np.ones(ei.shape[0]))
    slv = pkg.Solver(tol=1e-5, rank_init=2, max_iter=100000)
    slv.set_instance(inst)
    info = slv.solve()
    want = -float(ei.shape[0])
    assert info.status == pkg.CONVERGED, info.as_dict()
    assert abs(info.primal_obj - want) <= 1e-4 * abs(want)
    slv.close()


@pytest.mark.parametrize("n,p,seed", [(150, 0.05, 1), (300, 0.03, 2)])
def test_maxcut_random_against_oracle(pkg, n, p, seed):
    inst = si.maxcut_er(n, p, seed, weights="int5")
    prob = Problem.from_instance(inst)
    ref = oracle.solve(prob, mode="lr", tol=1e-6, rank_init=8)
    slv = pkg.Solver(tol=1e-5, rank_init=8)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    assert abs(info.primal_obj - ref.pobj) <= 1e-4 * abs(ref.pobj)
    got = slv.get_primal_dual()
    # certificates on the row-scaled problem the iteration runs on (reading A6):
    # the dense row 11^T has ||A_i||_F = n, so its residual in the original
    # units is n times the scaled one
    sp, scale = oracle.normalize_rows(prob)
    cert = oracle.certificates(sp, got["X"], -got["y"] / scale)
    assert cert["primal_eq"] <= 1e-4 and cert["rel_gap"] <= 1e-4 and cert["dual_min_eig_rel"] >= -1e-4
    slv.close()


@pytest.mark.parametrize("form", [0, 1], ids=["explicit", "factored"])
def test_equipartition_dense_row(pkg, form):
    """Equipartition (Sec. 5.1) with the structured row tr(11^T X) = 0, n > 128
    (Lanczos path), against the oracle's LR-PD-SDP and its certificates.  The
    factored operator carries the 11^T term as a column of ones."""
    n = 140
    rng = np.random.default_rng(12)
    ei, ej = si.erdos_renyi(n, 0.06, rng)
    inst = si.equipartition(n, ei, ej, np.ones(ei.shape[0]))
    prob = Problem.from_instance(inst)
    # PDHG stalls on this instance above 1e-5 (the FP64 oracle is still at a
    # relative gap of 3.4e-5 after 100 000 iterations), so both sides stop at
    # 1e-4; each objective is then within about 2e-4 of the optimum, and so of
    # each other (reading A21).  The certificates below hold at 1e-4.
    ref = oracle.solve(prob, mode="lr", tol=1e-4, rank_init=16, max_iter=20000)
    assert ref.status == 0  # converged
    slv = pkg.Solver(tol=1e-4, rank_init=16, max_iter=100000, operator_form=form)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    assert abs(info.primal_obj - ref.pobj) <= 2e-4 * abs(ref.pobj), (info.primal_obj, ref.pobj)
    got = slv.get_primal_dual()
    # certificates on the row-scaled problem the iteration runs on (reading A6):
    # the dense row 11^T has ||A_i||_F = n, so its residual in the original
    # units is n times the scaled one
    sp, scale = oracle.normalize_rows(prob)
    cert = oracle.certificates(sp, got["X"], -got["y"] / scale)
    assert cert["primal_eq"] <= 1e-4 and cert["rel_gap"] <= 1e-4 and cert["dual_min_eig_rel"] >= -1e-4
    slv.close()


def test_inequality_rows(pkg):
    """MaxCut plus inequality rows X_0j <= 0.3: multipliers >= 0, rows satisfied, certificate."""
    n = 140
    base = si.maxcut_er(n, 0.06, 4)
    extra = 8
    ptr = np.concatenate([base.A_rowptr, base.A_rowptr[-1] + np.arange(1, extra + 1)])
    col = np.concatenate([base.A_col, si.svec_index(np.zeros(extra, int), np.arange(1, extra + 1))])
    val = np.concatenate([base.A_val, np.full(extra, 0.5)])
    rhs = np.concatenate([base.rhs, np.full(extra, 0.3)])
    slv = pkg.Solver(tol=1e-5, rank_init=8)
    slv.set_problem(n, n, ptr, col, val, rhs, C_idx=base.C_idx, C_val=base.C_val)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    got = slv.get_primal_dual()
    prob = Problem.from_arrays(n, n, ptr, col, val, rhs, C_idx=base.C_idx, C_val=base.C_val)
    ref = oracle.solve(prob, mode="lr", tol=1e-6, rank_init=8)
    assert abs(info.primal_obj - ref.pobj) <= 1e-4 * abs(ref.pobj)
    assert np.all(got["y"][n:] <= 1e-12)  # paper's sign: y_ineq <= 0
    cert = oracle.certificates(prob, got["X"], -got["y"])
    assert cert["primal_ineq"] <= 1e-4 and cert["rel_gap"] <= 1e-4
    slv.close()


def test_mimo_box_rows_small_against_oracle(pkg):
    """Sec. 5.3 MIMO SDR with the elementwise bounds -1 <= X_ij <= 1 as
    2 * 300 inequality rows (n = 25, dense projection), against the oracle."""
    inst = si.mimo(24, np.random.default_rng(5), box=True)
    prob = Problem.from_instance(inst)
    ref = oracle.solve(prob, mode="lr", tol=1e-6, rank_init=2, max_iter=200000)
    assert ref.status == 0
    slv = pkg.Solver(tol=1e-5, rank_init=2, max_iter=200000)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    assert abs(info.primal_obj - ref.pobj) <= 1e-4 * (1 + abs(ref.pobj))
    got = slv.get_primal_dual()
    assert np.all(got["y"][inst.m_eq:] <= 1e-12)  # paper's sign: y_ineq <= 0
    cert = oracle.certificates(prob, got["X"], -got["y"])
    assert cert["primal_ineq"] <= 1e-4 and cert["rel_gap"] <= 1e-4
    slv.close()


def test_mimo_box_rows_lanczos_path(pkg):
    """n = 151 (block Krylov path) with 2 * 11 325 box rows as CSR rows.  The
    bounds are implied by diag(X) = 1 and X psd (|X_ij| <= sqrt(X_ii X_jj)),
    so the optimum equals the one without them.  The box duals are
    degenerate and the stop test's relative gap closes slowly on them
    (reading A23), so the boxed run has a fixed budget and the checks are the
    objective against the box-free optimum, the residuals, y_ineq <= 0 and
    the primal feasibility, at 1e-4."""
    res = {}
    for box in (False, True):
        inst = si.mimo(150, np.random.default_rng(8), box=box)
        slv = pkg.Solver(tol=1e-5, rank_init=2, max_iter=100000 if box else 400000)
        slv.set_instance(inst)
        info = slv.solve()
        if box:
            assert info.status in (pkg.CONVERGED, pkg.MAX_ITER), info.as_dict()
            assert max(info.rel_primal_res, info.rel_dual_res) <= 1e-5, info.as_dict()
        else:
            assert info.status == pkg.CONVERGED, info.as_dict()
        res[box] = (info, slv.get_primal_dual(), inst)
        slv.close()
    p0, p1 = res[False][0].primal_obj, res[True][0].primal_obj
    assert abs(p1 - p0) <= 1e-4 * abs(p0), (p0, p1)
    info, got, inst = res[True]
    assert np.all(got["y"][inst.m_eq:] <= 1e-12)
    cert = oracle.certificates(Problem.from_instance(inst), got["X"], -got["y"])
    assert cert["primal_eq"] <= 1e-4 and cert["primal_ineq"] <= 1e-4, cert


def test_sensor_positions_small(pkg):
    """Exact distances, every pair in range (n = 12, dense projection): the SDR
    is exact, Z has rank 2 and its block holds the true positions."""
    inst = si.sensor_network(10, 4, 2.0, seed=2)
    slv = pkg.Solver(tol=1e-6, rank_init=4, max_iter=400000)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    Z = slv.get_primal_dual()["X"]
    slv.close()
    rmse = np.sqrt(np.mean((Z[:2, 2:].T - inst.meta["sensors"]) ** 2))
    assert rmse < 1e-3, rmse
    lam = np.linalg.eigvalsh(Z)[::-1]
    assert lam[2] < 1e-3 * lam[0]


def test_sensor_positions_lanczos_path(pkg):
    """130 sensors, 5 anchors, every pair in range (n = 132, block Krylov path),
    20 000 iterations: the FP64 oracle's LR-PD-SDP reaches position RMSE 5.9e-4
    and rank 2 after the same count, so the GPU iterate must recover the
    positions to 2e-3 with a rank-2 Z."""
    inst = si.sensor_network(130, 5, 2.0, seed=4)
    slv = pkg.Solver(tol=1e-6, rank_init=4, max_iter=20000)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status in (pkg.CONVERGED, pkg.MAX_ITER), info.as_dict()
    Z = slv.get_primal_dual()["X"]
    slv.close()
    rmse = np.sqrt(np.mean((Z[:2, 2:].T - inst.meta["sensors"]) ** 2))
    assert rmse < 2e-3, rmse
    lam = np.linalg.eigvalsh(Z)[::-1]
    assert lam[2] < 1e-3 * lam[0]


# ---------------------------------------------------------------------------
# the n = 2000 MaxCut workload (weights 1..5), certified at full size
# ---------------------------------------------------------------------------

GOLDEN_C2 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_oracle.json")


@pytest.mark.parametrize("form", [0, 1], ids=["explicit", "factored"])
def test_maxcut_2000_objective_against_stored_oracle(pkg, form):
    """The bench workload as the bench runs it (tol 1e-4): objective within
    1e-4 relative of the FP64 oracle's solve to 1e-5 (``golden/c2_oracle.json``,
    written by ``golden/make_c2_oracle.py`` from ``oracle/`` alone)."""
    gold = json.load(open(GOLDEN_C2))
    assert gold["status"] == 0 and gold["tol"] <= 1e-5
    inst = si.config_maxcut_2000()
    slv = pkg.Solver(tol=1e-4, rank_init=8, block_size=16, operator_form=form)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    assert abs(info.primal_obj - gold["pobj"]) <= 1e-4 * abs(gold["pobj"]), (info.primal_obj, gold["pobj"])
    assert info.rel_gap <= 1e-4
    slv.close()


@pytest.mark.parametrize("form", [0, 1], ids=["explicit", "factored"])
def test_maxcut_2000_certified(pkg, form):
    """Run to 1e-5, the GPU pair certifies the optimum to 1e-4: primal
    feasibility, relative gap and dual feasibility (lambda_min(C + M*(y)))."""
    inst = si.config_maxcut_2000()
    slv = pkg.Solver(tol=1e-5, rank_init=8, block_size=16, operator_form=form)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    got = slv.get_primal_dual()
    prob = Problem.from_instance(inst)
    cert = oracle.certificates(prob, got["X"], -got["y"])
    assert cert["primal_eq"] <= 1e-4, cert
    assert cert["rel_gap"] <= 1e-4, cert
    assert cert["dual_min_eig_rel"] >= -1e-4, cert
    assert cert["x_min_eig_rel"] >= -1e-6, cert
    gold = json.load(open(GOLDEN_C2))
    assert abs(cert["pobj"] - gold["pobj"]) <= 1e-4 * abs(gold["pobj"])
    slv.close()


# ---------------------------------------------------------------------------
# error handling at the boundary
# ---------------------------------------------------------------------------

def test_invalid_inputs_rejected(pkg):
    slv = pkg.Solver()
    with pytest.raises(pkg.ProxSDPError) as e:
        slv.set_problem(4, 1, [0, 1], [99], [1.0], [1.0], C_idx=[0], C_val=[1.0])  # svec index out of range
    assert e.value.code == -1
    with pytest.raises(pkg.ProxSDPError) as e:
        slv.set_problem(4, 1, [0, 2, 1], [0, 2], [1.0, 1.0], [1.0, 1.0], C_idx=[0], C_val=[1.0])  # bad rowptr
    assert e.value.code == -1
    with pytest.raises(pkg.ProxSDPError) as e:
        slv.set_problem(4, 1, [0, 1], [0], [float("nan")], [1.0], C_idx=[0], C_val=[1.0])
    assert e.value.code == -1
    with pytest.raises(pkg.ProxSDPError) as e:
        slv.solve()  # no problem loaded
    assert e.value.code == -4
    slv.close()
