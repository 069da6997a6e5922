"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to a closed form, an identity, a library
routine used for a different purpose, a hand-worked example, or brute force,
chosen so that a dropped term, a wrong sign or index, or a transposed operand
in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle.sdp import ConstraintOperator, Problem, pd_iteration, svec_unpack
import sdp_instances as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# storage format and the constraint operator (Sec. 1.3)
# ---------------------------------------------------------------------------

def test_svec_unpack_matches_index_definition():
    n = 37
    for j in range(n):
        for i in range(j + 1):
            idx = j * (j + 1) // 2 + i
            pi, pj = svec_unpack([idx])
            assert (pi[0], pj[0]) == (i, j)


def _random_rows(n, m, rng, dense_row=True):
    rows = []
    for _ in range(m):
        k = rng.integers(1, 6)
        a = rng.integers(0, n, k)
        b = rng.integers(0, n, k)
        idx = np.unique(si.svec_index(a, b))
        rows.append((idx, rng.standard_normal(idx.shape[0])))
    if dense_row:
        rows.append((np.array([-1]), np.array([0.7])))
    ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    for k, (c, _) in enumerate(rows):
        ptr[k + 1] = ptr[k] + len(c)
    col = np.concatenate([c for c, _ in rows])
    val = np.concatenate([v for _, v in rows])
    return ptr, col, val


def test_constraint_operator_against_dense_trace_definition():
    rng = np.random.default_rng(11)
    n, m = 9, 12
    ptr, col, val = _random_rows(n, m, rng)
    M = ConstraintOperator(n, ptr, col, val)
    X = rng.standard_normal((n, n))
    X = X + X.T
    y = rng.standard_normal(M.m)
    # the definition: explicit dense symmetric A_i, tr(A_i X)
    mats = []
    for i in range(M.m):
        A = np.zeros((n, n))
        for e in range(ptr[i], ptr[i + 1]):
            if col[e] < 0:
                A[:, :] = val[e]
            else:
                p, q = svec_unpack([col[e]])
                A[p[0], q[0]] = val[e]
                A[q[0], p[0]] = val[e]
        mats.append(A)
    want = np.array([np.trace(A @ X) for A in mats])
    np.testing.assert_allclose(M.apply(X), want, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(M.adjoint(y), sum(yi * A for yi, A in zip(y, mats)), atol=1e-12)
    # adjointness <M(X), y> = <X, M*(y)>
    assert abs(M.apply(X) @ y - np.sum(X * M.adjoint(y))) < 1e-10
    # row norms
    np.testing.assert_allclose(M.row_frobenius_norms(), [np.linalg.norm(A) for A in mats], rtol=1e-13)


def test_operator_norm_against_svd_of_stacked_matrices():
    rng = np.random.default_rng(5)
    n, m = 7, 10
    ptr, col, val = _random_rows(n, m, rng)
    prob = Problem.from_arrays(n, m + 1, ptr, col, val, np.zeros(m + 1), C_dense=np.zeros((n, n)))
    stacked = np.stack([prob.M.matrix(i).ravel() for i in range(prob.M.m)])
    want = np.linalg.svd(stacked, compute_uv=False)[0]
    assert abs(oracle.operator_norm(prob) - want) < 1e-10 * want
    # diagonal-only constraints have orthonormal rows: ||M|| = 1
    p2 = Problem.from_instance(si.maxcut(6, *si.cycle_graph(6)))
    assert abs(oracle.operator_norm(p2) - 1.0) < 1e-12


def test_normalize_rows_keeps_feasible_set():
    rng = np.random.default_rng(3)
    n, m = 6, 8
    ptr, col, val = _random_rows(n, m, rng)
    rhs = rng.standard_normal(m + 1)
    prob = Problem.from_arrays(n, 4, ptr, col, val, rhs, C_dense=np.eye(n))
    sp, s = oracle.normalize_rows(prob)
    np.testing.assert_allclose(sp.M.row_frobenius_norms(), 1.0, rtol=1e-13)
    X = rng.standard_normal((n, n))
    X = X + X.T
    # A_i X - b_i scales by the same positive factor: same sign, same zero set
    np.testing.assert_allclose(sp.M.apply(X) - sp.rhs, s * (prob.M.apply(X) - prob.rhs), atol=1e-12)


# ---------------------------------------------------------------------------
# resolvents (Sec. 2.3) and the truncated projection (Sec. 3.1)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def known_spectrum():
    lam = np.array([5.0, 3.0, 2.5, 1.0, 0.4, 0.1, -0.2, -1.0, -3.0, -7.0, -20.0, -50.0])
    S, Q, lam = si.random_symmetric_with_spectrum(lam.shape[0], lam, seed=7)
    return S, Q, lam


def test_proj_psd_closed_form_and_cone_identities(known_spectrum):
    S, Q, lam = known_spectrum
    P = oracle.proj_psd(S)
    np.testing.assert_allclose(P, (Q * np.maximum(lam, 0)) @ Q.T, atol=1e-12)
    assert np.linalg.eigvalsh(P)[0] > -1e-12  # P psd
    assert np.linalg.eigvalsh(P - S)[0] > -1e-12  # P - S psd (polar cone)
    assert abs(np.sum(P * (P - S))) < 1e-10  # complementarity
    np.testing.assert_allclose(oracle.proj_psd(P), P, atol=1e-12)  # idempotent
    np.testing.assert_allclose(P - oracle.proj_psd(-S), S, atol=1e-12)  # Moreau for the cone


def test_aproj_picks_algebraically_largest_and_eym(known_spectrum):
    S, Q, lam = known_spectrum
    npos = int(np.sum(lam > 0))
    P_full = oracle.proj_psd(S)
    P, lam_desc, U = oracle.aproj_psd(S, npos)
    np.testing.assert_allclose(P, P_full, atol=1e-12)
    np.testing.assert_allclose(lam_desc, np.sort(lam)[::-1], atol=1e-12)
    for r in range(1, npos + 1):
        Pr, _, _ = oracle.aproj_psd(S, r)
        # the r largest *algebraic* eigenvalues (not the -50 / -20 of largest magnitude)
        np.testing.assert_allclose(Pr, (Q[:, :r] * lam[:r]) @ Q[:, :r].T, atol=1e-11)
        err2 = np.linalg.norm(P_full - Pr) ** 2
        # Eckart-Young-Mirsky, squared form: sum of the squared dropped positive eigenvalues
        assert abs(err2 - np.sum(np.maximum(lam[r:], 0) ** 2)) < 1e-10
        assert err2 <= (S.shape[0] - r) * max(lam[r - 1], 0) ** 2 + 1e-12
        assert np.linalg.eigvalsh(Pr)[0] > -1e-12


def test_box_resolvent_matches_prox_of_conjugate_by_numerical_minimisation():
    """Eq. resolvent_1: u - a proj(u/a) equals argmin_y a f*(y) + 1/2 ||y - u||^2,
    f the indicator of {=b} x {<=h}, so f*(y) = b^T y_1 + h^T y_2 on y_2 >= 0."""
    from scipy.optimize import minimize

    rng = np.random.default_rng(2)
    m_eq, p = 3, 4
    rhs = rng.standard_normal(m_eq + p)
    alpha = 0.37
    for _ in range(5):
        u = 2.0 * rng.standard_normal(m_eq + p)

        def obj(yv):
            return alpha * (rhs @ yv) + 0.5 * np.sum((yv - u) ** 2)

        bounds = [(None, None)] * m_eq + [(0.0, None)] * p
        res = minimize(obj, np.zeros_like(u), bounds=bounds, method="L-BFGS-B",
                       options=dict(ftol=1e-15, gtol=1e-12, maxiter=1000))
        np.testing.assert_allclose(oracle.dual_prox(u, alpha, rhs, m_eq), res.x, atol=1e-6)


def test_trace_resolvent_composition():
    """Eq. resolvent_2: prox of tr(C.) + I_psd at S is proj(S - alpha C); checked
    against direct numerical minimisation over X = L L^T for a 3 x 3 case."""
    from scipy.optimize import minimize

    rng = np.random.default_rng(4)
    n = 3
    S = rng.standard_normal((n, n)); S = S + S.T
    C = rng.standard_normal((n, n)); C = C + C.T
    alpha = 0.8
    want = oracle.proj_psd(S - alpha * C)

    def obj(v):
        L = v.reshape(n, n)
        X = L @ L.T
        return np.sum(C * X) + np.sum((X - S) ** 2) / (2 * alpha)

    best = None
    for trial in range(6):
        r = minimize(obj, rng.standard_normal(n * n), method="BFGS", options=dict(gtol=1e-10))
        if best is None or r.fun < best.fun:
            best = r
    L = best.x.reshape(n, n)
    np.testing.assert_allclose(L @ L.T, want, atol=1e-4)


# ---------------------------------------------------------------------------
# one iteration (Alg. 1) against hand-worked scalar cases
# ---------------------------------------------------------------------------

def test_scalar_iterations_match_hand_worked_golden():
    with open(os.path.join(GOLDEN, "scalar_steps.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        prob = Problem.from_arrays(1, c["m_eq"], [0, 1], [0], c["A"], c["rhs"], C_dense=[[c["C"]]])
        st = pd_iteration(prob, np.array([[c["X0"]]]), np.array(c["y0"]), c["alpha"])
        assert abs(st.S[0, 0] - c["S"]) < 1e-15, c["name"]
        assert abs(st.X[0, 0] - c["X1"]) < 1e-15, c["name"]
        np.testing.assert_allclose(st.y, c["y1"], atol=1e-15)
        assert abs(st.eps_primal - c["eps_primal"]) < 1e-15, c["name"]
        assert abs(st.eps_dual - c["eps_dual"]) < 1e-15, c["name"]


def test_optimal_pair_is_a_fixed_point_odd_cycle():
    """(X*, y*) of MaxCut on odd C_n (built from the spectrum of L) is left
    unchanged by Alg. 1 and by Alg. 2 at any rank >= 2, with zero residuals."""
    n = 9
    prob = Problem.from_instance(si.maxcut(n, *si.cycle_graph(n)))
    L = -4.0 * prob.C
    lam, U = np.linalg.eigh(L)
    top = U[:, -2:]
    Xs = (n / 2.0) * top @ top.T
    ys = np.full(n, lam[-1] / 4.0)
    np.testing.assert_allclose(np.diag(Xs), 1.0, atol=1e-12)
    for r in (None, 2, 3, 5):
        st = pd_iteration(prob, Xs, ys, 0.7, r)
        np.testing.assert_allclose(st.X, Xs, atol=1e-11)
        np.testing.assert_allclose(st.y, ys, atol=1e-11)
        assert st.eps_primal < 1e-9 and st.eps_dual < 1e-9


# ---------------------------------------------------------------------------
# closed-form optimal values (full solves)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [5, 6, 7, 16])
def test_maxcut_complete_graph_closed_form(n):
    prob = Problem.from_instance(si.maxcut(n, *si.complete_graph(n)))
    res = oracle.solve(prob, mode="full", tol=1e-8)
    assert res.status == 0
    assert abs(res.pobj - (-n * n / 4.0)) < 1e-6 * n * n


@pytest.mark.parametrize("n,mode", [(5, "full"), (7, "lr"), (6, "full"), (11, "lr"), (8, "lr")])
def test_maxcut_cycle_closed_form(n, mode):
    prob = Problem.from_instance(si.maxcut(n, *si.cycle_graph(n)))
    res = oracle.solve(prob, mode=mode, tol=1e-8, rank_init=1)
    want = -(n / 2.0) * (1.0 + math.cos(math.pi / n)) if n % 2 else -float(n)
    assert res.status == 0
    assert abs(res.pobj - want) < 1e-5 * abs(want)


@pytest.mark.parametrize("n,mode", [(64, "lr"), (101, "full")])
def test_maxcut_cycle_closed_form_larger(n, mode):
    """The cycle closed forms at n = 64 (even: n) and n = 101 (odd:
    (n/2)(1 + cos(pi/n))), tolerance 1e-6: Alg. 2 on the 64-cycle (about
    2 000 iterations), Alg. 1 on the 101-cycle (about 28 000 iterations,
    half a minute; PDHG approaches the odd-cycle optimum slowly)."""
    prob = Problem.from_instance(si.maxcut(n, *si.cycle_graph(n)))
    res = oracle.solve(prob, mode=mode, tol=1e-6, rank_init=1, max_iter=100000)
    want = -(n / 2.0) * (1.0 + math.cos(math.pi / n)) if n % 2 else -float(n)
    assert res.status == 0
    assert abs(res.pobj - want) < 1e-5 * abs(want)


@pytest.mark.parametrize("n", [6, 8])
def test_equipartition_closed_forms(n):
    ei, ej, w = si.complete_graph(n)
    res = oracle.solve(Problem.from_instance(si.equipartition(n, ei, ej, w)), mode="full", tol=1e-8)
    assert res.status == 0 and abs(res.pobj - n * n / 4.0) < 1e-5 * n * n
    ei, ej, w = si.cycle_graph(n)
    res = oracle.solve(Problem.from_instance(si.equipartition(n, ei, ej, w)), mode="full", tol=1e-8)
    want = (n / 2.0) * (1.0 - math.cos(2 * math.pi / n))
    assert res.status == 0 and abs(res.pobj - want) < 1e-5 * want


# ---------------------------------------------------------------------------
# brute force on tiny instances
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_maxcut_relaxation_brackets_brute_force(seed):
    n = 10
    rng = np.random.default_rng(100 + seed)
    ei, ej = si.erdos_renyi(n, 0.4, rng)
    w = rng.integers(1, 6, ei.shape[0]).astype(float)
    cut = oracle.brute_force_maxcut(n, ei, ej, w)
    res = oracle.solve(Problem.from_instance(si.maxcut(n, ei, ej, w)), mode="full", tol=1e-8)
    sdp = -res.pobj
    assert cut - 1e-6 <= sdp <= cut / 0.87856 + 1e-6


def test_maxcut_relaxation_exact_on_bipartite_graph():
    # complete bipartite K_{3,4}: the relaxation is tight (cut = all 12 edges)
    a = np.repeat(np.arange(3), 4)
    b = np.tile(np.arange(3, 7), 3)
    n = 7
    w = np.ones(a.shape[0])
    cut = oracle.brute_force_maxcut(n, a, b, w)
    assert cut == 12.0
    res = oracle.solve(Problem.from_instance(si.maxcut(n, a, b, w)), mode="full", tol=1e-9)
    assert abs(-res.pobj - cut) < 1e-5 * cut


def test_mimo_relaxation_bounds_brute_force():
    rng = np.random.default_rng(21)
    inst = si.mimo(8, rng)
    best, xbest = oracle.brute_force_binary_ls(inst.meta["H"], inst.meta["s"])
    res = oracle.solve(Problem.from_instance(inst), mode="full", tol=1e-9)
    assert res.pobj <= best + 1e-6 * (1 + best)
    lam = np.linalg.eigvalsh(res.X)
    if lam[-2] < 1e-4 * lam[-1]:  # rank-1 solution: the relaxation is exact (Sec. 5.3)
        assert abs(res.pobj - best) < 1e-4 * (1 + best)
        xs = np.sign(res.X[:-1, -1])
        np.testing.assert_array_equal(xs, xbest)


def test_mimo_box_rows_are_redundant():
    """The paper's MIMO SDR adds -1 <= X_ij <= 1 (Sec. 5.3).  With diag(X) = 1
    and X psd, |X_ij| <= sqrt(X_ii X_jj) = 1 already, so the bounds cut nothing:
    the optimum is the one without them.  The 2 n(n-1)/2 inequality rows keep
    non-negative multipliers (algorithm sign) and are satisfied."""
    no_box = Problem.from_instance(si.mimo(8, np.random.default_rng(5)))
    box = Problem.from_instance(si.mimo(8, np.random.default_rng(5), box=True))
    assert box.M.m == 9 + 2 * 36
    r0 = oracle.solve(no_box, mode="lr", tol=1e-7, rank_init=2, max_iter=200000)
    r1 = oracle.solve(box, mode="lr", tol=1e-7, rank_init=2, max_iter=200000)
    assert r0.status == 0 and r1.status == 0
    assert abs(r1.pobj - r0.pobj) <= 1e-5 * (1 + abs(r0.pobj))
    assert np.all(r1.y[box.m_eq:] >= 0.0)
    cert = oracle.certificates(box, r1.X, r1.y)
    assert cert["primal_ineq"] < 1e-6 and cert["rel_gap"] < 1e-5


@pytest.mark.parametrize("ns,na,radius,seed", [(8, 4, 2.0, 1), (10, 4, 2.0, 2), (12, 5, 0.9, 3)])
def test_sensor_positions_recovered_exactly(ns, na, radius, seed):
    """Sensor localisation (Sec. 5.2) with exact distances on a uniquely
    realisable network (every pair in range, or radius 0.9 in the unit square
    with 5 anchors): the SDR is exact, so the solution Z = [I X; X^T Y] has
    rank d = 2 and its block X holds the true sensor positions."""
    inst = si.sensor_network(ns, na, radius, seed=seed)
    res = oracle.solve(Problem.from_instance(inst), mode="full", tol=1e-8, max_iter=400000)
    assert res.status == 0
    pos = res.X[:2, 2:].T
    assert np.sqrt(np.mean((pos - inst.meta["sensors"]) ** 2)) < 1e-6
    lam = np.linalg.eigvalsh(res.X)[::-1]
    assert lam[2] < 1e-6 * lam[0] and lam[1] > 1e-2 * lam[0]


# ---------------------------------------------------------------------------
# certificates and the rank rule
# ---------------------------------------------------------------------------

def test_certificates_of_lr_solution_and_dual_sign():
    n = 24
    rng = np.random.default_rng(9)
    ei, ej = si.erdos_renyi(n, 0.3, rng)
    prob = Problem.from_instance(si.maxcut(n, ei, ej, np.ones(ei.shape[0])))
    res = oracle.solve(prob, mode="lr", tol=1e-7, rank_init=2)
    assert res.status == 0
    cert = oracle.certificates(prob, res.X, res.y)
    assert cert["primal_eq"] < 1e-5
    assert cert["x_min_eig_rel"] > -1e-8
    assert cert["dual_min_eig_rel"] > -1e-5
    assert cert["rel_gap"] < 1e-5
    # the paper's dual of Sec. 1.3: maximise b^T y_paper s.t. M*(y_paper) <= C
    Z = prob.C - prob.M.adjoint(res.y_paper)
    assert np.linalg.eigvalsh(Z)[0] > -1e-4
    assert abs(prob.rhs @ res.y_paper - res.pobj) < 1e-4 * (1 + abs(res.pobj))
    # exact solution agrees with the full-projection method
    full = oracle.solve(prob, mode="full", tol=1e-7)
    assert abs(full.pobj - res.pobj) < 1e-5 * abs(full.pobj)


def test_lr_rank_grows_past_solution_rank():
    """On odd C_n the optimum has rank 2; the rank test of Alg. 2 needs
    lambda_r <= 0, so LR-PD-SDP started at r = 1 must end with r > 2."""
    n = 9
    prob = Problem.from_instance(si.maxcut(n, *si.cycle_graph(n)))
    res = oracle.solve(prob, mode="lr", tol=1e-8, rank_init=1)
    assert res.status == 0 and res.rank >= 3
    assert res.rank_path[0] == 1 and sorted(set(res.rank_path)) == sorted(set(res.rank_path))
    assert np.linalg.matrix_rank(res.X, tol=1e-5 * np.abs(res.X).max()) == 2


def test_inequality_rows_keep_nonnegative_multipliers():
    """MaxCut with the redundant inequalities X_01 <= 0.5 and X_01 >= -2 (as -X_01 <= 2):
    multipliers of inequality rows stay >= 0 and the objective is unchanged when inactive."""
    n = 6
    base = si.maxcut(n, *si.cycle_graph(n))
    ptr = np.concatenate([base.A_rowptr, [n + 1, n + 2]])
    col = np.concatenate([base.A_col, [si.svec_index(0, 1), si.svec_index(0, 1)]])
    val = np.concatenate([base.A_val, [0.5, -0.5]])  # tr(A X) = X_01 (entry counted twice)
    rhs = np.concatenate([base.rhs, [0.5, 2.0]])
    prob = Problem.from_arrays(n, n, ptr, col, val, rhs, C_idx=base.C_idx, C_val=base.C_val)
    res = oracle.solve(prob, mode="full", tol=1e-8)
    assert res.status == 0
    assert np.all(res.y[n:] >= 0.0)
    assert res.X[0, 1] <= 0.5 + 1e-5
    cert = oracle.certificates(prob, res.X, res.y)
    assert cert["primal_ineq"] < 1e-5 and cert["rel_gap"] < 1e-5
