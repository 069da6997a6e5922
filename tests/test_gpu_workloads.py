"""Whole solves of the larger synthetic workloads to the 1e-4 target, checked
with certificates that do not depend on the iteration (Sec. 1.3 duality):
primal feasibility on the row-scaled problem (reading A6), the relative
duality gap, and dual feasibility lambda_min(C + M*(y)) >= -1e-4 (1 + ||C||_F)
computed by a sparse Lanczos eigensolver (scipy) on the CPU.

- sensor network localisation, 1000 sensors + 10 anchors (Sec. 5.2): C = 0,
  exact distances (a slowly converging feasibility problem: progress check);
- graph equipartition with the structured row tr(11^T X) = 0 on G(5000, 0.002)
  (Sec. 5.1), the largest single-GPU configuration (n = 5000, S = 100 MB):
  progress and consistency checks (a full solve to 1e-4 takes minutes).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import sdp_instances as si
from oracle.sdp import Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_05231_gb300 as p

    return p


def _dual_min_eig(prob, y_alg):
    sla = pytest.importorskip("scipy.sparse.linalg")
    Z = prob.C + prob.M.adjoint(y_alg)
    lam = sla.eigsh(Z, k=1, which="SA", tol=1e-9, maxiter=20000, return_eigenvectors=False)[0]
    return float(lam) / (1.0 + np.linalg.norm(prob.C, "fro"))


def _scaled_checks(inst, got):
    prob = Problem.from_instance(inst)
    sp, scale = oracle.normalize_rows(prob)
    y_alg = -got["y"] / scale
    MX = sp.M.apply(got["X"])
    b = sp.rhs[: sp.m_eq]
    primal = np.linalg.norm(MX[: sp.m_eq] - b) / (1.0 + np.linalg.norm(b))
    pobj = float(np.sum(sp.C * got["X"]))
    dobj = float(-sp.rhs @ y_alg)
    gap = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
    return sp, y_alg, primal, gap, pobj


def test_sensor_network_1000(pkg):
    """The sensor relaxation (C = 0, a feasibility problem) converges slowly
    under PDHG (the FP64 oracle needs tens of thousands of iterations on a
    200-sensor instance as well), so the full-size run checks that 3000
    iterations proceed without numeric trouble and shrink the residuals;
    per-iteration parity with the oracle on this family is
    test_one_iteration_matches_oracle[sensor-0-8]."""
    inst = si.config_sensor_1000()
    slv = pkg.Solver(tol=1e-4, rank_init=8, max_iter=50000)
    slv.set_instance(inst)
    first = slv.iterate(300)
    assert first.status != pkg.NUMERIC_ERROR
    later = slv.iterate(2700)
    assert later.status != pkg.NUMERIC_ERROR, later.as_dict()
    assert later.rel_primal_res < first.rel_primal_res and later.rel_dual_res < first.rel_dual_res
    got = slv.get_primal_dual()
    assert np.all(np.isfinite(got["X"])) and np.all(np.isfinite(got["y"]))
    slv.close()


def test_equipartition_5000(pkg):
    """n = 5000 (S = 100 MB; the fused orthogonalisation falls back to the
    multi-kernel path at this size).  PDHG needs tens of thousands of
    iterations for 1e-4 here, so the test runs 7500 iterations and checks
    that the residuals shrink, that the objective the solver reports equals
    tr(C X) of the returned X (computed on the host from the instance), and
    that the returned iterate is finite and nearly feasible."""
    inst = si.config_equipartition_5000()
    slv = pkg.Solver(tol=1e-4, rank_init=8, max_iter=10**6)
    slv.set_instance(inst)
    first = slv.iterate(1500)
    assert first.status != pkg.NUMERIC_ERROR
    later = slv.iterate(6000)
    assert later.status != pkg.NUMERIC_ERROR, later.as_dict()
    assert later.rel_primal_res < first.rel_primal_res
    got = slv.get_primal_dual()
    X = got["X"]
    prob = Problem.from_instance(inst)
    pobj = float(np.sum(prob.C * X))
    assert abs(pobj - later.primal_obj) <= 1e-6 * (1.0 + abs(pobj))
    assert np.all(np.isfinite(got["lam"])) and np.all(np.isfinite(got["y"]))
    # constraint residual of the row-scaled problem (diag X = 1 and 1^T X 1 = 0)
    sp, _ = oracle.normalize_rows(prob)
    MX = sp.M.apply(X)
    feas = np.linalg.norm(MX[: sp.m_eq] - sp.rhs[: sp.m_eq]) / (1.0 + np.linalg.norm(sp.rhs[: sp.m_eq]))
    assert feas <= 1e-2, feas
    slv.close()


def test_equipartition_5000_to_1e4_at_the_rank_cap(pkg):
    """n = 5000 run to the 1e-4 stop test: Alg. 2's rank rule asks for
    r = 128 once r = 64 (the Lanczos path's cap) stalls; with
    settings.at_max_rank = 1 the solve keeps iterating at r = 64 and meets the
    residual and gap tests there (about 50 000 iterations).  The FP64 oracle's
    certificates of the returned pair, computed on the host from the
    instance, check it independently of the solver's own reductions: primal
    feasibility, the dual slack C + M*(y) (its smallest eigenvalue) and the
    gap."""
    inst = si.config_equipartition_5000()
    slv = pkg.Solver(tol=1e-4, rank_init=16, max_iter=10**6, time_limit_s=500.0, check_every=200, at_max_rank=1)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    assert info.final_rank == 64
    got = slv.get_primal_dual()
    slv.close()
    # on the row-scaled problem the iteration runs on (reading A6): the dense
    # row 11^T has ||A_i||_F = n, so its residual in the original units is n
    # times the scaled one
    sp, scale = oracle.normalize_rows(Problem.from_instance(inst))
    cert = oracle.certificates(sp, got["X"], -got["y"] / scale)
    print("certificates", cert)
    assert cert["primal_eq"] <= 1e-4, cert
    assert cert["rel_gap"] <= 2e-4, cert  # the stop test's gap (reading A21)
    assert cert["x_min_eig_rel"] >= -1e-6, cert
    assert cert["dual_min_eig_rel"] >= -1e-4, cert
