"""The factored operator (operator_form = OP_FACTORED): the projection applies
S^k = V Lambda_+ V^T - alpha (C + M*(y^k)) from the factors of X^k and the
sparse pattern, never forming S^k.

In exact arithmetic both operator forms give the same iterates; in FP32 the
products differ by rounding only, so from a shared iterate the two runs stay
within 1e-4 relative in X and y over tens of iterations (the same bound the
one-iteration parity test uses against the oracle), and converged solves
reach the same objective within the 1e-5 solve tolerance.  The n x n buffer
of S is not allocated (checked from the device's free memory).
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


def _shared_iterate(inst, r, iters):
    prob = Problem.from_instance(inst)
    res = oracle.solve(prob, mode="lr", tol=1e-12, rank_init=r, max_iter=iters, max_rank=r)
    lam_x, U = np.linalg.eigh(res.X)
    return U[:, ::-1][:, :r].copy(), lam_x[::-1][:r].copy(), res.y_paper


@pytest.mark.parametrize("kind", ["maxcut", "equi"])
def test_factored_iterates_follow_explicit(pkg, kind):
    if kind == "maxcut":
        inst = si.maxcut_er(260, 0.04, 5, weights="int5")
    else:
        rng = np.random.default_rng(9)
        ei, ej = si.erdos_renyi(200, 0.05, rng)
        inst = si.equipartition(200, ei, ej, np.ones(ei.shape[0]))
    r = 8
    Vx, lx, yp = _shared_iterate(inst, r, 20)
    out = []
    for form in (pkg.OP_EXPLICIT, pkg.OP_FACTORED):
        slv = pkg.Solver(rank_init=r, max_rank=r, lanczos_tol=1e-6, lanczos_max_cycles=30, operator_form=form)
        slv.set_instance(inst)
        slv.set_iterate(Vx, lx, yp)
        info = slv.iterate(40)
        out.append((info, slv.get_primal_dual()))
        slv.close()
    (ie, ge), (i_f, gf) = out
    ex = np.linalg.norm(gf["X"] - ge["X"]) / np.linalg.norm(ge["X"])
    ey = np.linalg.norm(gf["y"] - ge["y"]) / max(np.linalg.norm(ge["y"]), 1e-12)
    assert ex <= 1e-4 and ey <= 1e-4, (ex, ey)
    assert abs(i_f.primal_obj - ie.primal_obj) <= 1e-4 * abs(ie.primal_obj)
    # the explicit path counts one product per Krylov step, the factored path too
    assert i_f.matvecs == ie.matvecs or abs(i_f.matvecs - ie.matvecs) <= 0.1 * ie.matvecs


def test_factored_solve_with_rank_growth(pkg):
    """From rank 1 the rank rule doubles r; the factored operator must follow
    the factor count of the current iterate across each change."""
    inst = si.maxcut_er(400, 0.03, 11, weights="int5")
    res = []
    for form in (pkg.OP_EXPLICIT, pkg.OP_FACTORED):
        slv = pkg.Solver(tol=1e-5, rank_init=1, max_iter=100000, operator_form=form)
        slv.set_instance(inst)
        info = slv.solve()
        assert info.status == pkg.CONVERGED, (form, info.as_dict())
        res.append(info)
        slv.close()
    ie, i_f = res
    assert i_f.rank_changes >= 1
    assert abs(i_f.primal_obj - ie.primal_obj) <= 2e-5 * abs(ie.primal_obj)


def test_factored_skips_the_dense_buffer(pkg):
    n = 6000
    inst = si.maxcut_er(n, 0.002, 3)
    used = {}
    for form in (pkg.OP_EXPLICIT, pkg.OP_FACTORED):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        slv = pkg.Solver(tol=1e-4, rank_init=8, operator_form=form)
        slv.set_instance(inst)
        torch.cuda.synchronize()
        used[form] = free0 - torch.cuda.mem_get_info()[0]
        info = slv.iterate(20)
        assert np.isfinite(info.primal_obj) and np.isfinite(info.rel_primal_res)
        slv.close()
    s_bytes = n * ((n + 31) // 32 * 32) * 4
    assert used[pkg.OP_EXPLICIT] - used[pkg.OP_FACTORED] >= 0.9 * s_bytes, used


def test_auto_form_picks_factored_for_sparse_patterns(pkg):
    """AUTO takes the factored operator when the union pattern holds at most
    n^2/8 entries: same memory footprint as OP_FACTORED on a sparse MaxCut."""
    n = 4000
    inst = si.maxcut_er(n, 0.003, 4)
    used = {}
    for form in (pkg.OP_FACTORED, pkg.OP_AUTO):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        slv = pkg.Solver(tol=1e-4, rank_init=8, operator_form=form)
        slv.set_instance(inst)
        torch.cuda.synchronize()
        used[form] = free0 - torch.cuda.mem_get_info()[0]
        slv.close()
    assert abs(used[pkg.OP_AUTO] - used[pkg.OP_FACTORED]) < 0.1 * n * n * 4, used


def test_operator_form_out_of_range_rejected(pkg):
    with pytest.raises(pkg.ProxSDPError):
        pkg.Solver(operator_form=3)
