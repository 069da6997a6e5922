"""Exit statuses and failure codes of a solve, made on the host (through the C ABI).

Each case reaches its status through the inputs or the settings only (an
iteration cap, a time cap, a rank cap, values that overflow FP32, a cap on
the handle's device memory); nothing here faults or stalls the GPU, and the
handle stays usable afterwards.  Also Alg. 2's saved feasible pair
(X_[r], y_[r]) of Sec. 3.2, which the rank rule keeps when the residuals
converge at an insufficient rank.
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


def _complete(n):
    return si.maxcut(n, *si.complete_graph(n))


def test_status_max_iter(pkg):
    inst = si.maxcut_er(300, 0.03, 2)
    for graphs in (1, 0):
        slv = pkg.Solver(max_iter=10, use_graphs=graphs, check_every=4)
        slv.set_instance(inst)
        info = slv.solve()
        assert info.status == pkg.MAX_ITER, info.as_dict()
        assert info.iters == 10
        slv.close()


def test_status_time_limit(pkg):
    inst = si.maxcut_er(300, 0.03, 2)
    slv = pkg.Solver(tol=1e-9, time_limit_s=1e-3, check_every=5)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.TIME_LIMIT, info.as_dict()
    assert 5 <= info.iters < 1000
    # the same handle solves normally afterwards
    slv2 = pkg.Solver(tol=1e-4)
    slv2.set_instance(inst)
    assert slv2.solve().status == pkg.CONVERGED
    slv.close()
    slv2.close()


@pytest.mark.parametrize("inst_kind", ["dense_path", "lanczos_path"])
def test_status_stalled_at_max_rank(pkg, inst_kind):
    """K_16 (optimum of rank 15) and G(300, 0.03) with the rank capped at 2:
    the rank test of Alg. 2 asks for r = 4, beyond the cap."""
    inst = _complete(16) if inst_kind == "dense_path" else si.maxcut_er(300, 0.03, 2)
    slv = pkg.Solver(tol=1e-6, rank_init=1, max_rank=2, max_iter=200000)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.STALLED_AT_MAX_RANK, info.as_dict()
    assert info.final_rank == 2
    got = slv.get_primal_dual()
    assert got["r"] <= 2
    slv.close()


@pytest.mark.parametrize("inst_kind", ["dense_path", "lanczos_path"])
def test_at_max_rank_keeps_iterating(pkg, inst_kind):
    """The same capped instances with settings.at_max_rank = 1: the solve
    stays at r = 2 and runs on instead of stopping.  Where it meets the stop
    test there (residuals and gap, the rank test waived at the cap) the pair
    is optimal: K_16 (n even) also has rank-1 optima, X = x x^T for any
    balanced +-1 vector x, and the value is the closed form n^2 / 4."""
    inst = _complete(16) if inst_kind == "dense_path" else si.maxcut_er(300, 0.03, 2)
    slv = pkg.Solver(tol=1e-6, rank_init=1, max_rank=2, max_iter=20000, at_max_rank=1)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status in (pkg.MAX_ITER, pkg.CONVERGED), info.as_dict()
    assert info.final_rank == 2
    if inst_kind == "dense_path":
        assert info.status == pkg.CONVERGED, info.as_dict()
        assert abs(info.primal_obj + 64.0) <= 1e-4 * 64.0, info.primal_obj
    slv.close()
    with pytest.raises(pkg.ProxSDPError) as e:
        pkg.Solver(at_max_rank=2)
    assert e.value.code == pkg.ERR_INVALID_ARG


def test_status_numeric_error(pkg):
    """C entries of 1e200 are finite in FP64 (accepted by set_problem) but
    overflow FP32 in S^k: the iteration reports NUMERIC_ERROR, and the handle
    still loads and solves a normal problem afterwards."""
    n = 60
    base = si.maxcut_er(n, 0.1, 5)
    slv = pkg.Solver(tol=1e-4, max_iter=2000, check_every=10)
    slv.set_problem(n, base.m_eq, base.A_rowptr, base.A_col, base.A_val, base.rhs, C_idx=base.C_idx,
                    C_val=np.asarray(base.C_val) * 1e200)
    info = slv.solve()
    assert info.status == pkg.NUMERIC_ERROR, info.as_dict()
    assert info.iters < 2000
    slv.set_instance(base)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    slv.close()


def test_status_out_of_memory_under_a_memory_cap(pkg):
    inst = si.config_maxcut_2000()
    slv = pkg.Solver(memory_limit_bytes=1 << 20)
    with pytest.raises(pkg.ProxSDPError) as e:
        slv.set_instance(inst)
    assert e.value.code == pkg.ERR_OOM
    with pytest.raises(pkg.ProxSDPError) as e:
        slv.solve()  # nothing was loaded
    assert e.value.code == pkg.ERR_BAD_STATE
    slv.close()
    # a cap above what the problem needs (S alone is 16 MB) lets it load and run
    slv = pkg.Solver(memory_limit_bytes=1 << 30, max_iter=20)
    slv.set_instance(inst)
    assert slv.solve().status == pkg.MAX_ITER
    slv.close()


def test_negative_memory_cap_rejected(pkg):
    with pytest.raises(pkg.ProxSDPError) as e:
        pkg.Solver(memory_limit_bytes=-1)
    assert e.value.code == pkg.ERR_INVALID_ARG


@pytest.mark.parametrize("n", [16, 7])
def test_saved_feasible_pair(pkg, n):
    """Rank 1 start on K_16 and on the 7-cycle: the oracle's Alg. 2 converges
    at r = 1 with an insufficient rank, saves (X_[1], y_[1]) and doubles r.
    The library keeps the last such pair; it is a psd iterate of at most the
    rank at which it was saved, feasible to the residual tolerance, and it
    precedes the final iterate."""
    inst = _complete(n) if n == 16 else si.maxcut(n, *si.cycle_graph(n))
    prob = Problem.from_instance(inst)
    ref = oracle.solve(prob, mode="lr", tol=1e-6, rank_init=1)
    assert ref.saved and ref.saved[0][1] == 1
    slv = pkg.Solver(tol=1e-6, rank_init=1)
    slv.set_instance(inst)
    info = slv.solve()
    assert info.status == pkg.CONVERGED, info.as_dict()
    assert info.rank_changes >= 1
    sv = slv.get_saved_pair()
    # the rank path is not pinned (it depends on FP32 vs FP64 trajectories):
    # the pair was saved at one of the ranks 1, 2, 4, ... below the final one
    assert 1 <= sv["r"] < info.final_rank and (sv["r"] & (sv["r"] - 1)) == 0
    assert 0 < sv["iter"] < info.iters
    cert = oracle.certificates(prob, sv["X"], -sv["y"])
    assert cert["primal_eq"] <= 1e-4, cert
    lam = np.linalg.eigvalsh(sv["X"])
    assert lam[0] >= -1e-6 * lam[-1]
    assert np.sum(lam > 1e-6 * lam[-1]) <= sv["r"]
    # a fresh solve that saves nothing reports BAD_STATE
    slv2 = pkg.Solver(tol=1e-4, rank_init=n)
    slv2.set_instance(inst)
    assert slv2.solve().status == pkg.CONVERGED
    with pytest.raises(pkg.ProxSDPError) as e:
        slv2.get_saved_pair()
    assert e.value.code == pkg.ERR_BAD_STATE
    slv.close()
    slv2.close()


@pytest.mark.parametrize("graphs", [1, 0])
def test_resume_after_interruption_follows_the_same_iterates(pkg, graphs):
    """An Alg. 2 run stopped after a fixed number of iterations and resumed
    reaches the stop test at the same iteration, rank and objective as the
    run without interruption (the iteration state stays on the device)."""
    inst = si.maxcut_er(300, 0.03, 2)
    ref = pkg.Solver(tol=1e-4, rank_init=2, check_every=10, use_graphs=graphs)
    ref.set_instance(inst)
    a = ref.solve()
    assert a.status == pkg.CONVERGED, a.as_dict()
    assert a.iters > 60
    slv = pkg.Solver(tol=1e-4, rank_init=2, check_every=10, use_graphs=graphs)
    slv.set_instance(inst)
    part = slv.iterate(a.iters // 3 + 7)
    assert part.status == pkg.MAX_ITER and part.iters == a.iters // 3 + 7
    b = slv.resume(5)  # a budget of five more iterations
    assert b.status == pkg.MAX_ITER and b.iters == part.iters + 5
    b = slv.resume()
    assert b.status == pkg.CONVERGED, b.as_dict()
    assert (b.iters, b.final_rank) == (a.iters, a.final_rank)
    assert b.primal_obj == a.primal_obj and b.dual_obj == a.dual_obj
    got, want = slv.get_primal_dual(), ref.get_primal_dual()
    np.testing.assert_array_equal(got["X"], want["X"])
    np.testing.assert_array_equal(got["y"], want["y"])
    # a converged iterate resumes to the stop test at once
    c = slv.resume()
    assert c.status == pkg.CONVERGED and c.iters - b.iters <= 1
    ref.close()
    slv.close()


def test_resume_from_saved_pair(pkg):
    """Restart Alg. 2 from its saved feasible pair (X_[r], y_[r]) of Sec. 3.2
    on a fresh handle (K_16, saved at r = 1): the run reaches the stop test at
    the optimum of the uninterrupted solve (objective within 1e-4,
    certificates at 1e-4)."""
    inst = _complete(16)
    slv = pkg.Solver(tol=1e-6, rank_init=1)
    slv.set_instance(inst)
    a = slv.solve()
    assert a.status == pkg.CONVERGED, a.as_dict()
    sv = slv.get_saved_pair()
    assert sv["r"] < a.final_rank
    res = pkg.Solver(tol=1e-6, rank_init=1)
    res.set_instance(inst)
    res.set_iterate(sv["V"], sv["lam"], sv["y"])
    b = res.resume()
    assert b.status == pkg.CONVERGED, b.as_dict()
    assert abs(b.primal_obj - a.primal_obj) <= 1e-4 * (1 + abs(a.primal_obj)), (a.primal_obj, b.primal_obj)
    got = res.get_primal_dual()
    cert = oracle.certificates(Problem.from_instance(inst), got["X"], -got["y"])
    assert cert["primal_eq"] <= 1e-4 and cert["rel_gap"] <= 1e-4, cert
    slv.close()
    res.close()


def test_resume_from_a_warm_start_on_the_block_lanczos_path(pkg):
    """G(300, 0.03): the leading half of a converged factorisation and its y
    as the starting iterate (set_iterate, rank r/2), then resume: Alg. 2 grows
    the rank back and stops at the optimum of the cold solve."""
    inst = si.maxcut_er(300, 0.03, 2)
    slv = pkg.Solver(tol=1e-5, rank_init=2)
    slv.set_instance(inst)
    a = slv.solve()
    assert a.status == pkg.CONVERGED, a.as_dict()
    got = slv.get_primal_dual(want_X=False)
    h = max(1, got["r"] // 2)
    res = pkg.Solver(tol=1e-5, rank_init=2)
    res.set_instance(inst)
    res.set_iterate(got["V"][:, :h], got["lam"][:h], got["y"])
    b = res.resume()
    assert b.status == pkg.CONVERGED, b.as_dict()
    assert abs(b.primal_obj - a.primal_obj) <= 1e-4 * (1 + abs(a.primal_obj)), (a.primal_obj, b.primal_obj)
    fin = res.get_primal_dual()
    cert = oracle.certificates(Problem.from_instance(inst), fin["X"], -fin["y"])
    assert cert["primal_eq"] <= 1e-4 and cert["rel_gap"] <= 1e-4, cert
    slv.close()
    res.close()


def test_resume_before_problem_is_bad_state(pkg):
    slv = pkg.Solver()
    with pytest.raises(pkg.ProxSDPError) as e:
        slv.resume()
    assert e.value.code == pkg.ERR_BAD_STATE
    slv.close()
