"""Batched solves (many independent SDPs of uneven size on one GPU): the MIMO
detection relaxation of Sec. 5.3 (diag(X) = 1, dense C), solved concurrently
through proxsdp_gpu_solve_batch.  Every kernel reduction has a fixed order, so
each instance must come out bit for bit as when it is solved alone; the small
instances are also checked against the oracle's LR-PD-SDP objective and its
optimality certificates."""
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


SIZES = [24, 47, 90, 140, 31, 200]


def _instances():
    rng = np.random.default_rng(21)
    return [si.mimo(N, rng) for N in SIZES]


def _solver(pkg, inst):
    s = pkg.Solver(tol=1e-4, rank_init=4, max_iter=200000)
    s.set_instance(inst)
    return s


def test_batch_equals_one_at_a_time_and_oracle(pkg):
    insts = _instances()
    solvers = [_solver(pkg, p) for p in insts]
    infos = pkg.solve_batch(solvers, host_threads=4)
    for inst, s, info in zip(insts, solvers, infos):
        assert info.status == pkg.CONVERGED, (inst.n, info.as_dict())
        alone = _solver(pkg, inst)
        ref = alone.solve()
        assert ref.iters == info.iters and ref.final_rank == info.final_rank
        assert ref.primal_obj == info.primal_obj and ref.rel_gap == info.rel_gap
        alone.close()
    for inst, s, info in list(zip(insts, solvers, infos))[:2]:  # N = 24, 47
        prob = Problem.from_instance(inst)
        want = oracle.solve(prob, mode="lr", tol=1e-7, rank_init=4)
        assert abs(info.primal_obj - want.pobj) <= 1e-4 * abs(want.pobj)
        got = s.get_primal_dual()
        cert = oracle.certificates(prob, got["X"], -got["y"])
        assert cert["primal_eq"] <= 1e-4 and cert["rel_gap"] <= 2e-4 and cert["dual_min_eig_rel"] >= -1e-4
    for s in solvers:
        s.close()


def test_batch_rejects_repeated_handles(pkg):
    s = _solver(pkg, _instances()[0])
    with pytest.raises(pkg.ProxSDPError) as e:
        pkg.solve_batch([s, s])
    assert e.value.code == -1
    s.close()
