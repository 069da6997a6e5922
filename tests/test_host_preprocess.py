"""Host-side logic of the boundary, on CPU: input validation of set_problem
and the row-scaled operator norm / step size (readings A5, A6), checked against
the oracle's independent computation (a dense or sparse eigensolver on the
Gram matrix, where the library uses a power iteration)."""
import numpy as np
import pytest

import oracle
import sdp_instances as si
from oracle.sdp import Problem


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_05231_gb300 as p

    return p


def _analyze(pkg, inst, **kw):
    return pkg.analyze_problem(inst.n, inst.m_eq, inst.A_rowptr, inst.A_col, inst.A_val, inst.rhs,
                               C_dense=inst.C_dense, C_idx=inst.C_idx, C_val=inst.C_val, **kw)


def _oracle_norm(inst):
    sp, _ = oracle.normalize_rows(Problem.from_instance(inst))
    return oracle.operator_norm(sp)


@pytest.mark.parametrize("make", [
    lambda: si.maxcut_er(60, 0.1, 0),
    lambda: si.equipartition(50, *si.cycle_graph(50)),
    lambda: si.sensor_network(40, 5, 0.35, seed=3),
    lambda: si.mimo(12, np.random.default_rng(1)),
])
def test_operator_norm_and_step_match_oracle(pkg, make):
    inst = make()
    out = _analyze(pkg, inst)
    want = _oracle_norm(inst)
    assert abs(out["norm_M"] - want) <= 1e-8 * want
    assert abs(out["alpha"] - 0.95 / want) <= 1e-8 / want
    C = Problem.from_instance(inst).C
    assert abs(out["norm_C"] - np.linalg.norm(C)) <= 1e-10 * (1 + np.linalg.norm(C))


def test_union_pattern_size(pkg):
    inst = si.maxcut_er(80, 0.1, 2)
    out = _analyze(pkg, inst)
    # diagonal (constraints and C) plus one entry per edge
    assert out["n_union"] == 80 + len(inst.meta["edges"][0])


def test_random_rows_with_dense_row_and_duplicates(pkg):
    rng = np.random.default_rng(4)
    n, m = 12, 9
    rows = []
    for _ in range(m):
        k = rng.integers(1, 5)
        idx = si.svec_index(rng.integers(0, n, k), rng.integers(0, n, k))
        rows.append((idx, rng.standard_normal(k)))  # duplicates within a row are summed
    rows.append((np.array([-1]), np.array([0.5])))
    ptr = np.cumsum([0] + [len(c) for c, _ in rows])
    col = np.concatenate([c for c, _ in rows])
    val = np.concatenate([v for _, v in rows])
    rhs = rng.standard_normal(m + 1)
    out = pkg.analyze_problem(n, 4, ptr, col, val, rhs, C_dense=np.eye(n))
    prob = Problem.from_arrays(n, 4, ptr, col, val, rhs, C_dense=np.eye(n))
    sp, _ = oracle.normalize_rows(prob)
    want = oracle.operator_norm(sp)
    assert abs(out["norm_M"] - want) <= 1e-8 * want


@pytest.mark.parametrize("bad", ["index", "rowptr", "nan", "dense_not_alone", "meq", "c_idx", "asym"])
def test_malformed_input_is_rejected(pkg, bad):
    n = 4
    ptr, col, val, rhs = [0, 1, 2], [0, 2], [1.0, 1.0], [1.0, 1.0]
    kw = dict(C_idx=[0], C_val=[1.0])
    m_eq = 2
    if bad == "index":
        col = [0, 10]
    elif bad == "rowptr":
        ptr = [0, 2, 1]
    elif bad == "nan":
        val = [1.0, float("nan")]
    elif bad == "dense_not_alone":
        ptr, col, val = [0, 2, 3], [-1, 0, 2], [1.0, 1.0, 1.0]
    elif bad == "meq":
        m_eq = 3
    elif bad == "c_idx":
        kw = dict(C_idx=[99], C_val=[1.0])
    elif bad == "asym":
        C = np.eye(n)
        C[0, 1] = 1.0
        kw = dict(C_dense=C)
    with pytest.raises(pkg.ProxSDPError) as e:
        pkg.analyze_problem(n, m_eq, ptr, col, val, rhs, **kw)
    assert e.value.code == -1


@pytest.mark.parametrize("form,ok", [(0, True), (1, True), (2, True), (3, False), (-1, False)])
def test_operator_form_setting_validated(pkg, form, ok):
    inst = si.maxcut_er(30, 0.2, 1)
    s = pkg.default_settings(operator_form=form)
    if ok:
        _analyze(pkg, inst, settings=s)
    else:
        with pytest.raises(pkg.ProxSDPError) as e:
            _analyze(pkg, inst, settings=s)
        assert e.value.code == -1
