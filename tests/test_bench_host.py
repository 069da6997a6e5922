"""Host-side arithmetic of bench.py that the JSON line reports, on the CPU:
the algorithmic HBM bytes of the projection per iteration and the host
description beside the oracle's timing."""
import bench


def test_projection_hbm_formula():
    # q = 2.125 block products per iteration plus one rebuild, full n^2 FP32 entries
    out = bench.projection_hbm(2000, {"matvecs": 5051, "iters": 2377}, 1388.0, 6783.5)
    q = 5051 / 2377
    want = (q + 1.0) * 2000 * 2000 * 4.0
    assert out["bytes_per_iter"] == round(want)
    assert abs(out["achieved_gbs"] - round(want * 1388.0 / 1e9, 1)) < 1e-9
    assert abs(out["frac"] - round(want * 1388.0 / 1e9 / 6783.5, 4)) < 1e-12
    assert out["q_products_per_iter"] == round(q, 3)


def test_projection_hbm_no_iterations():
    out = bench.projection_hbm(100, {"matvecs": 0, "iters": 0}, 0.0, 6783.5)
    assert out["bytes_per_iter"] == 100 * 100 * 4 and out["achieved_gbs"] == 0.0


def test_host_description_fields():
    h = bench.host_description()
    assert set(h) == {"cpu", "nproc", "blas", "blas_threads"}
    assert isinstance(h["nproc"], int) and h["nproc"] >= 1
    assert h["cpu"]


def test_sweep_tables_and_paper_column():
    # every size printed in the paper's Table 2 / Table 3 has its reference seconds
    for kind, (_, sizes) in bench.SWEEPS.items():
        for n in sizes:
            assert n in bench.PAPER_SECONDS[kind]
    assert bench.PAPER_SECONDS["table3"][5000] == 472.4


def test_arpack_step_matches_oracle_step():
    """The ARPACK leg's iteration equals the oracle's Alg. 2 step (exact
    truncated projection) on a small MaxCut instance."""
    import numpy as np

    import oracle
    import sdp_instances as si
    from oracle.sdp import Problem, normalize_rows, operator_norm

    prob = Problem.from_instance(si.maxcut_er(60, 0.2, 1, weights="int5"))
    sp, _ = normalize_rows(prob)
    alpha = 0.95 / operator_norm(sp)
    X = np.zeros((60, 60))
    y = np.zeros(sp.M.m)
    v0 = np.ones(60)
    for _ in range(5):
        ref = oracle.pd_iteration(sp, X, y, alpha, 6)
        X, y, v0 = bench.arpack_step(sp, X, y, alpha, 6, v0)
        assert np.linalg.norm(X - ref.X) <= 1e-8 * max(1.0, np.linalg.norm(ref.X))
        assert np.linalg.norm(y - ref.y) <= 1e-8 * max(1.0, np.linalg.norm(ref.y))
