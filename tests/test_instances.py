"""The seeded workload generators are deterministic and have the documented
shapes (SHA-256 prefixes of the arrays pin the exact instances)."""
import hashlib

import numpy as np
import pytest

import sdp_instances as si


def digest(p):
    m = hashlib.sha256()
    for a in (p.A_rowptr, p.A_col, p.A_val, p.rhs):
        m.update(np.ascontiguousarray(a).tobytes())
    if p.C_dense is not None:
        m.update(np.ascontiguousarray(p.C_dense).tobytes())
    else:
        m.update(np.ascontiguousarray(p.C_idx).tobytes())
        m.update(np.ascontiguousarray(p.C_val).tobytes())
    return m.hexdigest()[:16]


@pytest.mark.parametrize("fn,n,m,nnz,c_nnz,h", [
    (si.config_maxcut_small, 100, 100, 100, 620, "2bfcd5c02960d8e5"),
    (si.config_maxcut_2000, 2000, 2000, 2000, 22155, "01672be68410f28f"),
    (si.config_sensor_1000, 1002, 52953, 159820, 0, "2f2f8951c91fd9ca"),
    (si.config_equipartition_5000, 5000, 5001, 5001, 29956, "7a73ea4f3e0edfaa"),
])
def test_workload_instances(fn, n, m, nnz, c_nnz, h):
    p = fn()
    assert p.n == n and p.m_total == m and len(p.A_col) == nnz
    assert len(p.C_idx) == c_nnz
    assert digest(p) == h


def draws_digest(p):
    """Hash of the seeded draws of a MIMO instance (H, x, noise) and its rows.
    C = [[H^T H, -H^T s], [-s^T H, s^T s]] is a BLAS product whose last bits
    depend on the BLAS thread count, so it is checked against its definition
    instead of hashed."""
    m = hashlib.sha256()
    for a in (p.A_rowptr, p.A_col, p.A_val, p.rhs, p.meta["H"], p.meta["x"], p.meta["s"]):
        m.update(np.ascontiguousarray(a).tobytes())
    return m.hexdigest()[:16]


def test_mimo_batch():
    b = si.config_mimo_batch()
    assert len(b) == 256
    assert min(p.n for p in b) >= 33 and max(p.n for p in b) <= 513
    assert draws_digest(b[0]) == "0b1d805e0e1b9e93" and draws_digest(b[-1]) == "e8b48226eb399730"
    for p in (b[0], b[-1]):
        H, s = p.meta["H"], p.meta["s"]
        N = H.shape[1]
        C = p.C_dense
        np.testing.assert_allclose(C[:N, :N], H.T @ H, rtol=0, atol=1e-12)
        np.testing.assert_allclose(C[:N, N], -(H.T @ s), rtol=0, atol=1e-12)
        assert abs(C[N, N] - s @ s) <= 1e-12 * (s @ s)
    p = b[0]
    N = p.n - 1
    H, x, s = p.meta["H"], p.meta["x"], p.meta["s"]
    # tr(L [x;1][x;1]^T) = ||H x - s||^2 (the lifting of Sec. 5.3)
    z = np.append(x, 1.0)
    assert abs(z @ p.C_dense @ z - np.sum((H @ x - s) ** 2)) < 1e-9 * (1 + np.sum((H @ x - s) ** 2))


def test_sensor_constraints_encode_distances():
    p = si.sensor_network(30, 4, 0.4, seed=1)
    d = 2
    X = p.meta["sensors"]
    Z = np.zeros((p.n, p.n))
    Z[:d, :d] = np.eye(d)
    Z[:d, d:] = X.T
    Z[d:, :d] = X
    Z[d:, d:] = X @ X.T
    # every row evaluated at the true lifted point equals its right-hand side
    for i in range(p.m_total):
        val = 0.0
        for e in range(p.A_rowptr[i], p.A_rowptr[i + 1]):
            a, b = si.svec_unindex(p.A_col[e])
            val += p.A_val[e] * (Z[a, b] if a == b else 2 * Z[a, b])
        assert abs(val - p.rhs[i]) < 1e-12


@pytest.mark.parametrize("n,p,seed", [(50, 0.2, 0), (300, 0.01, 3)])
def test_erdos_renyi_rows_matches_full_draw(n, p, seed):
    a = si.erdos_renyi(n, p, np.random.default_rng(seed))
    b = si.erdos_renyi_rows(n, p, np.random.default_rng(seed))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
