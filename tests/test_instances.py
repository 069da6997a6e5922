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


def test_mimo_batch():
    b = si.config_mimo_batch()
    assert len(b) == 256
    assert min(p.n for p in b) >= 33 and max(p.n for p in b) <= 513
    assert digest(b[0]) == "c230e79c95fda86f" and digest(b[-1]) == "09909b5ff08ac547"
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
