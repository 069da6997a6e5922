"""Seeded synthetic SDP instances shaped like the paper's case studies (Sec. 5).

This module only *builds problem data*: graphs, sensor layouts, channel
matrices, and the matrices ``C``, ``A_i`` and right-hand sides of the general
SDP form of Sec. 1.3.  It contains none of the solver's arithmetic, so the
oracle tests and the CUDA path can both draw their inputs from it.

Storage format (shared by the C ABI ``proxsdp_gpu_set_problem``):

* A symmetric matrix is given by entries of its packed upper triangle
  ("svec" index, no sqrt(2) scaling): entry ``(i, j)`` with ``0 <= i <= j < n``
  has index ``j*(j+1)/2 + i``; a value ``a`` there means ``A[i,j] = A[j,i] = a``.
* The constraint operator ``M = [A; G]`` (Sec. 2) is a CSR matrix whose rows
  are the matrices ``A_1..A_m`` (equalities, ``tr(A_i X) = b_i``) followed by
  ``G_1..G_p`` (inequalities, ``tr(G_j X) <= h_j``), each row listing svec
  entries.  ``rhs = [b; h]``.
* A row whose single entry has column index ``-1`` is a *structured dense row*:
  the matrix ``a * 11^T`` (every entry equal to the value ``a``), used for the
  equipartition constraint ``tr(11^T X) = 0`` (Sec. 5.1) so that it need not be
  stored as n(n+1)/2 entries.
* ``C`` is either sparse (svec entries) or a dense n x n array.

Recipes (numpy ``default_rng(seed)``):

* Erdos-Renyi G(n, p): one ``rng.random()`` per vertex pair ``i < j`` in
  row-major order; edge when the draw is ``< p``.
* MaxCut relaxation (Sec. 1.4): ``min -1/4 tr(L X)`` s.t. ``diag(X) = 1``.
* Equipartition relaxation (Sec. 5.1): ``min 1/4 tr(L X)`` s.t. ``diag(X)=1``,
  ``tr(11^T X) = 0``.
* Sensor localisation (Sec. 5.2, Eqs. dist_sensors / dist_anchors):
  ``Z = [[I_d, X], [X^T, Y]]``; the identity block is imposed by equalities.
* Binary MIMO detection (Sec. 5.3): ``min tr(L X)`` with
  ``L = [[H^T H, -H^T s], [-s^T H, s^T s]]`` and ``diag(X) = 1``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

DENSE_ROW = -1  # column index marking a structured all-equal (a * 11^T) row


def svec_index(i, j):
    """Packed upper-triangle index of entry (i, j) (either order)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    lo = np.minimum(i, j)
    hi = np.maximum(i, j)
    return hi * (hi + 1) // 2 + lo


def svec_unindex(idx):
    """Inverse of :func:`svec_index`: returns (i, j) with i <= j."""
    idx = np.asarray(idx, dtype=np.int64)
    j = ((np.sqrt(8.0 * idx.astype(np.float64) + 1.0) - 1.0) / 2.0).astype(np.int64)
    # guard against rounding in the square root
    j = np.where(j * (j + 1) // 2 > idx, j - 1, j)
    j = np.where((j + 1) * (j + 2) // 2 <= idx, j + 1, j)
    i = idx - j * (j + 1) // 2
    return i, j


@dataclass
class SDPProblem:
    """Data of ``min tr(CX)  s.t.  A(X) = b, G(X) <= h, X psd`` (Sec. 1.3)."""

    n: int
    m_eq: int
    A_rowptr: np.ndarray  # int64, m_total + 1
    A_col: np.ndarray  # int64 svec index, or DENSE_ROW
    A_val: np.ndarray  # float64
    rhs: np.ndarray  # float64, m_total ([b; h])
    C_idx: Optional[np.ndarray] = None  # int64 svec index (sparse C)
    C_val: Optional[np.ndarray] = None  # float64
    C_dense: Optional[np.ndarray] = None  # float64 n x n (dense C)
    meta: dict = field(default_factory=dict)

    @property
    def m_total(self) -> int:
        return int(self.rhs.shape[0])

    def c_dense(self) -> np.ndarray:
        """Dense symmetric C (for small instances and tests)."""
        if self.C_dense is not None:
            return np.array(self.C_dense, dtype=np.float64)
        C = np.zeros((self.n, self.n))
        if self.C_idx is not None and len(self.C_idx):
            i, j = svec_unindex(self.C_idx)
            C[i, j] = self.C_val
            C[j, i] = self.C_val
        return C


def _csr_from_rows(rows: List[tuple]) -> tuple:
    """rows: list of (svec_idx_array, value_array)."""
    ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    for k, (c, _) in enumerate(rows):
        ptr[k + 1] = ptr[k] + len(c)
    col = np.concatenate([np.asarray(c, dtype=np.int64) for c, _ in rows]) if rows else np.zeros(0, np.int64)
    val = np.concatenate([np.asarray(v, dtype=np.float64) for _, v in rows]) if rows else np.zeros(0)
    return ptr, col, val


def erdos_renyi(n: int, p: float, rng: np.random.Generator):
    """Edges (i, j), i < j, of G(n, p); pairs drawn in row-major order."""
    iu, ju = np.triu_indices(n, 1)
    draws = rng.random(iu.shape[0])
    keep = draws < p
    return iu[keep].astype(np.int64), ju[keep].astype(np.int64)


def erdos_renyi_rows(n: int, p: float, rng: np.random.Generator):
    """The same edges as ``erdos_renyi`` (same draws, same row-major order),
    drawn one row at a time so that large n needs O(n) memory per row."""
    ei, ej = [], []
    for i in range(n - 1):
        d = rng.random(n - 1 - i)
        j = np.nonzero(d < p)[0] + i + 1
        ei.append(np.full(j.shape[0], i, dtype=np.int64))
        ej.append(j.astype(np.int64))
    if not ei:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(ei), np.concatenate(ej)


def laplacian_svec(n: int, ei, ej, w):
    """Graph Laplacian as sparse svec entries (diagonal first, then edges)."""
    deg = np.zeros(n)
    np.add.at(deg, ei, w)
    np.add.at(deg, ej, w)
    d_idx = svec_index(np.arange(n), np.arange(n))
    e_idx = svec_index(ei, ej)
    return np.concatenate([d_idx, e_idx]), np.concatenate([deg, -np.asarray(w, dtype=np.float64)])


def _diag_rows(n: int):
    ptr = np.arange(n + 1, dtype=np.int64)
    col = svec_index(np.arange(n), np.arange(n))
    val = np.ones(n)
    return ptr, col, val


def maxcut(n: int, ei, ej, w, name: str = "maxcut") -> SDPProblem:
    """``min -1/4 tr(L X)`` s.t. ``diag(X) = 1`` (Goemans-Williamson relaxation)."""
    li, lv = laplacian_svec(n, ei, ej, w)
    ptr, col, val = _diag_rows(n)
    return SDPProblem(n=n, m_eq=n, A_rowptr=ptr, A_col=col, A_val=val, rhs=np.ones(n),
                      C_idx=li, C_val=-0.25 * lv,
                      meta=dict(kind=name, edges=(ei, ej), weights=np.asarray(w, dtype=np.float64)))


def equipartition(n: int, ei, ej, w) -> SDPProblem:
    """``min 1/4 tr(L X)`` s.t. ``diag(X) = 1``, ``tr(11^T X) = 0`` (Sec. 5.1)."""
    li, lv = laplacian_svec(n, ei, ej, w)
    ptr, col, val = _diag_rows(n)
    ptr = np.concatenate([ptr, [ptr[-1] + 1]])
    col = np.concatenate([col, [DENSE_ROW]])
    val = np.concatenate([val, [1.0]])
    rhs = np.concatenate([np.ones(n), [0.0]])
    return SDPProblem(n=n, m_eq=n + 1, A_rowptr=ptr, A_col=col, A_val=val, rhs=rhs,
                      C_idx=li, C_val=0.25 * lv,
                      meta=dict(kind="equipartition", edges=(ei, ej), weights=np.asarray(w, dtype=np.float64)))


def complete_graph(n: int):
    iu, ju = np.triu_indices(n, 1)
    return iu.astype(np.int64), ju.astype(np.int64), np.ones(iu.shape[0])


def cycle_graph(n: int):
    i = np.arange(n, dtype=np.int64)
    j = (i + 1) % n
    return np.minimum(i, j), np.maximum(i, j), np.ones(n)


def sensor_network(n_sensors: int, n_anchors: int, radius: float, seed: int, d: int = 2) -> SDPProblem:
    """Sensor network localisation SDR (Sec. 5.2), variable ``Z`` of size d + n_sensors.

    ``C = 0`` (the paper's problem is a feasibility problem).  The ``I_d`` block
    is imposed by ``d(d+1)/2`` equalities.  Distances are exact.
    """
    rng = np.random.default_rng(seed)
    sensors = rng.random((n_sensors, d))
    anchors = rng.random((n_anchors, d))
    n = d + n_sensors
    rows = []
    rhs = []
    for a in range(d):
        for b in range(a, d):
            rows.append((svec_index([a], [b]), [1.0]))
            rhs.append(1.0 if a == b else 0.0)
    # sensor-sensor pairs in range (i < j)
    diff = sensors[:, None, :] - sensors[None, :, :]
    dist2 = np.einsum("ijk,ijk->ij", diff, diff)
    si, sj = np.nonzero(np.triu(dist2 < radius * radius, 1))
    for i, j in zip(si, sj):
        pi, pj = d + i, d + j
        rows.append((svec_index([pi, pj, pi], [pi, pj, pj]), [1.0, 1.0, -1.0]))
        rhs.append(dist2[i, j])
    # anchor-sensor pairs in range
    da = anchors[:, None, :] - sensors[None, :, :]
    adist2 = np.einsum("kjl,kjl->kj", da, da)
    ak, aj = np.nonzero(adist2 < radius * radius)
    for k, j in zip(ak, aj):
        pj = d + j
        idx = [svec_index(0, 0)] + [svec_index(t, pj) for t in range(d)] + [svec_index(pj, pj)]
        val = [float(anchors[k] @ anchors[k])] + [-float(anchors[k, t]) for t in range(d)] + [1.0]
        rows.append((np.array(idx, dtype=np.int64).ravel(), val))
        rhs.append(adist2[k, j])
    ptr, col, val = _csr_from_rows(rows)
    return SDPProblem(n=n, m_eq=len(rhs), A_rowptr=ptr, A_col=col, A_val=val,
                      rhs=np.asarray(rhs, dtype=np.float64),
                      C_idx=np.zeros(0, np.int64), C_val=np.zeros(0),
                      meta=dict(kind="sensor", sensors=sensors, anchors=anchors, d=d,
                                n_ss=len(si), n_as=len(ak)))


def mimo(N: int, rng: np.random.Generator, snr_noise_var: float = 0.1, box: bool = False,
         box_u: float = 1.0) -> SDPProblem:
    """Binary least-squares (MIMO detection) SDR of Sec. 5.3: diag(X) = 1 and,
    with ``box``, the paper's elementwise bounds -u <= X_ij <= u (u = 1 there;
    ``box_u``) for i < j as 2 * n(n-1)/2 inequality rows (X_ij <= u, for the
    pairs in ``np.triu_indices(n, 1)`` order, then -X_ij <= u; the diagonal is
    fixed by the equality rows).  Each row holds one off-diagonal svec entry
    of value +-1/2, so tr(A X) = +-X_ij."""
    H = rng.normal(0.0, np.sqrt(1.0 / N), (N, N))
    x = rng.choice(np.array([-1.0, 1.0]), N)
    s = H @ x + rng.normal(0.0, np.sqrt(snr_noise_var), N)
    n = N + 1
    C = np.empty((n, n))
    C[:N, :N] = H.T @ H
    C[:N, N] = -(H.T @ s)
    C[N, :N] = C[:N, N]
    C[N, N] = s @ s
    ptr, col, val = _diag_rows(n)
    rhs = np.ones(n)
    if box:
        iu, ju = np.triu_indices(n, 1)
        k = iu.shape[0]
        cols = svec_index(iu, ju)
        col = np.concatenate([col, cols, cols])
        val = np.concatenate([val, np.full(k, 0.5), np.full(k, -0.5)])
        ptr = np.concatenate([ptr, ptr[-1] + np.arange(1, 2 * k + 1, dtype=np.int64)])
        rhs = np.concatenate([rhs, np.full(2 * k, float(box_u))])
    return SDPProblem(n=n, m_eq=n, A_rowptr=ptr, A_col=col, A_val=val, rhs=rhs,
                      C_dense=C, meta=dict(kind="mimo", H=H, x=x, s=s, box=box, box_u=box_u))


# ---------------------------------------------------------------------------
# The five workload configurations
# ---------------------------------------------------------------------------

def maxcut_er(n: int, p: float, seed: int, weights: str = "unit") -> SDPProblem:
    rng = np.random.default_rng(seed)
    ei, ej = erdos_renyi(n, p, rng)
    if weights == "unit":
        w = np.ones(ei.shape[0])
    else:  # integer weights 1..5, drawn in edge order after the graph
        w = rng.integers(1, 6, size=ei.shape[0]).astype(np.float64)
    prob = maxcut(n, ei, ej, w)
    prob.meta.update(seed=seed, p=p)
    return prob


def maxcut_er_streaming(n: int = 16384, p: float = 0.001, seed: int = 5) -> SDPProblem:
    """MaxCut of G(n, p) with unit weights, sized so that the n x n FP32
    primal-step input (1 GiB at n = 16384) is far larger than the L2 cache."""
    rng = np.random.default_rng(seed)
    ei, ej = erdos_renyi_rows(n, p, rng)
    prob = maxcut(n, ei, ej, np.ones(ei.shape[0]))
    prob.meta.update(seed=seed, p=p)
    return prob


def config_maxcut_small() -> SDPProblem:
    """MaxCut, G(100, 0.1), unit weights, seed 0 (full-eigendecomposition case)."""
    return maxcut_er(100, 0.1, 0)


def config_maxcut_2000() -> SDPProblem:
    """MaxCut, G(2000, 0.01), weights uniform in {1..5}, seed 1."""
    return maxcut_er(2000, 0.01, 1, weights="int5")


def config_sensor_1000() -> SDPProblem:
    """Sensor network: 1000 sensors + 10 anchors in [0,1]^2, radius 0.2, seed 2."""
    return sensor_network(1000, 10, 0.2, seed=2)


def config_equipartition_5000() -> SDPProblem:
    """Equipartition, G(5000, 0.002), unit weights, seed 3."""
    rng = np.random.default_rng(3)
    ei, ej = erdos_renyi(5000, 0.002, rng)
    return equipartition(5000, ei, ej, np.ones(ei.shape[0]))


def config_mimo_batch(count: int = 256, seed: int = 4) -> List[SDPProblem]:
    """Batch of binary MIMO detection SDRs, N log-uniform in [32, 512], SNR 10 dB."""
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(np.log(32), np.log(512), count))).astype(int)
    return [mimo(int(N), rng) for N in sizes]


def random_symmetric_with_spectrum(n: int, eigenvalues, seed: int):
    """Q diag(lam) Q^T with Q from the QR of a seeded Gaussian matrix."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))
    lam = np.asarray(eigenvalues, dtype=np.float64)
    return (Q * lam) @ Q.T, Q, lam
