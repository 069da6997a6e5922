"""Plain FP64 oracle of the low-rank primal-dual SDP method.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Sections, equations and
algorithms cited below are those of "Exploiting Low-Rank Structure in
Semidefinite Programming by Approximate Operator Splitting" (Souto, Garcia,
Veiga).

Problem (Sec. 1.3, Eq. sdp_general)::

    minimize tr(C X)  s.t.  A(X) = b,  G(X) <= h,  X psd

with ``M = [A; G]`` (Sec. 2).  The iteration variable ``y`` is the multiplier
of ``M`` with the sign used by the algorithm (``y_ineq >= 0``); the paper's
dual variable of Sec. 1.3 is ``-y``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

DENSE_ROW = -1  # column index of a structured row ``a * 11^T``

# status codes (mirrored by the C ABI's proxsdp_gpu_status)
CONVERGED = 0
MAX_ITER = 1
STALLED_AT_MAX_RANK = 3


def svec_unpack(idx):
    """(i, j), i <= j, of packed upper-triangle indices ``j(j+1)/2 + i``."""
    idx = np.asarray(idx, dtype=np.int64)
    out_i = np.empty_like(idx)
    out_j = np.empty_like(idx)
    for k, v in enumerate(idx.ravel()):
        j = int(math.isqrt(8 * int(v) + 1) - 1) // 2
        out_j.ravel()[k] = j
        out_i.ravel()[k] = int(v) - j * (j + 1) // 2
    return out_i, out_j


class ConstraintOperator:
    """The linear operator ``M(X) = [tr(A_1 X); ...; tr(G_p X)]`` (Sec. 1.3).

    Built from CSR rows over packed upper-triangle ("svec") entries: an entry
    ``(i, j, a)`` puts ``a`` at both ``(i, j)`` and ``(j, i)`` of the row's
    symmetric matrix; a lone column index ``-1`` means the dense ``a * 11^T``.
    The adjoint is ``M*(y) = sum_i y_i A_i`` (Sec. 1.3).
    """

    def __init__(self, n, rowptr, col, val):
        self.n = int(n)
        self.rowptr = np.asarray(rowptr, dtype=np.int64)
        self.col = np.asarray(col, dtype=np.int64)
        self.val = np.asarray(val, dtype=np.float64)
        self.m = self.rowptr.shape[0] - 1
        self.row_of_entry = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        self.dense_rows = {}  # row -> a  (matrix a * 11^T)
        sparse = self.col >= 0
        for e in np.nonzero(~sparse)[0]:
            self.dense_rows[int(self.row_of_entry[e])] = float(self.val[e])
        self.ei, self.ej = svec_unpack(self.col[sparse])
        self.ea = self.val[sparse]
        self.erow = self.row_of_entry[sparse]

    def matrix(self, i):
        """Dense symmetric matrix of row ``i`` (the definition, for checks)."""
        A = np.zeros((self.n, self.n))
        if i in self.dense_rows:
            A[:, :] = self.dense_rows[i]
            return A
        sel = self.erow == i
        for p, q, a in zip(self.ei[sel], self.ej[sel], self.ea[sel]):
            A[p, q] = a
            A[q, p] = a
        return A

    def apply(self, X):
        """``M(X)_i = tr(A_i X)``, with ``tr(A X) = sum_pq A_pq X_pq``."""
        X = np.asarray(X, dtype=np.float64)
        out = np.zeros(self.m)
        # off-diagonal svec entries appear twice in the symmetric matrix
        weight = np.where(self.ei == self.ej, 1.0, 2.0)
        np.add.at(out, self.erow, weight * self.ea * X[self.ei, self.ej])
        for i, a in self.dense_rows.items():
            out[i] += a * X.sum()
        return out

    def adjoint(self, y):
        """``M*(y) = sum_i y_i A_i`` as a dense symmetric matrix."""
        y = np.asarray(y, dtype=np.float64)
        D = np.zeros((self.n, self.n))
        contrib = y[self.erow] * self.ea
        np.add.at(D, (self.ei, self.ej), contrib)
        off = self.ei != self.ej
        np.add.at(D, (self.ej[off], self.ei[off]), contrib[off])
        for i, a in self.dense_rows.items():
            D += y[i] * a
        return D

    def row_frobenius_norms(self):
        """``||A_i||_F`` of every row."""
        sq = np.zeros(self.m)
        weight = np.where(self.ei == self.ej, 1.0, 2.0)
        np.add.at(sq, self.erow, weight * self.ea ** 2)
        for i, a in self.dense_rows.items():
            sq[i] += a * a * self.n * self.n
        return np.sqrt(sq)

    def scaled(self, s):
        """Operator with every row ``i`` multiplied by ``s[i]``."""
        out = ConstraintOperator.__new__(ConstraintOperator)
        out.__dict__.update(self.__dict__)
        out.val = self.val * s[self.row_of_entry]
        out.ea = self.ea * s[self.erow]
        out.dense_rows = {i: a * s[i] for i, a in self.dense_rows.items()}
        return out

    def weighted_rows(self):
        """Sparse ``B`` (m x n(n+1)/2) with ``<A_i, A_j>_F = (B B^T)_ij``.

        An off-diagonal svec entry stands for two equal matrix entries, so it
        carries the weight ``sqrt(2)``; a dense row ``a 11^T`` is expanded.
        """
        import scipy.sparse as sp
        ntri = self.n * (self.n + 1) // 2
        key = self.ej * (self.ej + 1) // 2 + self.ei
        data = self.ea * np.where(self.ei == self.ej, 1.0, math.sqrt(2.0))
        rows, cols, vals = [self.erow], [key], [data]
        if self.dense_rows:
            jj, ii = np.triu_indices(self.n)  # jj <= ii: (row, col) = (jj, ii)
            dkey = ii * (ii + 1) // 2 + jj
            dw = np.where(ii == jj, 1.0, math.sqrt(2.0))
            for i, a in self.dense_rows.items():
                rows.append(np.full(dkey.shape[0], i))
                cols.append(dkey)
                vals.append(a * dw)
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.m, ntri))


@dataclass
class Problem:
    """Problem data in the oracle's own dense-C form."""

    n: int
    C: np.ndarray  # dense symmetric n x n
    M: ConstraintOperator
    rhs: np.ndarray  # [b; h]
    m_eq: int

    @staticmethod
    def from_arrays(n, m_eq, rowptr, col, val, rhs, C_dense=None, C_idx=None, C_val=None):
        C = np.zeros((n, n))
        if C_dense is not None:
            C = np.array(C_dense, dtype=np.float64)
        elif C_idx is not None and len(C_idx):
            i, j = svec_unpack(C_idx)
            np.add.at(C, (i, j), C_val)
            off = i != j
            np.add.at(C, (j[off], i[off]), np.asarray(C_val)[off])
        return Problem(n=int(n), C=C, M=ConstraintOperator(n, rowptr, col, val),
                       rhs=np.asarray(rhs, dtype=np.float64), m_eq=int(m_eq))

    @staticmethod
    def from_instance(p):
        """From an object with the ``sdp_instances.SDPProblem`` fields."""
        return Problem.from_arrays(p.n, p.m_eq, p.A_rowptr, p.A_col, p.A_val, p.rhs,
                                   C_dense=p.C_dense, C_idx=p.C_idx, C_val=p.C_val)


def normalize_rows(prob: Problem):
    """Row-scaled copy of the problem: every ``(A_i, rhs_i)`` divided by ``||A_i||_F``.

    The scaled SDP has the same feasible set and objective (a reformulation,
    not a change of the method); the returned ``scale`` maps the scaled dual
    back: ``y_original = y_scaled * scale``.
    """
    norms = prob.M.row_frobenius_norms()
    norms = np.where(norms > 0, norms, 1.0)
    s = 1.0 / norms
    return Problem(n=prob.n, C=prob.C, M=prob.M.scaled(s), rhs=prob.rhs * s, m_eq=prob.m_eq), s


def operator_norm(prob: Problem):
    """``||M||_2``: square root of the largest eigenvalue of ``Gram_ij = <A_i, A_j>_F``."""
    B = prob.M.weighted_rows()
    G = (B @ B.T)
    if G.shape[0] <= 3000:
        lam_max = np.linalg.eigvalsh(G.toarray())[-1]
    else:
        import scipy.sparse.linalg as spla
        lam_max = spla.eigsh(G.tocsc(), k=1, which="LA", tol=1e-12)[0][0]
    return float(np.sqrt(max(lam_max, 0.0)))


# ---------------------------------------------------------------------------
# Resolvents (Sec. 2.3)
# ---------------------------------------------------------------------------

def proj_psd(S):
    """Euclidean projection onto the psd cone (Sec. 2.3.2): ``sum max(0, l_i) u_i u_i^T``."""
    lam, U = np.linalg.eigh(np.asarray(S, dtype=np.float64))
    return (U * np.maximum(lam, 0.0)) @ U.T


def aproj_psd(S, r):
    """Truncated projection of Sec. 3.1 (Eq. trunc_eig).

    Keeps the ``r`` algebraically largest eigenpairs ``lambda_1 >= ... >= lambda_r``
    and returns ``(sum_{i<=r} max(0, lambda_i) u_i u_i^T, lambda_desc, U_desc)``
    where ``lambda_desc`` / ``U_desc`` are all eigenpairs in descending order.
    """
    lam, U = np.linalg.eigh(np.asarray(S, dtype=np.float64))
    lam = lam[::-1]
    U = U[:, ::-1]
    r = int(min(r, lam.shape[0]))
    P = (U[:, :r] * np.maximum(lam[:r], 0.0)) @ U[:, :r].T
    return P, lam, U


def proj_box(u, b, h, m_eq):
    """Projection onto ``{=b} x {<=h}`` (Sec. 2.3.1): ``[b; min(u_2, h)]``."""
    u = np.asarray(u, dtype=np.float64)
    out = np.empty_like(u)
    out[:m_eq] = b
    out[m_eq:] = np.minimum(u[m_eq:], h)
    return out


def dual_prox(u, alpha, rhs, m_eq):
    """Resolvent of ``alpha * d I*`` via the extended Moreau decomposition (Eq. resolvent_1).

    ``(I + alpha dI*)^{-1}(u) = u - alpha * proj_box(u / alpha)``.
    """
    rhs = np.asarray(rhs, dtype=np.float64)
    return u - alpha * proj_box(u / alpha, rhs[:m_eq], rhs[m_eq:], m_eq)


# ---------------------------------------------------------------------------
# One iteration of Alg. 1 / Alg. 2 and the residuals of Sec. 2.2
# ---------------------------------------------------------------------------

@dataclass
class StepResult:
    X: np.ndarray
    y: np.ndarray
    eps_primal: float
    eps_dual: float
    lam_desc: np.ndarray  # eigenvalues of S in descending order
    S: np.ndarray


def pd_iteration(prob: Problem, X, y, alpha, r=None):
    """One primal-dual iteration (Alg. 1; Alg. 2 when ``r`` is given).

    Primal step  ``X+ = proj(X - alpha (M*(y) + C))`` (exact, or ``aproj(., r)``),
    dual part 1  ``y_half = y + alpha M(2 X+ - X)``,
    dual part 2  ``y+ = y_half - alpha proj_box(y_half / alpha)``,
    residuals (Sec. 2.2, Eq. comb_residual)::

        eps_primal = || (X+ - X)/alpha - M*(y+ - y) ||_F
        eps_dual   = || (y+ - y)/alpha - M(X+ - X) ||_2
    """
    S = X - alpha * (prob.M.adjoint(y) + prob.C)
    if r is None:
        lam, U = np.linalg.eigh(S)
        Xn = (U * np.maximum(lam, 0.0)) @ U.T
        lam_desc = lam[::-1]
    else:
        Xn, lam_desc, _ = aproj_psd(S, r)
    y_half = y + alpha * prob.M.apply(2.0 * Xn - X)
    yn = dual_prox(y_half, alpha, prob.rhs, prob.m_eq)
    eps_p = np.linalg.norm((Xn - X) / alpha - prob.M.adjoint(yn - y), "fro")
    eps_d = np.linalg.norm((yn - y) / alpha - prob.M.apply(Xn - X))
    return StepResult(X=Xn, y=yn, eps_primal=float(eps_p), eps_dual=float(eps_d),
                      lam_desc=lam_desc, S=S)


@dataclass
class SolveResult:
    X: np.ndarray
    y: np.ndarray  # algorithm sign, original (unscaled) units
    y_paper: np.ndarray  # the paper's dual variable of Sec. 1.3 (= -y)
    status: int
    iters: int
    rank: int
    pobj: float
    dobj: float
    rel_primal: float
    rel_dual: float
    rel_gap: float
    rank_path: list = field(default_factory=list)
    saved: list = field(default_factory=list)  # (iteration, r) of saved X_[r]
    history: list = field(default_factory=list)


def solve(prob_in: Problem, mode="lr", tol=1e-4, max_iter=100000, rank_init=8,
          window=100, alpha_frac=0.95, eps_lambda=None, max_rank=None,
          normalize=True, record_history=False):
    """PD-SDP (``mode="full"``, Alg. 1) or LR-PD-SDP (``mode="lr"``, Alg. 2).

    Readings of points the paper leaves open (each listed in the design notes):

    * start ``X = 0``, ``y = 0``;
    * rows scaled to unit Frobenius norm, ``alpha = alpha_frac / ||M||_2``
      (the step condition ``0 < alpha < 1/||M||_2`` of Sec. 2.2);
    * the inner loop of Alg. 2 ends when ``max(rel_primal, rel_dual) <= tol``; the
      solve stops there when, in addition, the rank is sufficient and
      ``rel_gap <= tol`` (otherwise it keeps iterating at the same rank), with
      ``rel_primal = eps_primal / (1 + ||C||_F)``,
      ``rel_dual = eps_dual / (1 + ||rhs||_2)`` and
      ``rel_gap = |pobj - dobj| / (1 + |pobj| + |dobj|)``,
      ``pobj = tr(C X)``, ``dobj = -rhs^T y``;
    * rank test of Alg. 2 with the squared error bound of Sec. 3.1:
      the rank is sufficient when ``r = n`` or
      ``sqrt(n - r) * max(lambda_r, 0) <= eps_lambda * max(1, ||X||_F)``;
    * on convergence with an insufficient rank the pair is saved as the
      feasible ``(X_[r], y_[r])`` and ``r <- 2r``; when the combined residual
      has not decreased over the last ``window`` iterations (evaluated only
      ``window`` iterations after the last rank change) the rank doubles if it
      is insufficient, otherwise the iteration continues at the same rank.
    """
    n = prob_in.n
    if normalize:
        prob, scale = normalize_rows(prob_in)
    else:
        prob, scale = prob_in, np.ones(prob_in.M.m)
    if eps_lambda is None:
        eps_lambda = tol
    if max_rank is None:
        max_rank = n
    alpha = alpha_frac / operator_norm(prob)
    normC = np.linalg.norm(prob.C, "fro")
    normrhs = np.linalg.norm(prob.rhs)
    X = np.zeros((n, n))
    y = np.zeros(prob.M.m)
    r = n if mode == "full" else min(int(rank_init), n)
    k_change = 0
    eps_hist = []
    rank_path, saved, history = [], [], []
    status = MAX_ITER
    rel_p = rel_d = rel_gap = float("inf")
    pobj = dobj = 0.0
    it = 0
    for it in range(1, max_iter + 1):
        step = pd_iteration(prob, X, y, alpha, None if mode == "full" else r)
        X, y = step.X, step.y
        pobj = float(np.sum(prob.C * X))
        dobj = float(-prob.rhs @ y)
        rel_p = step.eps_primal / (1.0 + normC)
        rel_d = step.eps_dual / (1.0 + normrhs)
        rel_gap = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
        eps_comb = step.eps_primal + step.eps_dual
        eps_hist.append(eps_comb)
        rank_path.append(r)
        lam_r = step.lam_desc[r - 1]
        normX = np.linalg.norm(X, "fro")
        rank_ok = (r >= n) or (math.sqrt(n - r) * max(lam_r, 0.0) <= eps_lambda * max(1.0, normX))
        if record_history:
            history.append(dict(it=it, r=r, rel_p=rel_p, rel_d=rel_d, rel_gap=rel_gap,
                                pobj=pobj, lam_r=float(lam_r)))
        converged = max(rel_p, rel_d) <= tol  # the inner-loop test of Alg. 2 (relative residuals)
        if converged and rank_ok:
            if rel_gap <= tol:
                status = CONVERGED
                break
        elif converged:  # Alg. 2: save the feasible pair, then double the target rank
            saved.append((it, r))
            if r >= max_rank:
                status = STALLED_AT_MAX_RANK
                break
            r = min(2 * r, n, max_rank)
            k_change = it
        elif it - k_change >= window and it - 1 - window >= 0 and eps_comb >= eps_hist[it - 1 - window]:
            # eps^{k - l} exists only once l iterates precede k: before that no stall
            if not rank_ok:
                if r >= max_rank:
                    status = STALLED_AT_MAX_RANK
                    break
                r = min(2 * r, n, max_rank)
                k_change = it
    y_orig = y * scale
    return SolveResult(X=X, y=y_orig, y_paper=-y_orig, status=status, iters=it, rank=r,
                       pobj=float(np.sum(prob_in.C * X)), dobj=float(-prob_in.rhs @ y_orig),
                       rel_primal=rel_p, rel_dual=rel_d, rel_gap=rel_gap,
                       rank_path=rank_path, saved=saved, history=history)


# ---------------------------------------------------------------------------
# Certificates (independent of the iteration)
# ---------------------------------------------------------------------------

def certificates(prob: Problem, X, y):
    """Optimality certificates of a primal-dual pair ``(X, y)`` (algorithm sign).

    Weak duality: for feasible ``X`` and ``y`` with ``C + M*(y) psd`` and
    ``y_ineq >= 0``, ``tr(CX) >= -rhs^T y``; a small gap certifies optimality.
    """
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    MX = prob.M.apply(X)
    b, h = prob.rhs[:prob.m_eq], prob.rhs[prob.m_eq:]
    eq_res = np.linalg.norm(MX[:prob.m_eq] - b) / (1.0 + np.linalg.norm(b))
    ineq_res = np.linalg.norm(np.maximum(MX[prob.m_eq:] - h, 0.0)) / (1.0 + np.linalg.norm(h))
    lam_X = np.linalg.eigvalsh(X)
    Z = prob.C + prob.M.adjoint(y)
    lam_Z = np.linalg.eigvalsh(Z)
    pobj = float(np.sum(prob.C * X))
    dobj = float(-prob.rhs @ y)
    return dict(
        primal_eq=float(eq_res),
        primal_ineq=float(ineq_res),
        x_min_eig_rel=float(lam_X[0] / max(1.0, np.abs(lam_X).max())),
        dual_min_eig_rel=float(lam_Z[0] / (1.0 + np.linalg.norm(prob.C, "fro"))),
        y_ineq_min=float(y[prob.m_eq:].min()) if y.shape[0] > prob.m_eq else 0.0,
        pobj=pobj,
        dobj=dobj,
        rel_gap=abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj)),
    )


# ---------------------------------------------------------------------------
# Brute force references for tiny instances
# ---------------------------------------------------------------------------

def brute_force_maxcut(n, ei, ej, w):
    """Maximum cut weight over ``x in {-1,1}^n`` (x_0 = 1), Sec. 5.1.

    The cut weight ``1/4 sum w_ij (1 - x_i x_j)`` of Sec. 5.1 runs over ordered
    vertex pairs (``w_ij = w_ji``), i.e. it is the total weight of the edges
    whose ends lie on different sides; each undirected edge ``(ei, ej)`` is
    therefore counted with ``1/2 w (1 - x_i x_j)``.
    """
    best = -np.inf
    ei = np.asarray(ei)
    ej = np.asarray(ej)
    w = np.asarray(w, dtype=np.float64)
    for code in range(1 << (n - 1)):
        x = np.ones(n)
        for k in range(n - 1):
            if (code >> k) & 1:
                x[k + 1] = -1.0
        val = 0.5 * np.sum(w * (1.0 - x[ei] * x[ej]))
        best = max(best, val)
    return float(best)


def brute_force_binary_ls(H, s):
    """``min_x ||H x - s||^2`` over ``x in {-1,1}^N``; returns (value, x)."""
    N = H.shape[1]
    best, best_x = np.inf, None
    for code in range(1 << N):
        x = np.array([1.0 if (code >> k) & 1 else -1.0 for k in range(N)])
        v = float(np.sum((H @ x - s) ** 2))
        if v < best:
            best, best_x = v, x
    return best, best_x
