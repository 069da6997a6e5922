"""The element-wise box rows of Sec. 5.3 as a structured class: the per-entry
formulas that the library's box kernel applies, checked on the CPU against
the FP64 oracle's generic operators on the same bounds given as ordinary rows
(scaled to unit norm, as both sides run them).  Per pair i < j, with
s = sqrt(2) the row scale, u the bound and z = (2 X+ - X)_ij:
    y_up+ = max(0, y_up + alpha s (z - u)),  y_lo+ = max(0, y_lo - alpha s (z + u)),
the box part of M*(y) is s (y_up - y_lo) / 2 off the diagonal, and the box
rows' shares of eps_dual^2, <dy, M(dX)>, rhs^T y and ||M*(dy)||_F^2 are
    (dy_up/alpha - s dX_ij)^2 + (dy_lo/alpha + s dX_ij)^2,  s dX_ij (dy_up - dy_lo),
    s u (y_up + y_lo),  s^2 (dy_up - dy_lo)^2 / 2;
||M||_2^2 = max(||M_diag rows||^2, s^2) = 2."""
import numpy as np
import pytest

import oracle
import sdp_instances as si
from oracle.sdp import Problem, dual_prox, normalize_rows, operator_norm


def _psd(n, r, rng):
    V = rng.standard_normal((n, r))
    return V @ V.T / n


@pytest.mark.parametrize("u", [0.3, 1.0])
def test_box_dual_step_and_residual_shares_match_the_row_form(u):
    rng = np.random.default_rng(11)
    N = 9
    rows = si.mimo(N, np.random.default_rng(4), box=True, box_u=u)
    prob, scale = normalize_rows(Problem.from_instance(rows))
    n, m_eq = rows.n, rows.m_eq
    iu, ju = np.triu_indices(n, 1)
    k = iu.shape[0]
    s = np.sqrt(2.0)
    assert np.allclose(scale[m_eq:], s)  # each box row has ||A||_F = 1/sqrt(2)
    alpha = 0.95 / operator_norm(prob)
    X, Xn = _psd(n, 3, rng), _psd(n, 3, rng)
    y = np.concatenate([rng.standard_normal(m_eq), np.maximum(rng.standard_normal(2 * k), 0.0)])
    # the oracle's dual step on the row form
    yn = dual_prox(y + alpha * prob.M.apply(2.0 * Xn - X), alpha, prob.rhs, m_eq)
    # the structured formulas
    z = (2.0 * Xn - X)[iu, ju]
    yu, yl = y[m_eq:m_eq + k], y[m_eq + k:]
    yun = np.maximum(0.0, yu + alpha * s * (z - u))
    yln = np.maximum(0.0, yl - alpha * s * (z + u))
    np.testing.assert_allclose(yn[m_eq:m_eq + k], yun, rtol=0, atol=1e-14)
    np.testing.assert_allclose(yn[m_eq + k:], yln, rtol=0, atol=1e-14)
    # the box rows' shares of the residual and objective sums
    dy = yn - y
    dX = Xn - X
    mdx = prob.M.apply(dX)
    box = slice(m_eq, None)
    ed2_rows = np.sum((dy[box] / alpha - mdx[box]) ** 2)
    du, dl = yun - yu, yln - yl
    dxij = dX[iu, ju]
    ed2_box = np.sum((du / alpha - s * dxij) ** 2 + (dl / alpha + s * dxij) ** 2)
    assert abs(ed2_rows - ed2_box) <= 1e-12 * max(1.0, ed2_rows)
    cross_rows = dy[box] @ mdx[box]
    assert abs(cross_rows - np.sum(s * dxij * (du - dl))) <= 1e-12 * max(1.0, abs(cross_rows))
    rhsy_rows = prob.rhs[box] @ yn[box]
    assert abs(rhsy_rows - np.sum(s * u * (yun + yln))) <= 1e-12 * max(1.0, abs(rhsy_rows))
    # M*(dy): the box part alone, and its share of ||M*(dy)||^2 (no overlap with the diagonal rows)
    dy_box_only = np.concatenate([np.zeros(m_eq), dy[box]])
    B = prob.M.adjoint(dy_box_only)
    Bs = np.zeros((n, n))
    Bs[iu, ju] = s * (du - dl) / 2.0
    Bs = Bs + Bs.T
    np.testing.assert_allclose(B, Bs, rtol=0, atol=1e-14)
    assert abs(np.sum(B * B) - np.sum(s * s * (du - dl) ** 2 / 2.0)) <= 1e-12 * max(1.0, np.sum(B * B))
    dy_rows_only = np.concatenate([dy[:m_eq], np.zeros(2 * k)])
    assert abs(np.sum(prob.M.adjoint(dy_rows_only) * B)) <= 1e-14  # diagonal vs off-diagonal: orthogonal
    # ||M||_2^2 of the row form: the box part of M*M is s^2 times the off-diagonal projection
    assert abs(operator_norm(prob) ** 2 - max(1.0, s * s)) <= 1e-10
