"""Pins of the oracle's smoothed L2 projection (M + L^2 K) eps_h = b.

* element matrices: the textbook 1D mass and stiffness of linear and
  quadratic elements, the element volume as the sum of the mass matrix and a
  zero stiffness row sum;
* the assembled operator equals its Kronecker-sum form built in numpy;
* Jacobi-PCG agrees with the exact fast-diagonalisation solve;
* a constant eps_q is reproduced exactly for any L^2; for L^2 = 0 any Q_k
  field is reproduced; the projection conserves sum_q w_q |J| eps_q."""
import numpy as np
import pytest

from oracle import oracle as O


def _kron3(A, B, C):
    return np.kron(C, np.kron(B, A))      # local node a fastest


def test_q1_element_matrix_textbook():
    h = np.array([0.5, 0.25, 2.0])
    M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    Me, Ke = O.element_matrices(1, h)
    V = h.prod()
    assert np.allclose(Me, V * _kron3(M1, M1, M1), rtol=0, atol=1e-15)
    want = (h[1] * h[2] / h[0] * _kron3(K1, M1, M1) + h[0] * h[2] / h[1] * _kron3(M1, K1, M1)
            + h[0] * h[1] / h[2] * _kron3(M1, M1, K1))
    assert np.allclose(Ke, want, rtol=0, atol=1e-14)


def test_q2_element_matrix_textbook():
    h = np.array([0.3, 0.7, 1.1])
    M1 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0
    K1 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0
    Me, Ke = O.element_matrices(2, h)
    assert np.allclose(Me, h.prod() * _kron3(M1, M1, M1), rtol=0, atol=1e-15)
    want = (h[1] * h[2] / h[0] * _kron3(K1, M1, M1) + h[0] * h[2] / h[1] * _kron3(M1, K1, M1)
            + h[0] * h[1] / h[2] * _kron3(M1, M1, K1))
    assert np.allclose(Ke, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_element_matrix_invariants(k):
    h = np.array([0.2, 0.3, 0.5])
    Me, Ke = O.element_matrices(k, h)
    assert abs(Me.sum() - h.prod()) < 1e-15
    assert np.max(np.abs(Ke.sum(axis=1))) < 1e-13
    assert np.allclose(Me, Me.T) and np.allclose(Ke, Ke.T)
    assert np.linalg.eigvalsh(Me).min() > 0
    assert np.linalg.eigvalsh(Ke).min() > -1e-13


@pytest.mark.parametrize("k", [1, 2, 3])
def test_apply_equals_kronecker_sum(k):
    m = O.Mesh([0.0, 1.0, -1.0], [0.3, 0.2, 0.5], [3, 2, 4], k)
    rng = np.random.default_rng(k)
    xv = rng.standard_normal(m.n_nodes())
    L2 = 0.01
    y = O.apply(m, L2, xv)
    z = O.kron_apply(m, L2, xv)
    assert np.max(np.abs(y - z)) <= 1e-13 * np.max(np.abs(z))
    dg = O.diag(m, L2)
    e = np.zeros(m.n_nodes())
    for j in rng.integers(0, m.n_nodes(), 5):
        e[:] = 0
        e[j] = 1
        assert abs(O.apply(m, L2, e)[j] - dg[j]) <= 1e-14 * dg[j]


@pytest.mark.parametrize("k,L2", [(1, 0.0), (1, 2e-3), (2, 0.0), (2, 5e-3), (3, 1e-3)])
def test_cg_matches_fast_diagonalisation(k, L2):
    m = O.Mesh([0.0, 0.0, 0.0], [0.3, 0.25, 0.4], [4, 3, 5], k)
    rng = np.random.default_rng(7 + k)
    eps_q = 0.4 + 0.6 * rng.random((m.n_elem, m.Q))
    b = O.rhs(m, eps_q)
    x, it, res = O.cg(m, L2, b, rtol=1e-14)
    assert it > 0 and res <= 1e-14
    y = O.fdm_solve(m, L2, b)
    assert np.max(np.abs(x - y)) <= 1e-12 * np.max(np.abs(y))


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("L2", [0.0, 3e-3])
def test_constant_reproduced_and_conserved(k, L2):
    m = O.Mesh([0.0, 0.0, 0.0], [0.2, 0.3, 0.25], [3, 4, 2], k)
    eps_q = np.full((m.n_elem, m.Q), 0.637)
    b = O.rhs(m, eps_q)
    x, it, res = O.cg(m, L2, b, rtol=1e-15)
    assert np.max(np.abs(x - 0.637)) < 1e-13
    rng = np.random.default_rng(3)
    eps_q = rng.random((m.n_elem, m.Q))
    b = O.rhs(m, eps_q)
    g, w = O.gauss_rule(m.nq)
    wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1) * m.elem_volume
    total = np.sum(eps_q * wq[None, :])
    assert abs(b.sum() - total) <= 1e-14 * total
    x, it, res = O.cg(m, L2, b, rtol=1e-15)
    mass = O.apply(m, 0.0, x).sum()                  # 1^T M eps_h
    assert abs(mass - total) <= 1e-12 * total


@pytest.mark.parametrize("k", [1, 2, 3])
def test_l2_zero_reproduces_qk_field(k):
    m = O.Mesh([0.1, 0.0, -0.2], [0.2, 0.3, 0.25], [3, 2, 4], k)
    f = lambda p: (1.0 + p[..., 0] ** k) * (2.0 - p[..., 1]) * (0.5 + p[..., 2] ** k)  # noqa: E731
    qp = O.quadrature_points(m)
    b = O.rhs(m, f(qp))
    x, it, res = O.cg(m, 0.0, b, rtol=1e-15)
    want = f(O.node_coords(m))
    assert np.max(np.abs(x - want)) < 1e-12 * np.max(np.abs(want))
