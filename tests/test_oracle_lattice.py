"""Pins of the oracle's lattice tables and moment basis (Sec. II).

Each check compares the oracle against something the paper or the
mathematics fixes, never against a retyped copy of the oracle's own code.
"""
import itertools

import numpy as np
import pytest

from tests import golden_io

LATS = ["D1Q3", "D2Q9", "D3Q19", "D2Q5"]


def _lat(orc, name):
    return getattr(orc, name)


@pytest.mark.parametrize("name", LATS)
def test_equilibrium_moments(orc, name):
    """f^0 = rho w_i must carry density rho, zero flux and rho theta delta
    (eqs. f0_0 - f0_2); odd third moments vanish by symmetry."""
    theta = 1.0 / 3.0
    D, Q, v, w = orc.lattice(_lat(orc, name), theta)
    assert abs(w.sum() - 1.0) < 1e-15
    for a in range(3):
        assert abs((w * v[:, a]).sum()) < 1e-15
        for b in range(3):
            expect = theta if (a == b and a < D) else 0.0
            assert abs((w * v[:, a] * v[:, b]).sum() - expect) < 1e-15
            for c in range(3):
                assert abs((w * v[:, a] * v[:, b] * v[:, c]).sum()) < 1e-15


@pytest.mark.parametrize("name,D,Q,speeds", [
    ("D1Q3", 1, 3, {0: 1, 1: 2}),
    ("D2Q9", 2, 9, {0: 1, 1: 4, 2: 4}),
    ("D3Q19", 3, 19, {0: 1, 1: 6, 2: 12}),
    ("D2Q5", 2, 5, {0: 1, 1: 4}),
])
def test_velocity_sets(orc, name, D, Q, speeds):
    """Each velocity set is the set of integer vectors of the named shells,
    closed under v -> -v, with no repeats."""
    d, q, v, w = orc.lattice(_lat(orc, name))
    assert (d, q) == (D, Q)
    assert len({tuple(x) for x in v}) == Q
    assert {tuple(x) for x in v} == {tuple(-x) for x in v}
    counts = {}
    for x in v:
        counts[int((x * x).sum())] = counts.get(int((x * x).sum()), 0) + 1
    assert counts == speeds
    assert np.all(v[:, D:] == 0)
    # weights depend only on |v|^2
    for s in speeds:
        ws = w[(v * v).sum(1) == s]
        assert np.ptp(ws) == 0.0


@pytest.mark.parametrize("name", LATS)
@pytest.mark.parametrize("theta", [1.0 / 3.0, 0.2, 0.45])
def test_basis_orthonormal(orc, name, theta):
    """sum_i m_i^a w_i m_i^b = delta^{ab}, m^0 = 1 (Sec. II); completeness
    sum_a m_i^a n_j^a = delta_ij with n_i^a = m_i^a w_i."""
    if name != "D2Q5" and theta != 1.0 / 3.0:
        pytest.skip("theta is free only for the D2Q5 lattice")
    lat = _lat(orc, name)
    D, Q, v, w = orc.lattice(lat, theta)
    m = orc.basis(lat, theta)
    assert np.max(np.abs(m[0] - 1.0)) < 1e-15
    gram = m @ np.diag(w) @ m.T
    assert np.max(np.abs(gram - np.eye(Q))) < 1e-14
    n = (m * w[None, :]).T  # n[i, a]
    assert np.max(np.abs(m.T @ n.T - np.eye(Q))) < 1e-14
    # sum_i m_i^a w_i = delta^{a0} (Sec. II, moment equilibrium passage)
    assert np.max(np.abs(m @ w - np.eye(Q)[0])) < 1e-14


@pytest.mark.parametrize("theta", [1.0 / 3.0, 0.2, 0.1, 0.45])
def test_d2q5_matches_printed_matrix(orc, theta):
    """The oracle's Gram-Schmidt reproduces the D2Q5 moment matrix printed in
    Sec. II for any theta."""
    m = orc.basis(orc.D2Q5, theta)
    assert np.max(np.abs(m - golden_io.d2q5_matrix(theta))) < 1e-14


@pytest.mark.parametrize("name", ["D1Q3", "D2Q9", "D3Q19", "D2Q5"])
def test_velocity_rows(orc, name):
    """The basis holds the velocities as v_{i alpha} = sqrt(theta) m_i^{a(alpha)}
    (the identity Sec. III relies on)."""
    lat = _lat(orc, name)
    theta = 1.0 / 3.0
    D, Q, v, w = orc.lattice(lat, theta)
    m = orc.basis(lat, theta)
    for alpha in range(D):
        hits = [a for a in range(Q) if np.max(np.abs(v[:, alpha] - np.sqrt(theta) * m[a])) < 1e-14]
        assert len(hits) == 1


def test_d2q9_is_tensor_product_of_d1q3(orc):
    """With product weights the p-major Gram-Schmidt of v_x^p v_y^q equals the
    product of the D1Q3 basis functions (orthogonal polynomials in each axis)."""
    m1 = orc.basis(orc.D1Q3)
    _, _, v1, _ = orc.lattice(orc.D1Q3)
    col = {int(v1[i, 0]): i for i in range(3)}
    _, Q, v, w = orc.lattice(orc.D2Q9)
    m = orc.basis(orc.D2Q9)
    for p, q in itertools.product(range(3), range(3)):
        a = 3 * p + q
        expect = np.array([m1[p, col[int(vx)]] * m1[q, col[int(vy)]] for vx, vy, _ in v])
        assert np.max(np.abs(m[a] - expect)) < 1e-14


def test_d1q3_closed_form(orc):
    """D1Q3 basis in closed form: 1; sqrt3 v; (3 v^2 - 1)/sqrt2."""
    m = orc.basis(orc.D1Q3)
    expect = np.array([[1, 1, 1], [0, np.sqrt(3), -np.sqrt(3)], [-1 / np.sqrt(2), np.sqrt(2), np.sqrt(2)]])
    assert np.max(np.abs(m - expect)) < 1e-15


def test_d3q19_spans_polynomials(orc):
    """The D3Q19 basis is a triangular (Gram-Schmidt) transform of its 19
    monomials: each m^a is a combination of monomials 0..a with a positive
    leading coefficient, and the monomials are independent on D3Q19."""
    _, Q, v, w = orc.lattice(orc.D3Q19)
    m = orc.basis(orc.D3Q19)
    monos = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0),
             (0, 1, 1), (0, 0, 2), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 0, 2), (0, 2, 1), (0, 1, 2),
             (2, 2, 0), (2, 0, 2), (0, 2, 2)]
    P = np.array([[float(vx) ** p * float(vy) ** q * float(vz) ** r for vx, vy, vz in v] for p, q, r in monos])
    assert np.linalg.matrix_rank(P) == Q
    # m = T P with T lower triangular and positive diagonal
    T = m @ np.linalg.inv(P)
    assert np.max(np.abs(np.triu(T, 1))) < 1e-12
    assert np.all(np.diag(T) > 0)
