"""Pins of the oracle's random numbers and fluctuating collision.

- Philox4x32-10 against the published known-answer vectors (SC'11).
- Box-Muller / uniform variates against the normal and uniform laws.
- The f-space noise covariance the oracle's collision produces, against
  the paper's general fluctuation-dissipation expression (Sec. II, the
  <xi_i xi_j> formula that precedes the moment transform) with the
  f-space collision matrix, and against eq. xiglobal / xilocal.
"""
import math

import numpy as np
import pytest
from scipy import stats

from tests import golden_io

LATS = ["D1Q3", "D2Q9", "D3Q19", "D2Q5"]


def test_philox_known_answers(orc):
    for ctr, key, out in golden_io.philox_kat():
        assert orc.philox4x32_10(ctr, key).tolist() == out


def _many_normals(orc, dist, nsite=4000, nmom=8, t=3, seed=12345):
    return np.array([orc.site_noise(seed, 0, s, t, nmom, dist) for s in range(nsite)])


def test_gaussian_variates_are_standard_normal(orc):
    z = _many_normals(orc, orc.GAUSSIAN)
    flat = z.ravel()
    n = flat.size
    assert abs(flat.mean()) < 5 / math.sqrt(n)
    assert abs(flat.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(flat, fisher=False) - 3.0) < 5 * math.sqrt(24.0 / n)
    assert stats.kstest(flat, "norm").pvalue > 1e-4
    # moments drawn at one site are uncorrelated with each other
    c = np.corrcoef(z.T)
    assert np.max(np.abs(c - np.eye(c.shape[0]))) < 5 / math.sqrt(z.shape[0])
    # Box-Muller on 24-bit uniforms cuts the tails near sqrt(-2 ln 2^-25)
    assert np.max(np.abs(flat)) < math.sqrt(-2 * math.log(0.5 / 2**24)) + 1e-12


def test_uniform_variates(orc):
    """Flat noise of unit variance on (-sqrt3, sqrt3) (Sec. IV uses a flat law
    with half-width d^a = sqrt(3 var))."""
    z = _many_normals(orc, orc.UNIFORM).ravel()
    n = z.size
    assert np.all(np.abs(z) < math.sqrt(3.0))
    assert abs(z.var() - 1.0) < 5 * math.sqrt(0.8 / n)
    assert stats.kstest(z, "uniform", args=(-math.sqrt(3), 2 * math.sqrt(3))).pvalue > 1e-4


def test_noise_keying(orc):
    """Distinct (seed, lattice id, step, site) give distinct streams; a key
    gives the same stream every time; moment a = 4j + k + 1 takes word k of
    Philox call j."""
    base = orc.site_noise(7, 0, 11, 5, 18)
    assert np.array_equal(base, orc.site_noise(7, 0, 11, 5, 18))
    for other in [(8, 0, 11, 5), (7, 1, 11, 5), (7, 0, 12, 5), (7, 0, 11, 6), (7, 0, 11, 5 + 2**32)]:
        z = orc.site_noise(other[0], other[1], other[2], other[3], 18)
        assert not np.any(np.isclose(z, base, rtol=0, atol=1e-12))
    # call j = 1 feeds moments 5..8: same as the first four of a stream whose
    # step word carries j = 1 in its low bits (counter word 3 = t_hi*8 + j)
    z_short = orc.site_noise(7, 0, 11, 5, 4)
    assert np.array_equal(z_short, base[:4])
    w0 = orc.philox4x32_10([11, 0, 5, 0], [7, 0])
    u = ((w0 >> 8).astype(np.float64) + 0.5) / 2**24
    assert abs(math.sqrt(-2 * math.log(u[0])) * math.cos(2 * math.pi * u[1]) - base[0]) < 1e-15
    # uniform variates are an affine map of the same words
    zu = orc.site_noise(7, 0, 11, 5, 4, orc.UNIFORM)
    assert np.max(np.abs(zu - math.sqrt(3) * (2 * u - 1))) < 1e-15


def _noise_matrix(orc, lat, f0, tau, mode, rho_eq=0.0, theta=1.0 / 3.0):
    """B[i, a]: f-space response of one collision to unit variate z^{a+1}."""
    Q = orc.q_of(lat)
    base = orc.collide(lat, f0, np.zeros(Q - 1), tau, mode, rho_eq, theta)
    B = np.zeros((Q, Q - 1))
    for a in range(Q - 1):
        z = np.zeros(Q - 1)
        z[a] = 1.0
        B[:, a] = orc.collide(lat, f0, z, tau, mode, rho_eq, theta) - base
    return base, B


def _paper_xi_cov(w, Lam, rho):
    """<xi_i xi_j> = rho [ sum_kl L_ik L_jl (w_k w_l - w_k d_kl)
                            - sum_k L_jk (w_i w_k - w_i d_ik)
                            - sum_l L_il (w_l w_j - w_l d_lj) ]  (Sec. II)."""
    C = np.outer(w, w) - np.diag(w)
    return rho * (Lam @ C @ Lam.T - C @ Lam.T - Lam @ C)


@pytest.mark.parametrize("name", LATS)
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0, 1.5])
def test_srt_noise_covariance_matches_paper(orc, name, tau):
    """Local noise at density rho: B B^T equals the paper's f-space covariance
    with Lambda_ij = delta_ij / tau, i.e. rho (2 tau - 1)/tau^2 (diag w - w w^T)."""
    lat = getattr(orc, name)
    D, Q, v, w = orc.lattice(lat)
    rho = 37.5
    f0 = rho * w * (1 + 0.05 * np.cos(np.arange(Q)))  # off-equilibrium, same rho after rescale
    f0 *= rho / f0.sum()
    _, B = _noise_matrix(orc, lat, f0, tau, orc.NOISE_LOCAL)
    cov = B @ B.T
    paper = _paper_xi_cov(w, np.eye(Q) / tau, rho)
    assert np.max(np.abs(cov - paper)) < 1e-12 * rho
    closed = rho * (2 * tau - 1) / tau**2 * (np.diag(w) - np.outer(w, w))
    assert np.max(np.abs(cov - closed)) < 1e-12 * rho
    # noise creates no mass: sum_i xi_i = 0 for every variate
    assert np.max(np.abs(B.sum(0))) < 1e-13 * rho


@pytest.mark.parametrize("name", ["D2Q5", "D2Q9", "D3Q19"])
def test_mrt_noise_covariance_matches_paper(orc, name):
    """MRT (Lambda^{ab} = delta^{ab}/tau^a): the oracle's noise reproduces the
    paper's general f-space expression with Lambda_ij = sum_a n_i^a m_j^a / tau^a,
    which the paper reduces to eq. xiglobal in moment space."""
    lat = getattr(orc, name)
    D, Q, v, w = orc.lattice(lat)
    m = orc.basis(lat)
    rng = np.random.default_rng(3)
    taus = rng.uniform(0.55, 1.9, Q)
    rho = 12.0
    _, B = _noise_matrix(orc, lat, rho * w, taus, orc.NOISE_GLOBAL, rho_eq=rho)
    n = (m * w[None, :]).T
    Lam = n @ np.diag(1.0 / taus) @ m
    paper = _paper_xi_cov(w, Lam, rho)
    assert np.max(np.abs(B @ B.T - paper)) < 1e-12 * rho
    # in moment space the covariance is diagonal with rho (2 tau^a - 1)/tau_a^2 (eq. xiglobal)
    Mcov = m @ (B @ B.T) @ m.T
    expect = np.diag([0.0] + [rho * (2 * t - 1) / t**2 for t in taus[1:]])
    assert np.max(np.abs(Mcov - expect)) < 1e-12 * rho


@pytest.mark.parametrize("name", LATS)
def test_relaxation_without_noise(orc, name):
    """Noise off, SRT: f*_i = f_i + (w_i rho - f_i)/tau (eq. collision with
    Lambda_ij = delta_ij/tau, f^0 = rho w), and mass is conserved."""
    lat = getattr(orc, name)
    D, Q, v, w = orc.lattice(lat)
    rng = np.random.default_rng(5)
    fin = rng.uniform(0.5, 3.0, Q)
    for tau in (0.51, 0.8, 1.0, 1.7):
        out = orc.collide(lat, fin, np.zeros(Q - 1), tau, orc.NOISE_OFF)
        expect = fin + (w * fin.sum() - fin) / tau
        assert np.max(np.abs(out - expect)) < 1e-15 * Q * fin.sum()
        assert abs(out.sum() - fin.sum()) < 1e-15 * Q * fin.sum()


def test_local_noise_clamps_at_negative_density(orc):
    """Local noise treats rho <= 0 as zero density (Sec. IV); global noise
    does not look at the local density."""
    lat = orc.D2Q9
    D, Q, v, w = orc.lattice(lat)
    fin = -0.3 * w + 0.01 * np.arange(Q) - 0.01 * np.arange(Q).mean()
    assert fin.sum() < 0
    z = np.linspace(-1, 1, Q - 1)
    off = orc.collide(lat, fin, z, 0.8, orc.NOISE_OFF)
    loc = orc.collide(lat, fin, z, 0.8, orc.NOISE_LOCAL)
    assert np.array_equal(off, loc)
    glob = orc.collide(lat, fin, z, 0.8, orc.NOISE_GLOBAL, rho_eq=2.0)
    assert np.max(np.abs(glob - off)) > 0.1


def test_uniform_noise_half_width(orc):
    """Flat noise: the largest variate moves M^a by d^a = sqrt(3 rho (2tau-1)/tau^2)
    (Sec. IV)."""
    lat = orc.D2Q5
    D, Q, v, w = orc.lattice(lat)
    m = orc.basis(lat)
    rho, tau = 30.0, 0.7
    f0 = rho * w
    base = orc.collide(lat, f0, np.zeros(Q - 1), tau, orc.NOISE_LOCAL)
    z = np.zeros(Q - 1)
    z[2] = math.sqrt(3.0)
    out = orc.collide(lat, f0, z, tau, orc.NOISE_LOCAL)
    dM = m @ (out - base)
    d = math.sqrt(3 * rho * (2 * tau - 1) / tau**2)
    assert abs(dM[3] - d) < 1e-12 * rho
    assert np.max(np.abs(np.delete(dM, 3))) < 1e-12 * rho
