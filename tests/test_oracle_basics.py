"""Pins of the oracle's building blocks against closed forms and published values (CPU only)."""
import os

import numpy as np
import pytest
from scipy.special import dawsn, erf

from oracle import tdh

HERE = os.path.dirname(os.path.abspath(__file__))


def _gaussian_charge(N, box, sigma, centre):
    g = tdh.Grid(N, box)
    x = np.arange(N) * g.h
    r2 = ((x[:, None, None] - centre[2]) ** 2 + (x[None, :, None] - centre[1]) ** 2
          + (x[None, None, :] - centre[0]) ** 2)
    n = np.exp(-r2 / (2 * sigma ** 2)) / ((2 * np.pi) ** 1.5 * sigma ** 3)
    return g, x, n, np.sqrt(r2)


def test_coulomb_truncated_matches_erf_potential_of_gaussian():
    # A normalised Gaussian charge of width sigma has potential erf(r / (sqrt(2) sigma)) / r.
    g, x, n, r = _gaussian_charge(32, 8.0, 0.6, (4.0, 4.0, 4.0))
    u = tdh.coulomb_truncated(n, g)
    near = r < 3.0
    with np.errstate(invalid="ignore", divide="ignore"):
        exact = np.where(r > 0, erf(r / (np.sqrt(2) * 0.6)) / np.where(r > 0, r, 1),
                         np.sqrt(2 / np.pi) / 0.6)
    assert np.max(np.abs(u[near] - exact[near])) < 1e-7


def test_coulomb_periodic_matches_direct_fourier_series():
    # Periodic potential of the same charge, summed directly over reciprocal vectors (no FFT):
    # u(r) = (4 pi / Omega) sum_{G != 0} exp(-sigma^2 G^2 / 2) cos(G.(r - R)) / G^2.
    box, sigma, R = 8.0, 0.6, np.array([3.5, 4.25, 4.0])
    g, x, n, _ = _gaussian_charge(32, box, sigma, R)
    u = tdh.coulomb_periodic(n, g)
    m = np.arange(-20, 21)
    G = 2 * np.pi / box * np.array(np.meshgrid(m, m, m, indexing="ij")).reshape(3, -1).T
    G2 = np.sum(G * G, axis=1)
    keep = G2 > 0
    G, G2 = G[keep], G2[keep]
    amp = 4 * np.pi / box ** 3 * np.exp(-0.5 * sigma ** 2 * G2) / G2
    rng = np.random.default_rng(3)
    for _ in range(6):
        iz, iy, ix = rng.integers(0, 32, size=3)
        rr = np.array([x[ix], x[iy], x[iz]]) - R
        val = np.sum(amp * np.cos(G @ rr))
        assert abs(u[iz, iy, ix] - val) < 1e-9


def test_coulomb_periodic_drops_g0_and_is_linear_symmetric():
    g = tdh.Grid(8, 5.0)
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal((2, 8, 8, 8))
    ua, ub = tdh.coulomb_periodic(a, g), tdh.coulomb_periodic(b, g)
    assert abs(ua.mean()) < 1e-12  # G = 0 component removed
    assert abs(np.sum(a * ub) - np.sum(b * ua)) < 1e-10 * np.sum(np.abs(a * ub))
    assert np.sum(a * ua) > 0  # positive (semi)definite kernel


def test_splitmix64_published_vectors():
    with open(os.path.join(HERE, "golden", "splitmix64_vectors.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 8
    for seed, k, hexv in rows:
        assert tdh.splitmix64(int(seed), int(k)) == int(hexv, 16)


def test_coefficients_distribution():
    c = tdh.stochastic_coefficients(7, 40, 250, "gaussian")
    assert abs(c.mean()) < 0.03 and abs(c.var() - 1.0) < 0.03
    s = tdh.stochastic_coefficients(7, 40, 250, "sign")
    assert set(np.unique(s)) == {-1.0, 1.0} and abs(s.mean()) < 0.03
    # counter-based: a sub-block does not depend on the block's size
    assert np.array_equal(tdh.stochastic_coefficients(7, 3, 250, "gaussian"), c[:3])


def test_time_weights_reproduce_dawson_damped_sine_integral():
    # int_0^inf exp(-g^2 t^2 / 2) sin(W t) dt = (sqrt(2) / g) F(W / (sqrt(2) g)), F = Dawson.
    gamma = 0.5
    p = tdh.TDHParams(n_steps=4000, dt=0.005, gamma=gamma)
    t = np.arange(p.n_steps + 1) * p.dt
    w = tdh.time_weights(p)
    for om in (0.3, 1.0, 2.5):
        exact = np.sqrt(2) / gamma * dawsn(om / (np.sqrt(2) * gamma))
        assert abs(np.sum(w * np.sin(om * t)) - exact) < 1e-5
    assert w[0] == pytest.approx(0.5 * p.dt) and w[1] == pytest.approx(
        p.dt * np.exp(-0.5 * gamma ** 2 * p.dt ** 2))
