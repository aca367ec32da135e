"""Pins of the oracle's real spherical harmonics against scipy's complex
spherical harmonics (with the Condon-Shortley phase), orthonormality by
quadrature, and Y_00 = 1/(2 sqrt(pi))."""
import numpy as np
import pytest
from scipy.special import sph_harm_y


def _real_sh(l, m, d):
    theta = np.arccos(np.clip(d[2], -1, 1))
    phi = np.arctan2(d[1], d[0])
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    Y = sph_harm_y(l, abs(m), theta, phi)
    return np.sqrt(2.0) * (Y.real if m > 0 else Y.imag)


def test_y00(oracle_lib):
    Y = oracle_lib.sh_basis(0, [0.3, 0.4, np.sqrt(1 - 0.25)])
    assert Y[0] == pytest.approx(1.0 / (2.0 * np.sqrt(np.pi)), rel=1e-15)


def test_matches_scipy(oracle_lib):
    rng = np.random.default_rng(0)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y = oracle_lib.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert Y[l * l + l + m] == pytest.approx(_real_sh(l, m, d), abs=1e-12)


def test_low_order_signs(oracle_lib):
    """Condon-Shortley convention: Y_1,-1 = -c y, Y_10 = c z, Y_11 = -c x."""
    c = np.sqrt(3.0 / (4.0 * np.pi))
    d = np.array([0.48, 0.6, 0.64])
    Y = oracle_lib.sh_basis(1, d)
    assert Y[1] == pytest.approx(-c * d[1])
    assert Y[2] == pytest.approx(c * d[2])
    assert Y[3] == pytest.approx(-c * d[0])


def test_orthonormal_by_quadrature(oracle_lib):
    nz, nphi = 24, 48
    z, w = np.polynomial.legendre.leggauss(nz)
    phis = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    G = np.zeros((16, 16))
    for zi, wi in zip(z, w):
        s = np.sqrt(1 - zi * zi)
        for ph in phis:
            Y = oracle_lib.sh_basis(3, [s * np.cos(ph), s * np.sin(ph), zi])
            G += wi * (2 * np.pi / nphi) * np.outer(Y, Y)
    assert np.allclose(G, np.eye(16), atol=1e-12)
