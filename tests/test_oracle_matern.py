"""Pins for the oracle's Matern covariance (Eq. 5) and random-number generator."""
import os

import numpy as np
import pytest

import oracle
from tests import _ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_closed_forms_match_bessel_definition(nu):
    # Eq. 5 with SciPy's K_nu versus the oracle's closed forms.
    x = np.concatenate([np.logspace(-6, 1.7, 200), [0.0]])
    got = oracle.matern_corr(nu, x)
    want = _ref.matern_kv(nu, x)
    np.testing.assert_allclose(got, want, rtol=2e-13, atol=1e-300)


@pytest.mark.parametrize("nu", [0.25, 1.0, 2.0, 3.7])
def test_general_nu_quadrature_matches_scipy(nu):
    x = np.logspace(-3, 1.5, 40)
    got = oracle.matern_corr(nu, x)
    want = _ref.matern_kv(nu, x)
    np.testing.assert_allclose(got, want, rtol=1e-11)


def test_bessel_quadrature_half_integer_closed_form():
    # K_{1/2}(x) = sqrt(pi/(2x)) e^{-x} (DLMF 10.39.2), independent of SciPy.
    for x in [1e-3, 0.1, 1.0, 7.5, 40.0]:
        want = np.sqrt(np.pi / (2 * x)) * np.exp(-x)
        assert abs(oracle.bessel_k(0.5, x) / want - 1) < 1e-12


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_beta.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                er, nu, beta = map(float, line.split())
                rows.append((er, nu, beta))
    return rows


def test_table1_effective_range_pin():
    rows = _table1()
    assert len(rows) == 9
    th_rho = []
    for er, nu, beta in rows:
        th = oracle.theta(sigma2=2.0, beta=beta, nu=nu)
        c = oracle.cov(th, [0.0, 0.0], [er, 0.0], False) / 2.0
        th_rho.append(c)
    th_rho = np.array(th_rho)
    # every cell reaches the same correlation level at its effective range
    assert np.all(np.abs(th_rho - 0.022222) < 5e-6), th_rho
    # and a slip in the smoothness (e.g. the nu = 1.5 form used for nu = 2.5) breaks it
    wrong = oracle.matern_corr(1.5, np.array([0.1 / 0.014290]))[0]
    assert abs(wrong - 0.022222) > 1e-3


def test_cov_diagonal_and_nugget():
    th = oracle.theta(sigma2=1.7, beta=0.2, nu=1.5, nugget=0.03)
    s = [0.3, 0.4]
    assert oracle.cov(th, s, s, True) == pytest.approx(1.7 + 0.03, rel=1e-15)
    # two distinct observations at the same coordinates: no nugget (point identity)
    assert oracle.cov(th, s, s, False) == pytest.approx(1.7, rel=1e-15)


def test_anisotropic_reduces_to_isotropic():
    rng = np.random.default_rng(3)
    a, b = rng.random(3), rng.random(3)
    iso = oracle.theta(sigma2=1.3, beta=0.15, nu=2.5)
    ani = oracle.theta(sigma2=1.3, nu=2.5, ranges=[0.15, 0.15, 0.15])
    assert oracle.cov(iso, a, b, False) == pytest.approx(oracle.cov(ani, a, b, False), rel=1e-14)
    # stretching one axis and its range together leaves the covariance unchanged
    ani2 = oracle.theta(sigma2=1.3, nu=2.5, ranges=[0.15, 0.45, 0.15])
    a2, b2 = a.copy(), b.copy()
    a2[1] *= 3
    b2[1] *= 3
    assert oracle.cov(ani, a, b, False) == pytest.approx(oracle.cov(ani2, a2, b2, False), rel=1e-13)
    # and matches the dense SciPy construction
    want = _ref.cov_matrix(a[None], b[None], 1.3, None, 2.5, ranges=[0.15, 0.45, 0.15])[0, 0]
    assert oracle.cov(ani2, a, b, False) == pytest.approx(want, rel=1e-13)


def test_splitmix64_published_sequence():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                c, v = line.split()
                assert oracle.splitmix64(0, int(c)) == int(v, 16)
