"""The GPU march of the linear theory (Eq. 5, qsa_eq5_march) against the oracle's independent
integrator on the same discretisation, against the exact series of Eq. 5, and its own
invariants (snapshots, Gamma = 0)."""
import math

import numpy as np
import pytest

from oracle import linear_theory as lt
from paper_2607_24214_b300 import config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def march(cuda_ok):
    from paper_2607_24214_b300.qsa import eq5_march
    return eq5_march


def seeds(ks, xi):
    """psi(xi, 0) of a cold beam with a uniform unit density step: the oracle's initial data."""
    return np.array([-(1.0 - np.cos(xi)) / (k * k + 1.0) for k in ks])


def test_matches_oracle_integrator(march):
    p = config.v_pair_single_mode()
    ks = [0.5, 1.0, 2.0, 4.0, 9.0]
    gam = np.array([lt.growth_rate(k, p.species) for k in ks])
    dxi, n = 0.05, 401
    xi = np.arange(n) * dxi
    tau_end, n_tau = 5.0 / gam.min(), 400
    got = march(gam, seeds(ks, xi), np.zeros((len(ks), n)), dxi, tau_end, n_tau)[0]
    for m, k in enumerate(ks):
        want = lt.march_eq5(xi, tau_end, n_tau, gam[m], k=k)
        scale = np.abs(want).max()
        assert np.abs(got[m] - want).max() <= 1e-10 * scale, k


def test_matches_exact_series(march):
    """Gamma tau = 4 at xi in [0, 15]: the series of Eq. 5 within the O(dxi^2) trapezoid error."""
    G, k = 4e-3, 2.0
    dxi, n = 1.0 / 128, 15 * 128 + 1
    xi = np.arange(n) * dxi
    tau = 4.0 / G
    got = march([G], seeds([k], xi), np.zeros((1, n)), dxi, tau, 400)[0, 0]
    for x in (1.0, 2.0, 5.0, 10.0, 15.0):
        want = lt.psi_series(x, G * tau, k=k)
        i = int(round(x / dxi))
        assert abs(got[i] - want) <= 2e-4 * abs(want), x


def test_snapshots_are_the_shorter_runs(march):
    ks, dxi, n = [1.0, 3.0], 0.1, 120
    xi = np.arange(n) * dxi
    rng = np.random.default_rng(3)
    psi0, dpsi0 = rng.normal(size=(2, n)), rng.normal(size=(2, n)) * 1e-3
    gam = [2e-3, 5e-3]
    snaps = march(gam, psi0, dpsi0, dxi, 1000.0, 200, n_out=4)
    for o in range(4):
        one = march(gam, psi0, dpsi0, dxi, 250.0 * (o + 1), 50 * (o + 1))[0]
        np.testing.assert_array_equal(snaps[o], one)


def test_zero_gamma_is_free_motion(march):
    n, dxi = 64, 0.25
    rng = np.random.default_rng(5)
    psi0, dpsi0 = rng.normal(size=(1, n)), rng.normal(size=(1, n))
    got = march([0.0], psi0, dpsi0, dxi, 7.0, 35)[0]
    np.testing.assert_allclose(got, psi0 + 7.0 * dpsi0, rtol=1e-12, atol=1e-12)


def test_invalid_arguments(march):
    from paper_2607_24214_b300.qsa import QsaError
    z = np.zeros((1, 8))
    with pytest.raises(QsaError):
        march([1.0], np.zeros((1, 4096)), np.zeros((1, 4096)), 0.1, 1.0, 4)  # n_xi too large
    with pytest.raises(QsaError):
        march([1.0], z, z, 0.1, 1.0, 5, n_out=2)                            # 2 does not divide 5
    with pytest.raises(QsaError):
        march([-1.0], z, z, 0.1, 1.0, 4)                                     # Gamma < 0
    with pytest.raises(QsaError):
        march([1.0], z, z, 0.0, 1.0, 4)                                      # dxi = 0
