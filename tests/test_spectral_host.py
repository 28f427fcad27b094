"""Host side of the density of states (no GPU): the Chebyshev reconstruction
in `spectral.py` (coefficients of the broadened delta by Chebyshev-Gauss
quadrature, weighted sums of trace moments) against the dense spectrum of
the oracle's stiffness matrix, and the Gershgorin interval against the
eigenvalues.  The moments here are exact traces computed on the host; on the
GPU they come from rve_cheb_moments (tests/test_gpu_parity.py)."""
import numpy as np
import pytest

import oracle
from paper_1903_12227_gb300 import spectral


def _coef(n, seed, a_matrix=1.0, a_incl=5.0):
    g = np.random.default_rng(seed)
    return np.where(g.random((n, n)) < 0.45, a_incl, a_matrix)


def _trace_moments(A, K, lo, hi):
    """Tr T_k(A~), A~ = (2A - (hi+lo)) / (hi-lo), by the three-term recurrence."""
    m = A.shape[0]
    At = (2.0 * A - (hi + lo) * np.eye(m)) / (hi - lo)
    T0, T1 = np.eye(m), At.copy()
    mu = [np.trace(T0), np.trace(T1)]
    for _ in range(2, K):
        T0, T1 = T1, 2.0 * At @ T1 - T0
        mu.append(np.trace(T1))
    return np.array(mu)


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_gershgorin_interval_contains_the_spectrum(scheme):
    n, h = 16, 0.25
    d = {"a_matrix": 1.0, "a_incl": 5.0}
    lo, hi = spectral.spectral_bounds(d, scheme)
    ev = oracle.spectrum(_coef(n, 1), h, scheme)
    assert lo <= ev.min() + 1e-12 and ev.max() <= hi
    # and it is not loose by more than the Gershgorin factor of two
    assert ev.max() > 0.3 * hi


def test_chebyshev_reconstruction_matches_dense_broadening():
    # exact trace moments -> the broadened density of the dense spectrum (the
    # expansion of a Gaussian of width eta on an interval of width W converges
    # once K is a few times W / eta: here W / eta = 178, K = 800)
    n, h, eta, K = 12, 0.25, 0.15, 800
    coef = _coef(n, 2)
    A = oracle.csr_to_dense(oracle.assemble(coef, h), n * n)
    lo, hi = spectral.spectral_bounds({"a_matrix": 1.0, "a_incl": 5.0})
    mu = _trace_moments(A, K, lo, hi)
    t = np.linspace(lo, hi, 301)
    phi = spectral.dos_from_moments(mu, t, lo, hi, eta, n * n)
    ref = oracle.dos_gauss(oracle.spectrum(coef, h), t, eta)
    assert np.abs(phi - ref).max() < 1e-9 * ref.max()


def test_chebyshev_coefficients_reproduce_the_gaussian():
    # sum_k c_k(t) T_k(lambda~) = g_eta(t - lambda) on the interval
    lo, hi, eta, K = 0.0, 10.0, 0.3, 600
    t = np.array([1.0, 4.2, 9.5])
    c = spectral.cheb_coefficients(t, K, lo, hi, eta)
    lam = np.linspace(lo, hi, 57)
    x = (2.0 * lam - (hi + lo)) / (hi - lo)
    Tk = np.cos(np.arange(K)[:, None] * np.arccos(np.clip(x, -1, 1))[None, :])
    approx = c @ Tk
    exact = spectral.gauss(t[:, None] - lam[None, :], eta)
    assert np.abs(approx - exact).max() < 1e-9 * exact.max()
