"""Density of states of the stiffness matrix (the spectral-density appendix).

The paper defines the DOS of a symmetric matrix A of order m as
phi(t) = (1/m) sum_j delta(t - lambda_j) and broadens it with a Gaussian of
width eta (Eqs. "DOS", "DOS_gauss"):
    phi_eta(t) = (1/m) sum_j g_eta(t - lambda_j) = (1/m) Tr g_eta(t I - A).
Here the trace is taken by the kernel polynomial method: g_eta(t - .) is
expanded in Chebyshev polynomials of the spectrum mapped to [-1, 1],
    g_eta(t - lambda) ~ sum_k c_k(t) T_k(lambda~),
so phi_eta(t) = (1/m) sum_k c_k(t) Tr T_k(A~), and Tr T_k(A~) is estimated by
E[v^T T_k(A~) v] over random sign vectors v (Hutchinson), or exactly with
unit vectors.  The moments v^T T_k(A~) v come from the GPU
(rve_cheb_moments: matrix-free stencil, FP64); the coefficients c_k(t)
(Chebyshev-Gauss quadrature) and the weighted sums from the library's host
functions rve_dos_coefficients / rve_dos_from_moments.  This module only
marshals arguments.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rve


def spectral_bounds(d: dict, scheme=rve.CONSISTENT) -> tuple[float, float]:
    """[0, hi] containing the spectrum of A (Gershgorin: zero row sums and
    non-positive off-diagonals, so |row| <= 2 * centre = 4 w0 * (4 a_max))."""
    a_max = max(d["a_matrix"], d["a_incl"])
    w0 = 1.0 / 3.0 if scheme == rve.CONSISTENT else 0.5
    return 0.0, 16.0 * w0 * a_max * (1.0 + 1e-9)


def gauss(t, eta):
    return np.exp(-0.5 * (t / eta) ** 2) / (np.sqrt(2.0 * np.pi) * eta)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def cheb_coefficients(t: np.ndarray, K: int, lo: float, hi: float, eta: float,
                      quad: int | None = None) -> np.ndarray:
    """c[T, K]: Chebyshev coefficients of lambda -> g_eta(t - lambda) on
    [lo, hi], by Chebyshev-Gauss quadrature (rve_dos_coefficients)."""
    t = _f64(t).ravel()
    c = np.zeros((t.size, int(K)))
    rve.check(rve.lib().rve_dos_coefficients(rve._np_ptr(t), t.size, int(K), float(lo), float(hi),
                                             float(eta), int(quad or 0), rve._np_ptr(c)),
              "rve_dos_coefficients")
    return c


def dos_from_moments(mu: np.ndarray, t: np.ndarray, lo: float, hi: float, eta: float,
                     m: int) -> np.ndarray:
    """phi_eta(t) from trace moments mu[K] = Tr T_k(A~) (rve_dos_from_moments)."""
    mu, t = _f64(mu).ravel(), _f64(t).ravel()
    phi = np.zeros(t.size)
    rve.check(rve.lib().rve_dos_from_moments(rve._np_ptr(mu), mu.size, float(m), float(lo),
                                             float(hi), float(eta), rve._np_ptr(t), t.size,
                                             rve._np_ptr(phi)), "rve_dos_from_moments")
    return phi


def rademacher(nodes: int, count: int, seed: int, device) -> torch.Tensor:
    """count pairs of random sign vectors, [count, nodes, 2] float64."""
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    v = torch.randint(0, 2, (count, nodes, 2), generator=g, dtype=torch.int8)
    return (2.0 * v.to(torch.float64) - 1.0).to(device)


def dos(d: dict, mask: torch.Tensor, t: np.ndarray, eta: float, K: int = 512, vectors: int = 16,
        seed: int = 0, scheme=rve.CONSISTENT) -> np.ndarray:
    """phi_eta(t) of one realization's stiffness matrix, by stochastic
    Chebyshev moments with `vectors` random sign vectors (an even number)."""
    n = d["L"] * d["m0"]
    m = n * n
    lo, hi = spectral_bounds(d, scheme)
    pairs = vectors // 2
    words = m // 32
    # the same realization `pairs` times, two start vectors per copy
    batch = [d] * pairs
    masks = mask[:words].repeat(pairs)
    v = rademacher(m, pairs, seed, mask.device).reshape(pairs * m, 2)
    mu = rve.cheb_moments(batch, v, K, lo, hi, mask=masks, scheme=scheme)
    tr = mu.sum(dim=(0, 1)).cpu().numpy() / vectors          # E[v^T T_k v] = Tr T_k
    return dos_from_moments(tr, t, lo, hi, eta, m)
