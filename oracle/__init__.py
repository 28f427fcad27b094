"""FP64 CPU oracle for the RVE corrector method (arXiv:1903.12227).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path (the CUDA
library ``librve`` and its binding) never imports this package, and this
package imports nothing from the product.

The arithmetic lives in ``rve_oracle.c`` (plain C, FP64); this module compiles
it with gcc on first use and exposes thin numpy wrappers.  Each wrapper cites
the passage of the paper it follows in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rve_oracle.c")
_HDR = os.path.join(_HERE, "rve_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SCHEME_CONSISTENT = 0
SCHEME_LUMPED = 1


class Realization(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("m0", ctypes.c_int32),
                ("incl_cells", ctypes.c_int32), ("n_incl", ctypes.c_int32),
                ("a_matrix", ctypes.c_double), ("a_incl", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("index", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("A_energy", ctypes.c_double * 4), ("A_flux", ctypes.c_double * 4),
                ("relres_true", ctypes.c_double * 2), ("mean_a", ctypes.c_double),
                ("iters", ctypes.c_int32 * 2)]


class Result3(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32 * 3), ("relres_true", ctypes.c_double * 3),
                ("A_energy", ctypes.c_double * 9), ("A_flux", ctypes.c_double * 9),
                ("mean_a", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile rve_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-fopenmp", "-shared", "-std=c11",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u64, i64, i32, dbl = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        vp = ctypes.c_void_p
        L.orc_splitmix64_mix.restype = u64
        L.orc_splitmix64_mix.argtypes = [u64]
        L.orc_splitmix64_output.restype = u64
        L.orc_splitmix64_output.argtypes = [u64, u64]
        L.orc_realization_key.restype = u64
        L.orc_realization_key.argtypes = [u64, u64]
        L.orc_draw.restype = u64
        L.orc_draw.argtypes = [u64, ctypes.c_uint32, u64]
        L.orc_corners.argtypes = [ctypes.POINTER(Realization), vp]
        L.orc_gen_field.argtypes = [ctypes.POINTER(Realization), vp]
        L.orc_coef_from_mask.argtypes = [i64, vp, dbl, dbl, vp]
        L.orc_element_matrix.argtypes = [ctypes.c_int, dbl, vp]
        L.orc_assemble.restype = i64
        L.orc_assemble.argtypes = [i64, dbl, vp, ctypes.c_int, vp, vp, vp]
        L.orc_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
        L.orc_rhs.argtypes = [i64, dbl, vp, ctypes.c_int, vp]
        L.orc_laplacian_eig.restype = dbl
        L.orc_laplacian_eig.argtypes = [i64, i64, i64]
        L.orc_precond.argtypes = [i64, dbl, dbl, vp, vp]
        L.orc_pcg.restype = ctypes.c_int
        L.orc_pcg.argtypes = [i64, vp, vp, vp, dbl, dbl, vp, dbl, ctypes.c_int, vp, vp]
        L.orc_a_hom.argtypes = [i64, dbl, dbl, vp, ctypes.c_int, vp, vp, vp]
        L.orc_a_hom_grad.argtypes = [i64, dbl, dbl, ctypes.c_int, vp, vp, vp]
        L.orc_solve_coef.restype = ctypes.c_int
        L.orc_solve_coef.argtypes = [i64, i64, vp, dbl, ctypes.c_int, dbl, ctypes.c_int, dbl,
                                     vp, ctypes.POINTER(Result)]
        L.orc_solve_realization.restype = ctypes.c_int
        L.orc_solve_realization.argtypes = [ctypes.POINTER(Realization), ctypes.c_int, dbl,
                                            ctypes.c_int, dbl, vp, vp, ctypes.POINTER(Result)]
        L.orc_solve_batch.restype = ctypes.c_int
        L.orc_solve_batch.argtypes = [vp, ctypes.c_int, ctypes.c_int, dbl, ctypes.c_int, dbl,
                                      vp, ctypes.c_int]
        L.orc_statistics.argtypes = [i64, vp, dbl, ctypes.c_int, vp, vp, vp, vp, vp]
        L.orc3_statistics.restype = None
        L.orc3_statistics.argtypes = [i64, vp, dbl, vp, vp, vp]
        L.orc_mass_element.argtypes = [ctypes.c_int, dbl, vp]
        L.orc3_gen_field.argtypes = [ctypes.POINTER(Realization), vp]
        L.orc3_element_matrix.argtypes = [ctypes.c_int, dbl, vp]
        L.orc3_assemble.restype = i64
        L.orc3_assemble.argtypes = [i64, dbl, vp, ctypes.c_int, vp, vp, vp]
        L.orc3_rhs.argtypes = [i64, dbl, vp, ctypes.c_int, vp]
        L.orc3_precond.argtypes = [i64, dbl, dbl, vp, vp]
        L.orc3_pcg.restype = ctypes.c_int
        L.orc3_pcg.argtypes = [i64, vp, vp, vp, dbl, dbl, vp, dbl, ctypes.c_int, vp, vp]
        L.orc3_a_hom.argtypes = [i64, dbl, dbl, vp, ctypes.c_int, vp, vp, vp]
        L.orc3_solve_realization.restype = ctypes.c_int
        L.orc3_solve_realization.argtypes = [ctypes.POINTER(Realization), ctypes.c_int, dbl,
                                             ctypes.c_int, dbl, vp, vp, ctypes.POINTER(Result3)]
        L.orc_apply_mass.argtypes = [i64, dbl, ctypes.c_int, vp, vp]
        L.orc_solve_load.restype = ctypes.c_int
        L.orc_solve_load.argtypes = [i64, i64, vp, dbl, ctypes.c_int, vp, dbl, ctypes.c_int, dbl,
                                     vp, vp]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _real(d: dict) -> Realization:
    return Realization(int(d["L"]), int(d["m0"]), int(d["incl_cells"]), int(d["n_incl"]),
                       float(d["a_matrix"]), float(d["a_incl"]), int(d["seed"]) & (2**64 - 1),
                       int(d["index"]) & (2**64 - 1))


# ----------------------------------------------------------------- field --
def splitmix64_output(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64_output(seed & (2**64 - 1), k & (2**64 - 1)))


def corners(d: dict) -> np.ndarray:
    c = np.zeros((int(d["n_incl"]), 2), dtype=np.int32)
    lib().orc_corners(ctypes.byref(_real(d)), _p(c))
    return c


def gen_field(d: dict) -> np.ndarray:
    n = int(d["L"]) * int(d["m0"])
    m = np.zeros((n, n), dtype=np.uint8)
    lib().orc_gen_field(ctypes.byref(_real(d)), _p(m))
    return m


def coef_from_mask(mask: np.ndarray, a_matrix: float, a_incl: float) -> np.ndarray:
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    c = np.zeros(m.shape, dtype=np.float64)
    lib().orc_coef_from_mask(m.shape[0], _p(m), a_matrix, a_incl, _p(c))
    return c


# -------------------------------------------------------------- assembly --
def element_matrix(scheme: int, h: float) -> np.ndarray:
    E = np.zeros(16, dtype=np.float64)
    lib().orc_element_matrix(scheme, h, _p(E))
    return E.reshape(4, 4)


def assemble(coef: np.ndarray, h: float, scheme: int = SCHEME_CONSISTENT):
    """CSR stiffness (rowptr, colidx, vals) of Eq. "As_Kron" for cell values coef[n,n]."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    n = coef.shape[0]
    N = n * n
    rowptr = np.zeros(N + 1, dtype=np.int64)
    colidx = np.zeros(9 * N, dtype=np.int64)
    vals = np.zeros(9 * N, dtype=np.float64)
    nnz = lib().orc_assemble(n, h, _p(coef), scheme, _p(rowptr), _p(colidx), _p(vals))
    return rowptr, colidx[:nnz].copy(), vals[:nnz].copy()


def spmv(csr, x: np.ndarray) -> np.ndarray:
    rowptr, colidx, vals = csr
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.zeros_like(x)
    lib().orc_spmv(x.size, _p(rowptr), _p(colidx), _p(vals), _p(x), _p(y))
    return y


def csr_to_dense(csr, N: int) -> np.ndarray:
    rowptr, colidx, vals = csr
    A = np.zeros((N, N))
    for r in range(N):
        for k in range(rowptr[r], rowptr[r + 1]):
            A[r, colidx[k]] += vals[k]
    return A


def rhs(coef: np.ndarray, h: float, scheme: int = SCHEME_CONSISTENT) -> np.ndarray:
    """f[2, n, n]: Galerkin right-hand sides of the two corrector problems."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    n = coef.shape[0]
    f = np.zeros((2, n, n), dtype=np.float64)
    lib().orc_rhs(n, h, _p(coef), scheme, _p(f))
    return f


# ---------------------------------------------------------------- solver --
def mass_element(scheme: int, h: float) -> np.ndarray:
    M = np.zeros(16)
    lib().orc_mass_element(scheme, h, _p(M))
    return M.reshape(4, 4)


def apply_mass(x: np.ndarray, h: float, scheme: int = SCHEME_CONSISTENT) -> np.ndarray:
    """y = M x for nodal values x[n,n] (Q1 mass matrix of the scheme, periodic)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    lib().orc_apply_mass(x.shape[0], h, scheme, _p(x), _p(y))
    return y


def solve_load(coef: np.ndarray, L: int, m0: int, c0: float, b: np.ndarray,
               scheme: int = SCHEME_CONSISTENT, tol: float = 1e-12, max_iter: int = 20000,
               delta: float = 0.0):
    """Mean-zero u[n,n] with A u = b (b a mean-zero load vector); (u, iters, relres)."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    u = np.zeros_like(b)
    rr = ctypes.c_double(0.0)
    it = lib().orc_solve_load(L, m0, _p(coef), c0, scheme, _p(b), tol, max_iter, delta, _p(u),
                              ctypes.byref(rr))
    if it < 0:
        raise ValueError("orc_solve_load: n must be a power of two")
    return u, it, rr.value


def spectrum(coef: np.ndarray, h: float, scheme: int = SCHEME_CONSISTENT) -> np.ndarray:
    """All eigenvalues (ascending) of the assembled stiffness matrix, by a
    dense symmetric eigensolver (numpy.linalg.eigvalsh); small grids only."""
    n = coef.shape[0]
    return np.linalg.eigvalsh(csr_to_dense(assemble(coef, h, scheme), n * n))


def dos_gauss(eigs: np.ndarray, t: np.ndarray, eta: float) -> np.ndarray:
    """Gaussian-broadened density of states (1/m) sum_j g_eta(t - lambda_j)
    (the spectral-density appendix, Eq. "DOS_gauss")."""
    t = np.asarray(t, dtype=np.float64)
    g = np.exp(-0.5 * ((t[:, None] - eigs[None, :]) / eta) ** 2) / (np.sqrt(2 * np.pi) * eta)
    return g.sum(axis=1) / eigs.size


# ------------------------------------------------------------------ 3D --
def gen_field3(d: dict) -> np.ndarray:
    """Covered cells [n,n,n] (uint8) of a 3D realization (cubes)."""
    n = int(d["L"]) * int(d["m0"])
    mask = np.zeros((n, n, n), dtype=np.uint8)
    lib().orc3_gen_field(ctypes.byref(_real(d)), _p(mask))
    return mask


def element_matrix3(scheme: int, h: float) -> np.ndarray:
    E = np.zeros(64)
    lib().orc3_element_matrix(scheme, h, _p(E))
    return E.reshape(8, 8)


def assemble3(coef: np.ndarray, h: float, scheme: int = SCHEME_CONSISTENT):
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    n = coef.shape[0]
    N = n ** 3
    rowptr = np.zeros(N + 1, dtype=np.int64)
    colidx = np.zeros(27 * N, dtype=np.int64)
    vals = np.zeros(27 * N, dtype=np.float64)
    nnz = lib().orc3_assemble(n, h, _p(coef), scheme, _p(rowptr), _p(colidx), _p(vals))
    return rowptr, colidx[:nnz].copy(), vals[:nnz].copy()


def rhs3(coef: np.ndarray, h: float, scheme: int = SCHEME_CONSISTENT) -> np.ndarray:
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    n = coef.shape[0]
    f = np.zeros((3, n, n, n))
    lib().orc3_rhs(n, h, _p(coef), scheme, _p(f))
    return f


def precond3(r: np.ndarray, c0: float, delta: float = 0.0) -> np.ndarray:
    r = np.ascontiguousarray(r, dtype=np.float64)
    z = np.zeros_like(r)
    lib().orc3_precond(r.shape[0], c0, delta, _p(r), _p(z))
    return z


def solve_coef3(coef: np.ndarray, L: int, m0: int, c0: float, scheme: int = SCHEME_CONSISTENT,
                tol: float = 1e-12, max_iter: int = 5000) -> dict:
    """Three corrector solves and the 3x3 A_hom for a given cell coefficient [n,n,n]."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    n = coef.shape[0]
    h = 1.0 / m0
    rowptr, colidx, vals = assemble3(coef, h, scheme)
    f = rhs3(coef, h, scheme)
    u = np.zeros_like(f)
    iters, rel = [], []
    for i in range(3):
        rr = ctypes.c_double(0.0)
        it = lib().orc3_pcg(n, _p(rowptr), _p(colidx), _p(vals), c0, 0.0, _p(f[i]), tol, max_iter,
                            _p(u[i]), ctypes.byref(rr))
        iters.append(it)
        rel.append(rr.value)
    Ae, Af = np.zeros(9), np.zeros(9)
    lib().orc3_a_hom(n, h, float(L), _p(coef), scheme, _p(u), _p(Ae), _p(Af))
    return {"u": u, "iters": iters, "relres": rel, "A_energy": Ae.reshape(3, 3),
            "A_flux": Af.reshape(3, 3)}


def solve_realization3(d: dict, scheme: int = SCHEME_CONSISTENT, tol: float = 1e-12,
                       max_iter: int = 5000, want_u: bool = True) -> dict:
    n = int(d["L"]) * int(d["m0"])
    mask = np.zeros((n, n, n), dtype=np.uint8)
    u = np.zeros((3, n, n, n)) if want_u else None
    res = Result3()
    rc = lib().orc3_solve_realization(ctypes.byref(_real(d)), scheme, tol, max_iter, 0.0,
                                      _p(mask), _p(u) if want_u else None, ctypes.byref(res))
    if rc != 0:
        raise MemoryError("oracle 3D solve failed")
    return {"A_energy": np.array(res.A_energy).reshape(3, 3),
            "A_flux": np.array(res.A_flux).reshape(3, 3), "iters": list(res.iters),
            "relres": list(res.relres_true), "mean_a": res.mean_a, "u": u, "mask": mask}


def laplacian_eig(n: int, k1: int, k2: int) -> float:
    return float(lib().orc_laplacian_eig(n, k1, k2))


def precond(r: np.ndarray, c0: float, delta: float = 0.0) -> np.ndarray:
    r = np.ascontiguousarray(r, dtype=np.float64)
    n = r.shape[0]
    z = np.zeros_like(r)
    lib().orc_precond(n, c0, delta, _p(r), _p(z))
    return z


def pcg(csr, f: np.ndarray, c0: float, tol: float, max_iter: int, delta: float = 0.0):
    f = np.ascontiguousarray(f, dtype=np.float64)
    n = f.shape[0]
    u = np.zeros_like(f)
    rr = ctypes.c_double(0.0)
    rowptr, colidx, vals = csr
    it = lib().orc_pcg(n, _p(rowptr), _p(colidx), _p(vals), c0, delta, _p(f), tol, max_iter,
                       _p(u), ctypes.byref(rr))
    return u, int(it), float(rr.value)


def a_hom(coef: np.ndarray, u: np.ndarray, h: float, L: float, scheme: int = SCHEME_CONSISTENT):
    """(A_energy[2,2], A_flux[2,2]) from cell values and correctors u[2,n,n]."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    Ae = np.zeros(4)
    Af = np.zeros(4)
    lib().orc_a_hom(coef.shape[0], h, L, _p(coef), scheme, _p(u), _p(Ae), _p(Af))
    return Ae.reshape(2, 2), Af.reshape(2, 2)


def a_hom_grad(u: np.ndarray, G: np.ndarray, h: float, L: float,
               scheme: int = SCHEME_CONSISTENT) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64).ravel()
    n = u.shape[1]
    g = np.zeros((n, n))
    lib().orc_a_hom_grad(n, h, L, scheme, _p(u), _p(G), _p(g))
    return g


def solve_coef(coef: np.ndarray, L: int, m0: int, c0: float, scheme: int = SCHEME_CONSISTENT,
               tol: float = 1e-12, max_iter: int = 5000, delta: float = 0.0,
               want_u: bool = True):
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    n = coef.shape[0]
    u = np.zeros((2, n, n)) if want_u else None
    res = Result()
    rc = lib().orc_solve_coef(L, m0, _p(coef), c0, scheme, tol, max_iter, delta,
                              _p(u) if want_u else None, ctypes.byref(res))
    if rc != 0:
        raise ValueError(f"oracle solve failed (code {rc}; n must be a power of two)")
    return _result_dict(res, u)


def _result_dict(res: Result, u=None, mask=None) -> dict:
    out = {"A_energy": np.array(res.A_energy[:]).reshape(2, 2),
           "A_flux": np.array(res.A_flux[:]).reshape(2, 2),
           "relres_true": np.array(res.relres_true[:]),
           "iters": np.array(res.iters[:]), "mean_a": float(res.mean_a)}
    if u is not None:
        out["u"] = u
    if mask is not None:
        out["mask"] = mask
    return out


def solve_realization(d: dict, scheme: int = SCHEME_CONSISTENT, tol: float = 1e-12,
                      max_iter: int = 5000, delta: float = 0.0, want_u: bool = True) -> dict:
    n = int(d["L"]) * int(d["m0"])
    mask = np.zeros((n, n), dtype=np.uint8)
    u = np.zeros((2, n, n)) if want_u else None
    res = Result()
    rc = lib().orc_solve_realization(ctypes.byref(_real(d)), scheme, tol, max_iter, delta,
                                     _p(mask), _p(u) if want_u else None, ctypes.byref(res))
    if rc != 0:
        raise MemoryError("oracle solve failed")
    return _result_dict(res, u, mask)


def solve_batch(ds: list, scheme: int = SCHEME_CONSISTENT, tol: float = 1e-10,
                max_iter: int = 5000, delta: float = 0.0, threads: int = 0):
    """Many realizations, one per OpenMP thread.  Returns (A_energy[B,2,2], iters[B,2], threads)."""
    arr = (Realization * len(ds))(*[_real(d) for d in ds])
    res = (Result * len(ds))()
    used = lib().orc_solve_batch(ctypes.cast(arr, ctypes.c_void_p), len(ds), scheme, tol,
                                 max_iter, delta, ctypes.cast(res, ctypes.c_void_p), threads)
    A = np.array([np.array(r.A_energy[:]).reshape(2, 2) for r in res])
    it = np.array([r.iters[:] for r in res])
    return A, it, int(used)


def statistics(A: np.ndarray, L: float, d: int = 2) -> dict:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(-1, 4))
    N = A.shape[0]
    mean = np.zeros(4)
    var = np.zeros(4)
    Q = np.zeros(16)
    s12 = ctypes.c_double(0.0)
    sd = ctypes.c_double(0.0)
    lib().orc_statistics(N, _p(A), float(L), d, _p(mean), _p(var), ctypes.byref(s12),
                         ctypes.byref(sd), _p(Q))
    return {"mean": mean.reshape(2, 2), "var": var.reshape(2, 2), "std12_paper": s12.value,
            "stddiff_paper": sd.value, "Q": Q.reshape(4, 4)}


def statistics3(A: np.ndarray, L: float) -> dict:
    """Mean, unbiased variance and the 9x9 unfolding of L^3 cov(A) of 3D A_hom [N,3,3]."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(-1, 9))
    mean, var, Q = np.zeros(9), np.zeros(9), np.zeros(81)
    lib().orc3_statistics(A.shape[0], _p(A), float(L), _p(mean), _p(var), _p(Q))
    return {"mean": mean.reshape(3, 3), "var": var.reshape(3, 3), "Q": Q.reshape(9, 9)}
