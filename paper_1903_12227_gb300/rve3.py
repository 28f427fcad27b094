"""Python binding of the 3D entry points of librve (rve3_* in include/rve.h).

Argument marshalling only.  Layouts: a batch of cubic realizations is packed
back to back, n^3 nodes each (node (i1, i2, i3) at (i1 n + i2) n + i3); the
cube mask holds one byte per cell; vectors of the three correctors are
float64 ``[nodes, 3]``, so an equal-size batch views as
``u.view(batch, n, n, n, 3)``.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import torch

from . import rve
from .rve import CONSISTENT, Realization, RveError, _ptr, _require_cuda, _stream, check


class Solve3Opts(ctypes.Structure):
    """rve3_solve_opts (40 bytes); zero fields take the library defaults."""
    _fields_ = [("scheme", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("tol", ctypes.c_double), ("delta", ctypes.c_double),
                ("inner_tol", ctypes.c_double)]


class Solve3Info(ctypes.Structure):
    """rve3_solve_info (48 bytes)."""
    _fields_ = [("iters", ctypes.c_int32 * 3), ("status", ctypes.c_int32),
                ("refinements", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("relres", ctypes.c_double * 3)]


INFO3_BYTES = ctypes.sizeof(Solve3Info)
_bound = False


def lib() -> ctypes.CDLL:
    global _bound
    L = rve.lib()
    if not _bound:
        vp, i32, i64, sz, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
        L.rve3_nodes.restype = i64
        L.rve3_nodes.argtypes = [vp, i32]
        L.rve3_workspace_size.restype = sz
        L.rve3_workspace_size.argtypes = [vp, i32]
        L.rve3_gen_field.restype = i32
        L.rve3_gen_field.argtypes = [vp, i32, vp, vp]
        L.rve3_rhs.restype = i32
        L.rve3_rhs.argtypes = [vp, i32, vp, vp, i32, vp, vp, sz, vp]
        L.rve3_apply_stiffness.restype = i32
        L.rve3_apply_stiffness.argtypes = [vp, i32, vp, vp, i32, vp, vp, vp, sz, vp]
        L.rve3_apply_precond.restype = i32
        L.rve3_apply_precond.argtypes = [vp, i32, dbl, vp, vp, vp, sz, vp]
        L.rve3_solve_correctors.restype = i32
        L.rve3_solve_correctors.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, sz, vp]
        L.rve3_a_hom.restype = i32
        L.rve3_a_hom.argtypes = [vp, i32, vp, vp, i32, vp, vp, vp, vp, sz, vp]
        L.rve3_profile_read.restype = i32
        L.rve3_profile_read.argtypes = [vp, vp]
        L.rve3_statistics.restype = i32
        L.rve3_statistics.argtypes = [vp, i64, dbl, vp, vp, vp]
        _bound = True
    return L


class Batch3:
    """A host array of rve_realization describing cubic realizations."""

    def __init__(self, descs: Sequence[dict]):
        self.descs = list(descs)
        self.count = len(self.descs)
        self.arr = (Realization * self.count)(*[
            Realization(int(d["L"]), int(d["m0"]), int(d["incl_cells"]), int(d["n_incl"]),
                        float(d["a_matrix"]), float(d["a_incl"]),
                        int(d["seed"]) & (2**64 - 1), int(d["index"]) & (2**64 - 1))
            for d in self.descs])
        self.ns = [int(d["L"]) * int(d["m0"]) for d in self.descs]
        self.nodes = sum(n ** 3 for n in self.ns)

    @property
    def ptr(self) -> ctypes.c_void_p:
        return ctypes.cast(self.arr, ctypes.c_void_p)

    def offsets(self) -> list:
        out, o = [], 0
        for n in self.ns:
            out.append(o)
            o += n ** 3
        return out


def as_batch3(b) -> Batch3:
    return b if isinstance(b, Batch3) else Batch3(b)


def make_opts3(scheme=CONSISTENT, precision=rve.FP64, tol=1e-10, max_iter=0, delta=0.0,
               check_every=0, inner_tol=0.0) -> Solve3Opts:
    return Solve3Opts(scheme, precision, max_iter, check_every, tol, delta, inner_tol)


def workspace_size3(batch) -> int:
    b = as_batch3(batch)
    nb = lib().rve3_workspace_size(b.ptr, b.count)
    if nb == 0:
        raise RveError("rve3_workspace_size: invalid batch")
    return int(nb)


def _ws(b: Batch3, ws, device):
    nb = workspace_size3(b)
    if ws is None or ws.numel() < nb:
        ws = rve.workspace(nb, device)
    return ws


def _device(*ts):
    for t in ts:
        if t is not None:
            return t.device
    return torch.device("cuda", torch.cuda.current_device())


def gen_field(batch, device=None, stream=None) -> torch.Tensor:
    """Cube mask, uint8 [nodes] (one byte per cell)."""
    _require_cuda()
    b = as_batch3(batch)
    dev = torch.device(device) if device is not None else _device()
    mask = torch.empty(b.nodes, dtype=torch.uint8, device=dev)
    check(lib().rve3_gen_field(b.ptr, b.count, _ptr(mask), _stream(stream)), "rve3_gen_field")
    return mask


def rhs(batch, mask=None, coef=None, scheme=CONSISTENT, ws=None, stream=None) -> torch.Tensor:
    """The three corrector loads, float64 [nodes, 3]."""
    _require_cuda()
    b = as_batch3(batch)
    dev = _device(mask, coef)
    ws = _ws(b, ws, dev)
    f = torch.empty(b.nodes, 3, dtype=torch.float64, device=dev)
    check(lib().rve3_rhs(b.ptr, b.count, _ptr(mask), _ptr(coef), scheme, _ptr(f), _ptr(ws),
                         ws.numel(), _stream(stream)), "rve3_rhs")
    return f


def apply_stiffness(batch, x: torch.Tensor, mask=None, coef=None, scheme=CONSISTENT, ws=None,
                    stream=None) -> torch.Tensor:
    """y = A x for float64 [nodes, 3]."""
    _require_cuda()
    b = as_batch3(batch)
    if x.dtype != torch.float64 or tuple(x.shape) != (b.nodes, 3):
        raise ValueError("x must be float64 [nodes, 3]")
    ws = _ws(b, ws, x.device)
    y = torch.empty_like(x)
    check(lib().rve3_apply_stiffness(b.ptr, b.count, _ptr(mask), _ptr(coef), scheme, _ptr(x),
                                     _ptr(y), _ptr(ws), ws.numel(), _stream(stream)),
          "rve3_apply_stiffness")
    return y


def apply_precond(batch, x: torch.Tensor, delta=0.0, ws=None, stream=None) -> torch.Tensor:
    """y = B^{-1} x, B = c0 A_Delta + delta I, for float64 [nodes, 3]."""
    _require_cuda()
    b = as_batch3(batch)
    if x.dtype != torch.float64 or tuple(x.shape) != (b.nodes, 3):
        raise ValueError("x must be float64 [nodes, 3]")
    ws = _ws(b, ws, x.device)
    y = torch.empty_like(x)
    check(lib().rve3_apply_precond(b.ptr, b.count, float(delta), _ptr(x), _ptr(y), _ptr(ws),
                                   ws.numel(), _stream(stream)), "rve3_apply_precond")
    return y


def solve(batch, mask=None, coef=None, opts: Solve3Opts | None = None, ws=None, stream=None):
    """The three correctors u [nodes, 3] float64 and the raw info tensor."""
    _require_cuda()
    b = as_batch3(batch)
    opts = opts or make_opts3()
    dev = _device(mask, coef)
    ws = _ws(b, ws, dev)
    u = torch.empty(b.nodes, 3, dtype=torch.float64, device=dev)
    info = torch.empty(b.count * INFO3_BYTES, dtype=torch.uint8, device=dev)
    check(lib().rve3_solve_correctors(b.ptr, b.count, _ptr(mask), _ptr(coef), ctypes.byref(opts),
                                      _ptr(u), _ptr(info), _ptr(ws), ws.numel(),
                                      _stream(stream)), "rve3_solve_correctors")
    return u, info


def decode_info(info: torch.Tensor) -> list:
    raw = info.cpu().numpy().tobytes()
    out = []
    for k in range(len(raw) // INFO3_BYTES):
        s = Solve3Info.from_buffer_copy(raw[k * INFO3_BYTES:(k + 1) * INFO3_BYTES])
        out.append({"iters": list(s.iters), "status": int(s.status),
                    "refinements": int(s.refinements), "relres": list(s.relres)})
    return out


def a_hom(batch, u: torch.Tensor, mask=None, coef=None, scheme=CONSISTENT, ws=None,
          want_flux: bool = False, stream=None):
    """Energy-form A [batch, 3, 3] (and the flux form if asked), float64."""
    _require_cuda()
    b = as_batch3(batch)
    ws = _ws(b, ws, u.device)
    A = torch.empty(b.count, 9, dtype=torch.float64, device=u.device)
    Af = torch.empty(b.count, 9, dtype=torch.float64, device=u.device) if want_flux else None
    check(lib().rve3_a_hom(b.ptr, b.count, _ptr(mask), _ptr(coef), scheme, _ptr(u), _ptr(A),
                           _ptr(Af), _ptr(ws), ws.numel(), _stream(stream)), "rve3_a_hom")
    A = A.view(b.count, 3, 3)
    return (A, Af.view(b.count, 3, 3)) if want_flux else A


def statistics(A, L: float) -> dict:
    """Ensemble mean, unbiased variance and Q = L^3 cov (9x9 unfolding of the
    quartic tensor) of 3D A_hom [N, 3, 3] (host arithmetic, index order)."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(A.cpu() if hasattr(A, "cpu") else A,
                                        dtype=np.float64).reshape(-1, 9))
    mean, var, Q = np.zeros(9), np.zeros(9), np.zeros(81)
    p = lambda x: ctypes.c_void_p(x.ctypes.data)
    check(lib().rve3_statistics(p(a), a.shape[0], float(L), p(mean), p(var), p(Q)),
          "rve3_statistics")
    return {"mean": mean.reshape(3, 3), "var": var.reshape(3, 3), "Q": Q.reshape(9, 9)}


PROFILE_KINDS = ("stiffness", "lines", "zsolve", "vector", "scalar", "resid64")


def profile_read() -> dict:
    """Per-kind totals {kind: (ms, launches)} of the 3D solver's launches
    since the last read (collected while rve.profile_enable(True))."""
    ms = (ctypes.c_double * len(PROFILE_KINDS))()
    cnt = (ctypes.c_int64 * len(PROFILE_KINDS))()
    k = lib().rve3_profile_read(ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(cnt, ctypes.c_void_p))
    return {PROFILE_KINDS[j]: (ms[j], int(cnt[j])) for j in range(k)}


def homogenize(batch, scheme=CONSISTENT, tol=1e-10, delta=0.0, precision=rve.FP64, stream=None):
    """Field, correctors and A_hom of every realization: (A [batch,3,3], info list)."""
    b = as_batch3(batch)
    mask = gen_field(b, stream=stream)
    ws = _ws(b, None, mask.device)
    u, info = solve(b, mask=mask, opts=make_opts3(scheme=scheme, precision=precision, tol=tol,
                                                  delta=delta), ws=ws, stream=stream)
    A = a_hom(b, u, mask=mask, scheme=scheme, ws=ws, stream=stream)
    return A, decode_info(info)
