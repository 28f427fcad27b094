"""Python binding of librve (the C ABI in include/rve.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  PyTorch provides device memory (tensors, workspaces) and streams.
The binding fails loudly if ``librve.so`` is missing or no GPU is present;
there is no CPU fallback.

Layouts (see include/rve.h): a batch of realizations is packed back to back;
per node the two correctors are interleaved, so a solution tensor has shape
``[nodes, 2]`` (float64), i.e. ``[sum_b n_b^2, 2]``; for equal-size batches
``u.view(batch, n, n, 2)``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librve.so")

RVE_OK, RVE_EINVAL, RVE_ENOCONV, RVE_ENAN, RVE_ETIMEOUT, RVE_ECUDA, RVE_ENOMEM, RVE_ESCRATCH = range(8)
NOALLOC_MAX_NODES = 1 << 24
FP64, MIXED = 0, 1
CONSISTENT, LUMPED = 0, 1
PATH_FUSED, PATH_PLAIN, PATH_PERSISTENT = 0, 1, 2


class Realization(ctypes.Structure):
    """rve_realization (48 bytes)."""
    _fields_ = [("L", ctypes.c_int32), ("m0", ctypes.c_int32),
                ("incl_cells", ctypes.c_int32), ("n_incl", ctypes.c_int32),
                ("a_matrix", ctypes.c_double), ("a_incl", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("index", ctypes.c_uint64)]


class SolveOpts(ctypes.Structure):
    """rve_solve_opts; zero fields take the library defaults."""
    _fields_ = [("scheme", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("path", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("tol", ctypes.c_double), ("delta", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("tile_rows", ctypes.c_int32),
                ("col_tile", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("timeout_us", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32 * 2), ("status", ctypes.c_int32),
                ("refinements", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("relres", ctypes.c_double * 2)]


INFO_BYTES = ctypes.sizeof(SolveInfo)
_lib = None


class RveError(RuntimeError):
    pass


def lib() -> ctypes.CDLL:
    """Load librve.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RveError(f"{LIB_PATH} not found: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                 ctypes.c_double, ctypes.c_size_t)
        L.rve_status_string.restype = ctypes.c_char_p
        L.rve_status_string.argtypes = [i32]
        L.rve_version.restype = i32
        L.rve_last_error.restype = ctypes.c_char_p
        L.rve_last_error.argtypes = []
        L.rve_mask_words.restype = i64
        L.rve_mask_words.argtypes = [vp, i32]
        L.rve_nodes.restype = i64
        L.rve_nodes.argtypes = [vp, i32]
        L.rve_gen_field.restype = i32
        L.rve_gen_field.argtypes = [vp, i32, vp, vp]
        L.rve_coef_from_mask.restype = i32
        L.rve_coef_from_mask.argtypes = [vp, i32, vp, vp, vp]
        L.rve_rhs.restype = i32
        L.rve_rhs.argtypes = [vp, i32, vp, vp, vp, vp]
        L.rve_apply_stiffness.restype = i32
        L.rve_apply_stiffness.argtypes = [vp, i32, vp, vp, i32, i32, vp, vp, vp]
        L.rve_apply_precond.restype = i32
        L.rve_apply_precond.argtypes = [vp, i32, dbl, i32, vp, vp, vp, sz, vp]
        L.rve_workspace_size.restype = sz
        L.rve_workspace_size.argtypes = [vp, i32, vp]
        L.rve_solve_correctors.restype = i32
        L.rve_solve_correctors.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, sz, vp]
        L.rve_solve_rhs.restype = i32
        L.rve_solve_rhs.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.rve_apply_mass.restype = i32
        L.rve_apply_mass.argtypes = [vp, i32, i32, vp, vp, vp]
        L.rve_cheb_workspace_size.restype = sz
        L.rve_cheb_workspace_size.argtypes = [vp, i32]
        L.rve_cheb_moments.restype = i32
        L.rve_cheb_moments.argtypes = [vp, i32, vp, vp, i32, vp, i32, ctypes.c_double,
                                       ctypes.c_double, vp, vp, sz, vp]
        L.rve_dos_coefficients.restype = i32
        L.rve_dos_coefficients.argtypes = [vp, i32, i32, dbl, dbl, dbl, i32, vp]
        L.rve_dos_from_moments.restype = i32
        L.rve_dos_from_moments.argtypes = [vp, i32, dbl, dbl, dbl, dbl, vp, i32, vp]
        L.rve_a_hom.restype = i32
        L.rve_a_hom.argtypes = [vp, i32, vp, vp, i32, i32, vp, vp, vp, vp, vp, sz, vp]
        L.rve_a_hom_backward.restype = i32
        L.rve_a_hom_backward.argtypes = [vp, i32, i32, vp, vp, vp, vp]
        L.rve_homogenize_workspace_size.restype = sz
        L.rve_homogenize_workspace_size.argtypes = [vp, i32, vp]
        L.rve_homogenize_host.restype = i32
        L.rve_homogenize_host.argtypes = [vp, i32, vp, vp, vp, vp, sz, vp]
        L.rve_statistics.restype = i32
        L.rve_statistics.argtypes = [vp, i64, dbl, i32, vp, vp, vp, vp, vp]
        L.rve_plan_create.restype = i32
        L.rve_plan_create.argtypes = [vp, i32, vp, ctypes.POINTER(vp)]
        L.rve_plan_workspace_size.restype = sz
        L.rve_plan_workspace_size.argtypes = [vp]
        L.rve_plan_execute.restype = i32
        L.rve_plan_execute.argtypes = [vp, vp, vp, vp, sz, vp]
        L.rve_plan_destroy.restype = None
        L.rve_plan_destroy.argtypes = [vp]
        L.rve_autotune.restype = i32
        L.rve_autotune.argtypes = [vp, i32, vp, vp, sz, vp]
        L.rve_tuner_save.restype = i32
        L.rve_tuner_save.argtypes = [ctypes.c_char_p]
        L.rve_tuner_load.restype = i32
        L.rve_tuner_load.argtypes = [ctypes.c_char_p]
        L.rve_tuner_lookup.restype = i32
        L.rve_tuner_lookup.argtypes = [i32, i32, i32, vp, vp]
        L.rve_tuner_clear.restype = None
        L.rve_tuner_clear.argtypes = []
        L.rve_profile_enable.restype = None
        L.rve_profile_enable.argtypes = [i32]
        L.rve_profile_read.restype = i32
        L.rve_profile_read.argtypes = [vp, vp]
        L.rve_launch_count.restype = i64
        L.rve_launch_count.argtypes = []
        _lib = L
    return _lib


def check(status: int, what: str = "") -> None:
    if status != RVE_OK:
        msg = lib().rve_status_string(status).decode()
        if status == RVE_ECUDA:
            msg += f" ({lib().rve_last_error().decode()})"
        raise RveError(f"{what}: {msg}" if what else msg)


def _require_cuda():
    if not torch.cuda.is_available():
        raise RveError("librve needs a CUDA GPU; none is available")


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(None)
    return ctypes.c_void_p(t.data_ptr())


def _np_ptr(a) -> ctypes.c_void_p:
    """Address of a C-contiguous numpy array (host memory)."""
    return ctypes.c_void_p(a.ctypes.data)


class Batch:
    """A host array of rve_realization built from workload dicts."""

    def __init__(self, descs: Sequence[dict]):
        self.descs = list(descs)
        self.count = len(self.descs)
        self.arr = (Realization * self.count)(*[
            Realization(int(d["L"]), int(d["m0"]), int(d["incl_cells"]), int(d["n_incl"]),
                        float(d["a_matrix"]), float(d["a_incl"]),
                        int(d["seed"]) & (2**64 - 1), int(d["index"]) & (2**64 - 1))
            for d in self.descs])
        self.ns = [int(d["L"]) * int(d["m0"]) for d in self.descs]
        self.nodes = sum(n * n for n in self.ns)
        self.words = self.nodes // 32

    @property
    def ptr(self) -> ctypes.c_void_p:
        return ctypes.cast(self.arr, ctypes.c_void_p)

    def offsets(self) -> list:
        out, o = [], 0
        for n in self.ns:
            out.append(o)
            o += n * n
        return out


def as_batch(b) -> Batch:
    return b if isinstance(b, Batch) else Batch(b)


def make_opts(scheme=CONSISTENT, precision=FP64, path=PATH_FUSED, tol=1e-10, max_iter=0,
              delta=0.0, inner_tol=0.0, tile_rows=0, col_tile=0, check_every=0,
              timeout_us=0, flags=0) -> SolveOpts:
    return SolveOpts(scheme, precision, path, max_iter, tol, delta, inner_tol, tile_rows,
                     col_tile, check_every, timeout_us, flags, 0)


def _dev(device):
    return torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())


# ------------------------------------------------------------------ calls --
def gen_field(batch, device=None, stream=None) -> torch.Tensor:
    """Bitmask of the covered cells, int32 words [words] (Sec. 2, Eq. "Stoch-decomp")."""
    _require_cuda()
    b = as_batch(batch)
    mask = torch.empty(b.words, dtype=torch.int32, device=_dev(device))
    check(lib().rve_gen_field(b.ptr, b.count, _ptr(mask), _stream(stream)), "rve_gen_field")
    return mask


def rhs(batch, mask=None, coef=None, device=None, stream=None) -> torch.Tensor:
    _require_cuda()
    b = as_batch(batch)
    f = torch.empty(b.nodes, 2, dtype=torch.float64, device=_dev(device))
    check(lib().rve_rhs(b.ptr, b.count, _ptr(mask), _ptr(coef), _ptr(f), _stream(stream)),
          "rve_rhs")
    return f


def apply_stiffness(batch, x: torch.Tensor, mask=None, coef=None, scheme=CONSISTENT,
                    stream=None) -> torch.Tensor:
    _require_cuda()
    b = as_batch(batch)
    prec = FP64 if x.dtype == torch.float64 else MIXED
    y = torch.empty_like(x)
    check(lib().rve_apply_stiffness(b.ptr, b.count, _ptr(mask), _ptr(coef), scheme, prec,
                                    _ptr(x), _ptr(y), _stream(stream)), "rve_apply_stiffness")
    return y


def workspace(nbytes: int, device=None) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=_dev(device))


def apply_precond(batch, x: torch.Tensor, delta: float = 0.0, stream=None) -> torch.Tensor:
    _require_cuda()
    b = as_batch(batch)
    prec = FP64 if x.dtype == torch.float64 else MIXED
    nb = lib().rve_workspace_size(b.ptr, b.count, None)
    if nb == 0:
        raise RveError("rve_workspace_size: invalid batch")
    ws = workspace(nb, x.device)
    y = torch.empty_like(x)
    check(lib().rve_apply_precond(b.ptr, b.count, float(delta), prec, _ptr(x), _ptr(y),
                                  _ptr(ws), ws.numel(), _stream(stream)), "rve_apply_precond")
    return y


def workspace_size(batch, opts: SolveOpts | None = None) -> int:
    b = as_batch(batch)
    nb = lib().rve_workspace_size(b.ptr, b.count, ctypes.byref(opts) if opts else None)
    if nb == 0:
        raise RveError("rve_workspace_size: invalid batch or options")
    return int(nb)


def info_to_dicts(info: torch.Tensor, count: int) -> list:
    raw = info.cpu().numpy().tobytes()
    arr = (SolveInfo * count).from_buffer_copy(raw)
    return [_info_dict(a) for a in arr]


def _info_dict(a: SolveInfo) -> dict:
    return {"iters": (a.iters[0], a.iters[1]), "status": a.status, "refinements": a.refinements,
            "steps": a.steps, "relres": (a.relres[0], a.relres[1])}


def solve(batch, mask=None, coef=None, opts: SolveOpts | None = None, ws=None, u=None,
          info=None, stream=None, device=None, f: torch.Tensor | None = None):
    """Correctors u [nodes, 2] float64 and the raw info tensor (Sec. 3.4, 4.1).
    With `f` (device float64 [nodes, 2], each component mean-zero per
    realization) the two load vectors of f are solved for instead."""
    _require_cuda()
    b = as_batch(batch)
    opts = opts or make_opts()
    dev = (mask if mask is not None else coef).device if (mask is not None or coef is not None) else _dev(device)
    nb = workspace_size(b, opts)
    if ws is None or ws.numel() < nb:
        ws = workspace(nb, dev)
    if u is None:
        u = torch.empty(b.nodes, 2, dtype=torch.float64, device=dev)
    if info is None:
        info = torch.empty(b.count * INFO_BYTES, dtype=torch.uint8, device=dev)
    if f is None:
        check(lib().rve_solve_correctors(b.ptr, b.count, _ptr(mask), _ptr(coef),
                                         ctypes.byref(opts), _ptr(u), _ptr(info), _ptr(ws),
                                         ws.numel(), _stream(stream)), "rve_solve_correctors")
    else:
        if f.dtype != torch.float64 or tuple(f.shape) != (b.nodes, 2):
            raise ValueError("f must be float64 [nodes, 2]")
        check(lib().rve_solve_rhs(b.ptr, b.count, _ptr(mask), _ptr(coef), _ptr(f),
                                  ctypes.byref(opts), _ptr(u), _ptr(info), _ptr(ws),
                                  ws.numel(), _stream(stream)), "rve_solve_rhs")
    return u, info


def cheb_moments(batch, v: torch.Tensor, K: int, lo: float, hi: float, mask=None, coef=None,
                 scheme=CONSISTENT, stream=None) -> torch.Tensor:
    """mu [B, 2, K] (device float64): v_c^T T_k(A~) v_c for the two start
    vectors per realization (rve_cheb_moments), A~ = (2A - (hi+lo)) / (hi-lo)."""
    _require_cuda()
    b = as_batch(batch)
    if v.dtype != torch.float64 or tuple(v.shape) != (b.nodes, 2):
        raise ValueError("v must be float64 [nodes, 2]")
    nb = lib().rve_cheb_workspace_size(b.ptr, b.count)
    if nb == 0:
        raise RveError("rve_cheb_workspace_size: invalid batch")
    ws = workspace(nb, v.device)
    mu = torch.empty(b.count, 2, K, dtype=torch.float64, device=v.device)
    check(lib().rve_cheb_moments(b.ptr, b.count, _ptr(mask), _ptr(coef), scheme, _ptr(v), int(K),
                                 float(lo), float(hi), _ptr(mu), _ptr(ws), ws.numel(),
                                 _stream(stream)), "rve_cheb_moments")
    return mu


def apply_mass(batch, x: torch.Tensor, scheme=CONSISTENT, stream=None) -> torch.Tensor:
    """y = M x (Q1 mass matrix of the scheme) for float64 [nodes, 2] nodal values."""
    _require_cuda()
    b = as_batch(batch)
    if x.dtype != torch.float64:
        raise ValueError("apply_mass takes float64 nodal values")
    y = torch.empty_like(x)
    check(lib().rve_apply_mass(b.ptr, b.count, scheme, _ptr(x), _ptr(y), _stream(stream)),
          "rve_apply_mass")
    return y


def coef_from_mask(batch, mask: torch.Tensor, stream=None) -> torch.Tensor:
    """Cell values [nodes] float64 (a_matrix / a_incl) from the bitmask."""
    _require_cuda()
    b = as_batch(batch)
    coef = torch.empty(b.nodes, dtype=torch.float64, device=mask.device)
    check(lib().rve_coef_from_mask(b.ptr, b.count, _ptr(mask), _ptr(coef), _stream(stream)),
          "rve_coef_from_mask")
    return coef


def a_hom(batch, u: torch.Tensor, mask=None, coef=None, scheme=CONSISTENT, ws=None,
          want_flux: bool = False, stream=None, precision=FP64, want_lo: bool = False):
    """Energy-form A [batch, 2, 2] (and the flux form if asked), float64.

    precision FP64 sums in double-double arithmetic (A correctly rounded; with
    want_lo the low parts A_lo [batch, 2, 2] are returned too, A + A_lo being
    the energy to ~1e-30 relative); MIXED sums in double words on the FP32
    pipe (the mixed-precision pipeline's reduction).  Returns A, or a tuple
    (A, A_flux) / (A, A_lo) / (A, A_lo, A_flux) as asked."""
    _require_cuda()
    b = as_batch(batch)
    if want_lo and precision != FP64:
        raise ValueError("A_lo exists for precision FP64 only")
    nb = workspace_size(b, make_opts(scheme=scheme))
    if ws is None or ws.numel() < nb:
        ws = workspace(nb, u.device)
    A = torch.empty(b.count, 4, dtype=torch.float64, device=u.device)
    Af = torch.empty(b.count, 4, dtype=torch.float64, device=u.device) if want_flux else None
    Alo = torch.empty(b.count, 4, dtype=torch.float64, device=u.device) if want_lo else None
    check(lib().rve_a_hom(b.ptr, b.count, _ptr(mask), _ptr(coef), scheme, precision, _ptr(u),
                          _ptr(A), _ptr(Alo), _ptr(Af), _ptr(ws), ws.numel(), _stream(stream)),
          "rve_a_hom")
    out = [A.view(b.count, 2, 2)]
    if want_lo:
        out.append(Alo.view(b.count, 2, 2))
    if want_flux:
        out.append(Af.view(b.count, 2, 2))
    return out[0] if len(out) == 1 else tuple(out)


def a_hom_backward(batch, u: torch.Tensor, gradA: torch.Tensor, scheme=CONSISTENT,
                   stream=None) -> torch.Tensor:
    """d(sum_ij G_ij A_ij)/d a_c per cell, float64 [nodes]."""
    _require_cuda()
    b = as_batch(batch)
    G = gradA.detach().to(torch.float64).contiguous().view(b.count, 4)
    g = torch.empty(b.nodes, dtype=torch.float64, device=u.device)
    check(lib().rve_a_hom_backward(b.ptr, b.count, scheme, _ptr(u), _ptr(G), _ptr(g),
                                   _stream(stream)), "rve_a_hom_backward")
    return g


def homogenize_host(batch, opts: SolveOpts | None = None, ws=None, stream=None, device=None):
    """Whole pipeline with host in/out: returns (A numpy [B,2,2], info list)."""
    import numpy as np
    _require_cuda()
    b = as_batch(batch)
    opts = opts or make_opts()
    nb = lib().rve_homogenize_workspace_size(b.ptr, b.count, ctypes.byref(opts))
    if nb == 0:
        raise RveError("rve_homogenize_workspace_size: invalid batch or options")
    if ws is None or ws.numel() < nb:
        ws = workspace(nb, device)
    A = np.zeros((b.count, 4), dtype=np.float64)
    info = (SolveInfo * b.count)()
    check(lib().rve_homogenize_host(b.ptr, b.count, ctypes.byref(opts),
                                    A.ctypes.data_as(ctypes.c_void_p),
                                    ctypes.cast(info, ctypes.c_void_p), _ptr(ws), ws.numel(),
                                    _stream(stream)), "rve_homogenize_host")
    return A.reshape(b.count, 2, 2), [_info_dict(i) for i in info]


class Plan:
    """Whole pipeline of a fixed batch captured once into a CUDA graph
    (rve_plan_*): opts.path PATH_PERSISTENT solves in one persistent launch,
    PATH_FUSED runs the fused kernels inside a conditional while node.
    execute() returns A [B,2,2] (device, float64) and the raw info tensor;
    calls after the first relaunch the graph."""

    def __init__(self, batch, opts: SolveOpts | None = None, device=None):
        _require_cuda()
        self.batch = as_batch(batch)
        self.opts = opts or make_opts(precision=MIXED, path=PATH_PERSISTENT)
        h = ctypes.c_void_p()
        check(lib().rve_plan_create(self.batch.ptr, self.batch.count, ctypes.byref(self.opts),
                                    ctypes.byref(h)), "rve_plan_create")
        self.handle = h
        dev = _dev(device)
        self.ws = workspace(lib().rve_plan_workspace_size(h), dev)
        self.A = torch.empty(self.batch.count, 4, dtype=torch.float64, device=dev)
        self.info = torch.empty(self.batch.count * INFO_BYTES, dtype=torch.uint8, device=dev)
        # graphs cannot be captured on the legacy default stream: own stream
        self.stream = torch.cuda.Stream(device=dev)

    def execute(self):
        """Launch (capturing on the first call) on the plan's stream; the
        caller's current stream then waits for it."""
        cur = torch.cuda.current_stream(self.A.device)
        self.stream.wait_stream(cur)
        check(lib().rve_plan_execute(self.handle, _ptr(self.A), _ptr(self.info), _ptr(self.ws),
                                     self.ws.numel(), _stream(self.stream)), "rve_plan_execute")
        cur.wait_stream(self.stream)
        return self.A.view(self.batch.count, 2, 2), self.info

    def close(self):
        if getattr(self, "handle", None):
            lib().rve_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(batch, opts: SolveOpts | None = None, ws_bytes: int | None = None, stream=None,
             device=None) -> None:
    """Time candidate tile shapes per grid size and record the fastest (rve_autotune)."""
    _require_cuda()
    b = as_batch(batch)
    opts = opts or make_opts()
    if ws_bytes is None:
        sub = Batch(b.descs[:16])
        ws_bytes = 4 * workspace_size(sub, make_opts(precision=FP64)) + (64 << 20)
    ws = workspace(ws_bytes, device)
    check(lib().rve_autotune(b.ptr, b.count, ctypes.byref(opts), _ptr(ws), ws.numel(),
                             _stream(stream)), "rve_autotune")


def tuner_save(path: str) -> None:
    check(lib().rve_tuner_save(path.encode()), "rve_tuner_save")


def tuner_load(path: str) -> None:
    check(lib().rve_tuner_load(path.encode()), "rve_tuner_load")


def tuner_lookup(n: int, precision: int, persistent: bool):
    ts, bc = ctypes.c_int32(0), ctypes.c_int32(0)
    found = lib().rve_tuner_lookup(n, precision, 1 if persistent else 0, ctypes.byref(ts),
                                   ctypes.byref(bc))
    return (ts.value, bc.value) if found else None


def tuner_clear() -> None:
    lib().rve_tuner_clear()


def statistics(A, L: float, d: int = 2) -> dict:
    """Ensemble statistics of homogenized matrices A [N,2,2] (host, FP64, index order)."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(-1, 4))
    mean, var, Q = np.zeros(4), np.zeros(4), np.zeros(16)
    s12, sd = ctypes.c_double(0.0), ctypes.c_double(0.0)
    vp = ctypes.c_void_p
    check(lib().rve_statistics(a.ctypes.data_as(vp), a.shape[0], float(L), int(d),
                               mean.ctypes.data_as(vp), var.ctypes.data_as(vp), ctypes.byref(s12),
                               ctypes.byref(sd), Q.ctypes.data_as(vp)), "rve_statistics")
    return {"mean": mean.reshape(2, 2), "var": var.reshape(2, 2), "std12_paper": s12.value,
            "stddiff_paper": sd.value, "Q": Q.reshape(4, 4), "count": a.shape[0]}


def profile_enable(on: bool = True) -> None:
    lib().rve_profile_enable(1 if on else 0)


def profile_read() -> dict:
    import numpy as np
    ms = np.zeros(5)
    ln = np.zeros(5, dtype=np.int64)
    lib().rve_profile_read(ms.ctypes.data_as(ctypes.c_void_p), ln.ctypes.data_as(ctypes.c_void_p))
    names = ("refine", "stencil", "update_row", "column", "control")
    return {k: {"ms": float(ms[i]), "launches": int(ln[i])} for i, k in enumerate(names)}


def launch_count() -> int:
    return int(lib().rve_launch_count())


def unpack_mask(mask: torch.Tensor, batch) -> list:
    """Per-realization boolean [n, n] CPU tensors from the packed bitmask."""
    b = as_batch(batch)
    words = mask.cpu().view(torch.int32).numpy().view("uint32")
    import numpy as np
    out, w0 = [], 0
    for n in b.ns:
        nw = n * n // 32
        bits = np.unpackbits(words[w0:w0 + nw].view(np.uint8), bitorder="little")
        out.append(bits.reshape(n, n).astype(bool))
        w0 += nw
    return out


# ------------------------------------------------------------- autograd --
class AHom(torch.autograd.Function):
    """A_hom (energy form) as a differentiable function of the cell values.

    forward(coef [nodes] float64, batch, opts) -> A [batch, 2, 2]; the solve
    runs on the library's fused path with the preconditioner scale taken from
    each realization's two coefficient values.  backward returns
    dA/dcoef contracted with the incoming gradient, from the hand-written
    adjoint kernel (self-adjoint problem: no second solve).
    """

    @staticmethod
    def forward(ctx, coef: torch.Tensor, batch, opts: SolveOpts | None = None):
        b = as_batch(batch)
        opts = opts or make_opts()
        coef = coef.detach().to(torch.float64).contiguous()
        u, info = solve(b, coef=coef, opts=opts)
        A = a_hom(b, u, coef=coef, scheme=opts.scheme, precision=opts.precision)
        ctx.save_for_backward(u)
        ctx.batch = b
        ctx.scheme = opts.scheme
        ctx.info = info
        return A

    @staticmethod
    def backward(ctx, gA: torch.Tensor):
        (u,) = ctx.saved_tensors
        g = a_hom_backward(ctx.batch, u, gA, scheme=ctx.scheme)
        return g, None, None
