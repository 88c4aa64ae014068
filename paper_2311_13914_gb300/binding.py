"""Thin ctypes binding of libbidomain.so (include/bidomain.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host, copied by the library) or CUDA
torch tensors (device pointers, ordered on the given stream).  The functions
keep the C names; errors raise BidomainError carrying the status code.
Loading fails loudly when the compiled library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbidomain.so")

BD_OK = 0
BD_EINVAL = -1
BD_ENOMEM = -2
BD_ENOTCONV = -3
BD_EBREAKDOWN = -4
BD_ETIMEOUT = -5
BD_ECUDA = -6
BD_EINCONSISTENT = -7
BD_ERANGE = -8
BD_ESTATE = -9


class BidomainError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {strerror(status)} ({status})")
        self.status = status


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double)]


class Params(C.Structure):
    _fields_ = [("chi", C.c_double), ("cm", C.c_double), ("dt", C.c_double),
                ("sil", C.c_double), ("sit", C.c_double), ("sel", C.c_double),
                ("set", C.c_double)]


class AmgOptions(C.Structure):
    _fields_ = [("theta", C.c_double), ("coarse_eq_limit", C.c_int), ("max_levels", C.c_int),
                ("cheb_degree", C.c_int), ("esteig_steps", C.c_int), ("square_levels", C.c_int),
                ("eig_lo", C.c_double), ("eig_hi", C.c_double), ("seed", C.c_ulonglong),
                ("precision", C.c_int), ("autotune", C.c_int)]


class SolveOptions(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_it", C.c_int), ("warm_start", C.c_int),
                ("strict", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("rel_res", C.c_double),
                ("true_rel_res", C.c_double), ("solve_ms", C.c_double),
                ("total_iters", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelProfile(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("total_ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double), ("precision", C.c_int), ("fp64_ops", C.c_double)]


class ServerOptions(C.Structure):
    _fields_ = [("hbm_budget", C.c_longlong), ("max_active", C.c_int), ("precision", C.c_int),
                ("rtol", C.c_double), ("max_it", C.c_int)]


class RequestInfo(C.Structure):
    _fields_ = [("state", C.c_int), ("steps_done", C.c_int), ("total_iters", C.c_longlong),
                ("submit_ms", C.c_double), ("admit_ms", C.c_double), ("done_ms", C.c_double),
                ("footprint", C.c_longlong), ("n_nodes", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RmParams(C.Structure):
    _fields_ = [("G", C.c_double), ("vth", C.c_double), ("vp", C.c_double),
                ("eta1", C.c_double), ("eta2", C.c_double), ("eta3", C.c_double)]


#: every entry point declared in include/bidomain.h
EXPORTS = (
    "bd_strerror", "bd_launch_count", "bd_spgemm_path_counts", "bd_dot_exact", "bd_dot_exact_noalloc",
    "amg_options_default", "solve_options_default", "bd_rm_params_default",
    "bd_assemble", "bd_system_info", "bd_system_export", "bd_system_destroy",
    "amg_setup", "amg_setup_from_csr", "amg_num_levels", "amg_level_info", "amg_level_lanes",
    "amg_set_level_lanes", "amg_export_level",
    "amg_vcycle", "amg_solve", "amg_destroy", "amg_batch_create", "amg_batch_solve",
    "amg_batch_destroy", "amg_stack_create", "amg_stack_solve", "amg_stack_info", "amg_stack_destroy",
    "amg_profile_enable", "amg_profile_read", "amg_profile_breakdown",
    "bd_sim_create", "bd_sim_set_state", "bd_sim_get_state", "bd_step", "bd_sim_destroy",
    "bd_elliptic_setup", "bd_dsim_create", "bd_dsim_set_state", "bd_dsim_get_state", "bd_dsim_step",
    "bd_dsim_destroy",
    "bd_server_options_default", "bd_server_create", "bd_server_submit", "bd_server_tick",
    "bd_server_drain", "bd_server_request", "bd_server_result", "bd_server_stats",
    "bd_server_destroy",
)

_lock = threading.Lock()
_lib = None
_P = C.POINTER
_vp = C.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
            L = C.CDLL(LIB_PATH)
            L.bd_strerror.restype = C.c_char_p
            L.bd_strerror.argtypes = [C.c_int]
            L.bd_dot_exact.argtypes = [_vp, _vp, C.c_longlong, C.c_int, _P(C.c_double), _vp]
            L.bd_dot_exact_noalloc.argtypes = [_vp, _vp, C.c_longlong, _vp, _vp]
            L.bd_launch_count.argtypes = []
            L.bd_launch_count.restype = C.c_longlong
            L.bd_spgemm_path_counts.argtypes = [_P(C.c_longlong), _P(C.c_longlong)]
            L.amg_options_default.argtypes = [_P(AmgOptions)]
            L.amg_options_default.restype = None
            L.solve_options_default.argtypes = [_P(SolveOptions)]
            L.solve_options_default.restype = None
            L.bd_rm_params_default.argtypes = [_P(RmParams)]
            L.bd_rm_params_default.restype = None
            L.bd_assemble.argtypes = [_P(Mesh), _P(Params), _vp, C.c_int, _vp, _P(_vp)]
            L.bd_system_info.argtypes = [_vp, _P(C.c_int), _P(C.c_longlong)]
            L.bd_system_export.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
            L.bd_system_destroy.argtypes = [_vp]
            L.bd_system_destroy.restype = None
            L.amg_setup.argtypes = [_vp, _P(AmgOptions), _vp, _P(_vp)]
            L.amg_setup_from_csr.argtypes = [C.c_int, _vp, _vp, _vp, C.c_int, _P(AmgOptions), _vp,
                                             _P(_vp)]
            L.amg_num_levels.argtypes = [_vp, _P(C.c_int)]
            L.amg_level_info.argtypes = [_vp, C.c_int, _P(C.c_int), _P(C.c_longlong),
                                         _P(C.c_int), _P(C.c_double), _P(C.c_longlong)]
            L.amg_level_lanes.argtypes = [_vp, C.c_int, _P(C.c_int)]
            L.amg_set_level_lanes.argtypes = [_vp, C.c_int, _P(C.c_int), _vp]
            L.amg_export_level.argtypes = [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
            L.amg_vcycle.argtypes = [_vp, _vp, _vp, C.c_int, _vp]
            L.amg_solve.argtypes = [_vp, _vp, _vp, C.c_int, _P(SolveOptions), _vp, _P(SolveInfo)]
            L.amg_batch_create.argtypes = [_P(_vp), C.c_int, _P(_vp)]
            L.amg_batch_solve.argtypes = [_vp, _P(_vp), _P(_vp), _P(SolveOptions), _vp, _P(SolveInfo)]
            L.amg_batch_destroy.argtypes = [_vp]
            L.amg_batch_destroy.restype = None
            L.amg_stack_create.argtypes = [_P(_vp), C.c_int, _vp, _P(_vp)]
            L.amg_stack_solve.argtypes = [_vp, _P(_vp), _P(_vp), _P(SolveOptions), _vp, _P(SolveInfo)]
            L.amg_stack_info.argtypes = [_vp, _P(C.c_int), _P(C.c_longlong)]
            L.amg_stack_destroy.argtypes = [_vp]
            L.amg_stack_destroy.restype = None
            L.amg_profile_enable.argtypes = [_vp, C.c_int]
            L.amg_profile_read.argtypes = [_vp, _P(KernelProfile)]
            L.amg_profile_breakdown.argtypes = [_vp, _P(C.c_double), _P(C.c_longlong)]
            L.amg_destroy.argtypes = [_vp]
            L.amg_destroy.restype = None
            L.bd_sim_create.argtypes = [_vp, _vp, _P(RmParams), _vp, C.c_int, C.c_double, _vp,
                                        _P(_vp)]
            L.bd_sim_set_state.argtypes = [_vp, _vp, _vp, _vp, C.c_int, _vp]
            L.bd_sim_get_state.argtypes = [_vp, _vp, _vp, _vp, C.c_int, _vp]
            L.bd_step.argtypes = [_vp, C.c_int, _P(SolveOptions), _vp, _P(SolveInfo)]
            L.bd_sim_destroy.argtypes = [_vp]
            L.bd_sim_destroy.restype = None
            L.bd_elliptic_setup.argtypes = [_vp, _P(AmgOptions), _vp, _P(_vp)]
            L.bd_dsim_create.argtypes = [_vp, _vp, _P(RmParams), _vp, C.c_int, C.c_double, C.c_int,
                                         _vp, _P(_vp)]
            L.bd_dsim_set_state.argtypes = [_vp, _vp, _vp, _vp, C.c_int, _vp]
            L.bd_dsim_get_state.argtypes = [_vp, _vp, _vp, _vp, C.c_int, _vp]
            L.bd_dsim_step.argtypes = [_vp, C.c_int, _P(SolveOptions), _vp, _P(SolveInfo),
                                       _P(SolveInfo)]
            L.bd_dsim_destroy.argtypes = [_vp]
            L.bd_dsim_destroy.restype = None
            L.bd_server_options_default.argtypes = [_P(ServerOptions)]
            L.bd_server_options_default.restype = None
            L.bd_server_create.argtypes = [_P(ServerOptions), _P(_vp)]
            L.bd_server_submit.argtypes = [_vp, _P(Mesh), _P(Params), _vp, _vp, C.c_double, C.c_int,
                                           _P(C.c_longlong)]
            L.bd_server_tick.argtypes = [_vp, _P(C.c_int), _P(C.c_int)]
            L.bd_server_drain.argtypes = [_vp]
            L.bd_server_request.argtypes = [_vp, C.c_longlong, _P(RequestInfo)]
            L.bd_server_result.argtypes = [_vp, C.c_longlong, _vp, _vp, _vp]
            L.bd_server_stats.argtypes = [_vp, _P(C.c_longlong), _P(C.c_longlong), _P(C.c_longlong)]
            L.bd_server_destroy.argtypes = [_vp]
            L.bd_server_destroy.restype = None
            _lib = L
    return _lib


def bd_launch_count() -> int:
    return lib().bd_launch_count()


def bd_spgemm_path_counts() -> tuple:
    """(hash-path calls, dense-path calls) of the setup's SpGEMM so far."""
    a, b = C.c_longlong(0), C.c_longlong(0)
    _check(lib().bd_spgemm_path_counts(C.byref(a), C.byref(b)), "bd_spgemm_path_counts")
    return a.value, b.value


def strerror(status: int) -> str:
    return lib().bd_strerror(status).decode()


def _check(st: int, what: str):
    if st != BD_OK:
        raise BidomainError(st, what)


def _arr(a, dtype):
    """(pointer, on_device, keepalive) for a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, 0, None
    mod = type(a).__module__
    if mod.startswith("torch"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {np.float64: "torch.float64", np.int32: "torch.int32"}[dtype]
        if str(a.dtype) != want:
            raise ValueError(f"tensor dtype must be {want}")
        return C.c_void_p(a.data_ptr()), int(a.is_cuda), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(_vp), 0, arr


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------------ handles
class _Handle:
    _destroy = None

    def __init__(self, ptr, keep=()):
        self.ptr = ptr
        self._keep = keep

    def close(self):
        if self.ptr:
            getattr(lib(), self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System(_Handle):
    _destroy = "bd_system_destroy"


class Hierarchy(_Handle):
    _destroy = "amg_destroy"


class Sim(_Handle):
    _destroy = "bd_sim_destroy"


# ------------------------------------------------------------------ defaults
def amg_options_default(**over) -> AmgOptions:
    o = AmgOptions()
    lib().amg_options_default(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def solve_options_default(**over) -> SolveOptions:
    o = SolveOptions()
    lib().solve_options_default(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def bd_rm_params_default(**over) -> RmParams:
    p = RmParams()
    lib().bd_rm_params_default(C.byref(p))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def bd_dot_exact(x, y, stream=None) -> float:
    px, dx, kx = _arr(x, np.float64)
    py, dy, ky = _arr(y, np.float64)
    if dx != dy:
        raise ValueError("x and y must both be host arrays or both device tensors")
    n = kx.numel() if dx else kx.size
    out = C.c_double()
    _check(lib().bd_dot_exact(px, py, n, dx, C.byref(out), _stream(stream)), "bd_dot_exact")
    return out.value


def bd_dot_exact_noalloc(x, y, out, stream=None):
    """Allocation-free reproducible dot of two CUDA tensors into the first
    element of the CUDA tensor `out` (stream-ordered, no synchronisation).
    stream=None runs on torch's current stream, the one the inputs were most
    likely written on."""
    import torch

    px, dx, kx = _arr(x, np.float64)
    py, dy, ky = _arr(y, np.float64)
    po, do, ko = _arr(out, np.float64)
    if not (dx and dy and do):
        raise ValueError("x, y and out must be CUDA tensors")
    if kx.numel() != ky.numel():
        raise ValueError("x and y must have the same length")
    if ko.numel() < 1:
        raise ValueError("out must hold at least one element")
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().bd_dot_exact_noalloc(px, py, kx.numel(), po, _stream(stream)),
           "bd_dot_exact_noalloc")
    return out


# ------------------------------------------------------------------ a0
def bd_assemble(mesh: dict, params: dict, fib, stream=None) -> System:
    m = Mesh(mesh["nx"], mesh["ny"], mesh["nz"], mesh["lx"], mesh["ly"], mesh["lz"])
    p = Params(params["chi"], params["cm"], params["dt"], params["sil"], params["sit"],
               params["sel"], params["set"])
    fp, dev, keep = _arr(fib, np.float64)
    out = _vp()
    _check(lib().bd_assemble(C.byref(m), C.byref(p), fp, dev, _stream(stream), C.byref(out)),
           "bd_assemble")
    return System(out)


def bd_system_info(sys: System):
    n, nnz = C.c_int(), C.c_longlong()
    _check(lib().bd_system_info(sys.ptr, C.byref(n), C.byref(nnz)), "bd_system_info")
    return n.value, nnz.value


def bd_system_export(sys: System, stream=None):
    """Returns (row_ptr, col, val, M) as numpy arrays (scalar CSR of A)."""
    N, nnz = bd_system_info(sys)
    rp = np.zeros(2 * N + 1, np.int32)
    ci = np.zeros(nnz, np.int32)
    v = np.zeros(nnz)
    M = np.zeros(N)
    _check(lib().bd_system_export(sys.ptr, rp.ctypes.data_as(_vp), ci.ctypes.data_as(_vp),
                                  v.ctypes.data_as(_vp), M.ctypes.data_as(_vp), _stream(stream)),
           "bd_system_export")
    return rp, ci, v, M


# ------------------------------------------------------------------ a1..a9
def amg_setup(sys: System, opts: AmgOptions | None = None, stream=None) -> Hierarchy:
    out = _vp()
    o = opts if opts is not None else amg_options_default()
    _check(lib().amg_setup(sys.ptr, C.byref(o), _stream(stream), C.byref(out)), "amg_setup")
    return Hierarchy(out)


def amg_setup_from_csr(n: int, row_ptr, col, val, opts: AmgOptions | None = None,
                       stream=None) -> Hierarchy:
    rp, d1, k1 = _arr(row_ptr, np.int32)
    ci, d2, k2 = _arr(col, np.int32)
    v, d3, k3 = _arr(val, np.float64)
    if not (d1 == d2 == d3):
        raise ValueError("row_ptr, col and val must all be on the host or all on the device")
    out = _vp()
    o = opts if opts is not None else amg_options_default()
    _check(lib().amg_setup_from_csr(n, rp, ci, v, d1, C.byref(o), _stream(stream), C.byref(out)),
           "amg_setup_from_csr")
    return Hierarchy(out)


def amg_num_levels(h: Hierarchy) -> int:
    n = C.c_int()
    _check(lib().amg_num_levels(h.ptr, C.byref(n)), "amg_num_levels")
    return n.value


def amg_level_info(h: Hierarchy, level: int) -> dict:
    n, nnz, na, lam, pn = C.c_int(), C.c_longlong(), C.c_int(), C.c_double(), C.c_longlong()
    _check(lib().amg_level_info(h.ptr, level, C.byref(n), C.byref(nnz), C.byref(na), C.byref(lam),
                                C.byref(pn)), "amg_level_info")
    return dict(n=n.value, nnz=nnz.value, n_agg=na.value, lam=lam.value, p_nnz=pn.value)


def amg_level_lanes(h: Hierarchy, level: int) -> tuple:
    """Form of A_l, R_l, P_l in the V-cycle: T > 0 block CSR with T lanes per
    row, -K the sliced form with K lanes per row, 0 not applied in block form."""
    lanes = (C.c_int * 3)()
    _check(lib().amg_level_lanes(h.ptr, level, lanes), "amg_level_lanes")
    return tuple(lanes)


def amg_set_level_lanes(h: Hierarchy, level: int, lanes, stream=None) -> None:
    """Override the forms of A_l, R_l, P_l (values as amg_level_lanes gives
    them, 0 keeps one)."""
    arr = (C.c_int * 3)(*[int(t) for t in lanes])
    _check(lib().amg_set_level_lanes(h.ptr, level, arr, _stream(stream)), "amg_set_level_lanes")


def amg_export_level(h: Hierarchy, level: int, stream=None) -> dict:
    info = amg_level_info(h, level)
    n, nnz, pn = info["n"], info["nnz"], info["p_nnz"]
    N = n // 2
    arp, aci, av = np.zeros(n + 1, np.int32), np.zeros(nnz, np.int32), np.zeros(nnz)
    mis, agg = np.zeros(N, np.uint8), np.zeros(N, np.int32)
    prp, pci, pv = np.zeros(n + 1, np.int32), np.zeros(pn, np.int32), np.zeros(pn)
    ptr = lambda a: a.ctypes.data_as(_vp)  # noqa: E731
    last = info["n_agg"] == 0
    _check(lib().amg_export_level(h.ptr, level, ptr(arp), ptr(aci), ptr(av),
                                  None if last else ptr(mis), None if last else ptr(agg),
                                  None if last else ptr(prp), None if last else ptr(pci),
                                  None if last else ptr(pv), _stream(stream)), "amg_export_level")
    out = dict(info, A=(arp, aci, av))
    if not last:
        out.update(mis=mis, agg=agg, P=(prp, pci, pv))
    return out


# ------------------------------------------------------------------ a10, a11
def amg_vcycle(h: Hierarchy, r, z=None, stream=None):
    rp, d1, k1 = _arr(r, np.float64)
    if d1:
        zp, d2, k2 = _arr(z, np.float64)
        _check(lib().amg_vcycle(h.ptr, rp, zp, 1, _stream(stream)), "amg_vcycle")
        return z
    out = np.zeros_like(np.asarray(r, dtype=np.float64))
    _check(lib().amg_vcycle(h.ptr, rp, out.ctypes.data_as(_vp), 0, _stream(stream)), "amg_vcycle")
    return out


def amg_solve(h: Hierarchy, f, x=None, opts: SolveOptions | None = None, stream=None,
              raise_on_error: bool = True):
    """Solve A x = f.  numpy in -> numpy out (x created if None); torch CUDA
    tensors are used in place.  Returns (x, info dict)."""
    o = opts if opts is not None else solve_options_default()
    fp, dev, kf = _arr(f, np.float64)
    if x is None:
        if dev:
            raise ValueError("pass a device x for device f")
        x = np.zeros(np.asarray(f).shape, np.float64)
    xp, dx, kx = _arr(x, np.float64)
    if dx != dev:
        raise ValueError("f and x must both be host arrays or both device tensors")
    if not dev and kx is not x:
        raise ValueError("host x must be a contiguous float64 numpy array")
    info = SolveInfo()
    st = lib().amg_solve(h.ptr, fp, xp, dev, C.byref(o), _stream(stream), C.byref(info))
    if raise_on_error and st not in (BD_OK,):
        raise BidomainError(st, "amg_solve")
    return x, info.as_dict()


class Batch(_Handle):
    _destroy = "amg_batch_destroy"


def amg_batch_create(hs) -> Batch:
    """One CUDA graph over the whole solves of distinct hierarchies hs."""
    arr = (_vp * len(hs))(*[h.ptr for h in hs])
    out = _vp()
    _check(lib().amg_batch_create(arr, len(hs), C.byref(out)), "amg_batch_create")
    return Batch(out, keep=tuple(hs))


def amg_batch_solve(b: Batch, fs, xs, opts: SolveOptions | None = None, stream=None,
                    raise_on_error: bool = True) -> list:
    """Solve every system of the batch in one graph launch.  fs, xs: CUDA
    float64 tensors (x used in place).  Returns the per-solve info dicts."""
    n = len(fs)
    if len(xs) != n:
        raise ValueError("fs and xs differ in length")
    fp, xp = (_vp * n)(), (_vp * n)()
    for k in range(n):
        pf, df, _ = _arr(fs[k], np.float64)
        px, dx, _ = _arr(xs[k], np.float64)
        if not (df and dx):
            raise ValueError("batched solves take CUDA tensors")
        fp[k], xp[k] = pf, px
    o = opts if opts is not None else solve_options_default()
    infos = (SolveInfo * n)()
    st = lib().amg_batch_solve(b.ptr, fp, xp, C.byref(o), _stream(stream), infos)
    if raise_on_error and st != BD_OK:
        raise BidomainError(st, "amg_batch_solve")
    return [i.as_dict() for i in infos]


class Stack(_Handle):
    _destroy = "amg_stack_destroy"


def amg_stack_create(hs, stream=None) -> Stack:
    """Stack the hierarchies hs level by level: one launch per V-cycle step
    for all of them (the hierarchies must outlive the stack)."""
    arr = (_vp * len(hs))(*[h.ptr for h in hs])
    out = _vp()
    _check(lib().amg_stack_create(arr, len(hs), _stream(stream), C.byref(out)), "amg_stack_create")
    return Stack(out, keep=tuple(hs))


def amg_stack_solve(b: Stack, fs, xs, opts: SolveOptions | None = None, stream=None,
                    raise_on_error: bool = True) -> list:
    """Solve every member system in one graph launch.  fs, xs: CUDA float64
    tensors (x used in place).  Returns the per-member info dicts."""
    n = len(fs)
    if len(xs) != n:
        raise ValueError("fs and xs differ in length")
    fp, xp = (_vp * n)(), (_vp * n)()
    for k in range(n):
        pf, df, _ = _arr(fs[k], np.float64)
        px, dx, _ = _arr(xs[k], np.float64)
        if not (df and dx):
            raise ValueError("stacked solves take CUDA tensors")
        fp[k], xp[k] = pf, px
    o = opts if opts is not None else solve_options_default()
    infos = (SolveInfo * n)()
    st = lib().amg_stack_solve(b.ptr, fp, xp, C.byref(o), _stream(stream), infos)
    if raise_on_error and st != BD_OK:
        raise BidomainError(st, "amg_stack_solve")
    return [i.as_dict() for i in infos]


def amg_stack_info(b: Stack) -> dict:
    lv, nl = C.c_int(0), C.c_longlong(0)
    _check(lib().amg_stack_info(b.ptr, C.byref(lv), C.byref(nl)), "amg_stack_info")
    return {"levels": lv.value, "launches_per_iteration": nl.value}


def amg_profile_enable(h: Hierarchy, enable: int = 1):
    """0 off, 1 finest-operator timing, 2 also the per-step breakdown."""
    _check(lib().amg_profile_enable(h.ptr, int(enable)), "amg_profile_enable")


PROFILE_ROLES = ("pre", "residual", "restrict", "prolong", "post1", "post2")
PROFILE_STEPS = ("coarse", "vcycle_in", "vcycle_out", "z_stats", "p_update", "A_p", "x_r_update")


def amg_profile_breakdown(h: Hierarchy) -> dict:
    """{step name: (ms, count)} of the per-step breakdown (profiling level 2)."""
    ms, cnt = (C.c_double * 256)(), (C.c_longlong * 256)()
    _check(lib().amg_profile_breakdown(h.ptr, ms, cnt), "amg_profile_breakdown")
    out = {}
    for i in range(256):
        if cnt[i]:
            lv, role = divmod(i, 16)
            name = PROFILE_STEPS[role] if lv == 15 else f"L{lv}_{PROFILE_ROLES[role]}"
            out[name] = (ms[i], cnt[i])
    return out


def amg_profile_read(h: Hierarchy) -> dict:
    p = KernelProfile()
    _check(lib().amg_profile_read(h.ptr, C.byref(p)), "amg_profile_read")
    return {k: getattr(p, k) for k, _ in p._fields_}


# ------------------------------------------------------------------ a12
def bd_sim_create(sys: System, h: Hierarchy, rm: RmParams | None = None, stim=None,
                  stim_ms: float = 0.0, stream=None) -> Sim:
    sp_, dev, ks = _arr(stim, np.float64)
    out = _vp()
    r = rm if rm is not None else bd_rm_params_default()
    _check(lib().bd_sim_create(sys.ptr, h.ptr, C.byref(r), sp_, dev, stim_ms, _stream(stream),
                               C.byref(out)), "bd_sim_create")
    return Sim(out, keep=(sys, h))


def bd_sim_set_state(sim: Sim, v=None, ue=None, w=None, stream=None):
    a, d1, k1 = _arr(v, np.float64)
    b, d2, k2 = _arr(ue, np.float64)
    c, d3, k3 = _arr(w, np.float64)
    dev = max(d1, d2, d3)
    _check(lib().bd_sim_set_state(sim.ptr, a, b, c, dev, _stream(stream)), "bd_sim_set_state")


def bd_sim_get_state(sim: Sim, N: int, stream=None, out=None):
    """Copy (v, u_e, w) to host arrays; `out` may give three float64 host
    arrays or CPU tensors (e.g. pinned) of length N to fill."""
    if out is None:
        out = (np.zeros(N), np.zeros(N), np.zeros(N))
    ptrs = [_arr(a, np.float64) for a in out]
    if any(d for _, d, _ in ptrs):
        raise ValueError("bd_sim_get_state copies to host arrays")
    for (_, _, k), a in zip(ptrs, out):
        if k is not a:
            raise ValueError("output arrays must be contiguous float64")
    _check(lib().bd_sim_get_state(sim.ptr, ptrs[0][0], ptrs[1][0], ptrs[2][0], 0, _stream(stream)),
           "bd_sim_get_state")
    return out


# ------------------------------------------------------------------ decoupled scheme
class DSim(_Handle):
    _destroy = "bd_dsim_destroy"


def bd_elliptic_setup(sys: System, opts: AmgOptions | None = None, stream=None) -> Hierarchy:
    """Hierarchy of the elliptic operator Ai + Ae (as [I, 0; 0, Ai + Ae])."""
    out = _vp()
    o = opts if opts is not None else amg_options_default()
    _check(lib().bd_elliptic_setup(sys.ptr, C.byref(o), _stream(stream), C.byref(out)),
           "bd_elliptic_setup")
    return Hierarchy(out)


def bd_dsim_create(sys: System, h_elliptic: Hierarchy, rm: RmParams | None = None, stim=None,
                   stim_ms: float = 0.0, jacobi: bool = True, stream=None) -> DSim:
    sp_, dev, ks = _arr(stim, np.float64)
    out = _vp()
    r = rm if rm is not None else bd_rm_params_default()
    _check(lib().bd_dsim_create(sys.ptr, h_elliptic.ptr, C.byref(r), sp_, dev, stim_ms,
                                int(bool(jacobi)), _stream(stream), C.byref(out)), "bd_dsim_create")
    return DSim(out, keep=(sys, h_elliptic))


def bd_dsim_set_state(sim: DSim, v=None, ue=None, w=None, stream=None):
    a, d1, k1 = _arr(v, np.float64)
    b, d2, k2 = _arr(ue, np.float64)
    c, d3, k3 = _arr(w, np.float64)
    dev = max(d1, d2, d3)
    _check(lib().bd_dsim_set_state(sim.ptr, a, b, c, dev, _stream(stream)), "bd_dsim_set_state")


def bd_dsim_get_state(sim: DSim, N: int, stream=None):
    out = (np.zeros(N), np.zeros(N), np.zeros(N))
    ptrs = [_arr(a, np.float64) for a in out]
    _check(lib().bd_dsim_get_state(sim.ptr, ptrs[0][0], ptrs[1][0], ptrs[2][0], 0, _stream(stream)),
           "bd_dsim_get_state")
    return out


def bd_dsim_step(sim: DSim, nsteps: int, opts: SolveOptions | None = None, stream=None,
                 raise_on_error: bool = True) -> tuple:
    """Returns (elliptic info, parabolic info) of the last step, with totals."""
    o = opts if opts is not None else solve_options_default()
    ie, ip = SolveInfo(), SolveInfo()
    st = lib().bd_dsim_step(sim.ptr, nsteps, C.byref(o), _stream(stream), C.byref(ie), C.byref(ip))
    if raise_on_error and st != BD_OK:
        raise BidomainError(st, "bd_dsim_step")
    return ie.as_dict(), ip.as_dict()


def bd_step(sim: Sim, nsteps: int, opts: SolveOptions | None = None, stream=None,
            raise_on_error: bool = True) -> dict:
    o = opts if opts is not None else solve_options_default()
    info = SolveInfo()
    st = lib().bd_step(sim.ptr, nsteps, C.byref(o), _stream(stream), C.byref(info))
    if raise_on_error and st != BD_OK:
        raise BidomainError(st, "bd_step")
    return info.as_dict()


# ------------------------------------------------------------------ serving
class Server(_Handle):
    _destroy = "bd_server_destroy"


def bd_server_options_default(**over) -> ServerOptions:
    o = ServerOptions()
    lib().bd_server_options_default(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def bd_server_create(opts: ServerOptions | None = None) -> Server:
    out = _vp()
    o = opts if opts is not None else bd_server_options_default()
    _check(lib().bd_server_create(C.byref(o), C.byref(out)), "bd_server_create")
    return Server(out)


def bd_server_submit(srv: Server, mesh: dict, params: dict, fib, stim=None, stim_ms: float = 0.0,
                     nsteps: int = 1) -> int:
    m = Mesh(mesh["nx"], mesh["ny"], mesh["nz"], mesh["lx"], mesh["ly"], mesh["lz"])
    p = Params(params["chi"], params["cm"], params["dt"], params["sil"], params["sit"],
               params["sel"], params["set"])
    f = np.ascontiguousarray(fib, dtype=np.float64).reshape(-1)
    st_ = None if stim is None else np.ascontiguousarray(stim, dtype=np.float64)
    rid = C.c_longlong()
    _check(lib().bd_server_submit(srv.ptr, C.byref(m), C.byref(p), f.ctypes.data_as(_vp),
                                  None if st_ is None else st_.ctypes.data_as(_vp), stim_ms, nsteps,
                                  C.byref(rid)), "bd_server_submit")
    return rid.value


def bd_server_tick(srv: Server):
    a, q = C.c_int(), C.c_int()
    _check(lib().bd_server_tick(srv.ptr, C.byref(a), C.byref(q)), "bd_server_tick")
    return a.value, q.value


def bd_server_drain(srv: Server):
    _check(lib().bd_server_drain(srv.ptr), "bd_server_drain")


def bd_server_request(srv: Server, rid: int) -> dict:
    r = RequestInfo()
    _check(lib().bd_server_request(srv.ptr, rid, C.byref(r)), "bd_server_request")
    return r.as_dict()


def bd_server_result(srv: Server, rid: int):
    n = bd_server_request(srv, rid)["n_nodes"]
    v, ue, w = np.zeros(n), np.zeros(n), np.zeros(n)
    _check(lib().bd_server_result(srv.ptr, rid, v.ctypes.data_as(_vp), ue.ctypes.data_as(_vp),
                                  w.ctypes.data_as(_vp)), "bd_server_result")
    return v, ue, w


def bd_server_stats(srv: Server) -> dict:
    a, b, c = C.c_longlong(), C.c_longlong(), C.c_longlong()
    _check(lib().bd_server_stats(srv.ptr, C.byref(a), C.byref(b), C.byref(c)), "bd_server_stats")
    return dict(solves=a.value, resident_bytes=b.value, budget_bytes=c.value)
