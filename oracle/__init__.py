"""FP64 CPU oracle for the coupled-Bidomain SA-AMG-PCG hot path.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` load it; the product library never does.  It
shares no code with the CUDA path.  The arithmetic lives in ``bd_oracle.c``
(plain C, compiled with ``-ffp-contract=off``); this module only marshals numpy
/ scipy arrays in and out through ctypes.

Every function follows a passage of arXiv 2311.13914 (cited in bd_oracle.c).
Pins that tie it to the paper and to mathematics, not to itself, live in
``tests/test_oracle_*.py``.  Every function is pinned: assembly (closed-form
stencils, patch test, second-order convergence, and the fibre field sampled at
the Gauss z-levels against an independent quadrature), the correctly rounded
dot, strength, the squared strength graph (against a dense (I + W)^2), MIS and
aggregation (brute force on the plain and the squared graph), prolongators,
Galerkin operators (dense triple product), eigen-estimate (closed-form 1-D
Laplacian, dense bisection), smoother (closed-form error polynomial), coarse
solve, V-cycle and PCG (dense pseudo-inverse), the time step (explicit Euler
when space-clamped) and the decoupled scheme (dense solves).  The paper prints
no worked example for this system, so no stored value comes from it; the
stored 100-step and large-slab runs are written from this module alone.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bd_oracle.c")
_HDR = os.path.join(_HERE, "bd_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile bd_oracle.c into oracle/_build/liboracle.so (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_SO) or max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_SO)
    if stale:
        tmp = _SO + f".tmp{os.getpid()}"
        try:
            # the solve phase's independent loops in parallel (bitwise the same
            # results for any thread count); serial if OpenMP is unavailable
            subprocess.check_call(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _CSR(C.Structure):
    _fields_ = [("nrows", C.c_int), ("ncols", C.c_int), ("nnz", C.c_int64),
                ("rp", C.POINTER(C.c_int64)), ("ci", C.POINTER(C.c_int)),
                ("v", C.POINTER(C.c_double))]


class _Opts(C.Structure):
    _fields_ = [("theta", C.c_double), ("coarse_eq_limit", C.c_int), ("max_levels", C.c_int),
                ("cheb_degree", C.c_int), ("esteig_steps", C.c_int), ("eig_lo", C.c_double),
                ("eig_hi", C.c_double), ("seed", C.c_uint64), ("square_levels", C.c_int)]


class _RM(C.Structure):
    _fields_ = [("G", C.c_double), ("vth", C.c_double), ("vp", C.c_double),
                ("eta1", C.c_double), ("eta2", C.c_double), ("eta3", C.c_double)]


_P = C.POINTER
_d = C.c_double
_i = C.c_int
_i64 = C.c_int64
_u64 = C.c_uint64
_vp = C.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.oc_csr_free.argtypes = [_P(_CSR)]
            L.oc_dot_exact.argtypes = [_i64, _vp, _vp]
            L.oc_set_threads.argtypes = [_i]
            L.oc_get_threads.argtypes = []
            L.oc_dot_exact.restype = _d
            L.oc_sum_exact.argtypes = [_i64, _vp]
            L.oc_sum_exact.restype = _d
            L.oc_assemble.argtypes = [_i, _i, _i, _d, _d, _d, _vp, _d, _d, _d, _d, _d, _d, _d,
                                      _P(_CSR), _P(_CSR), _vp, _P(_CSR)]
            L.oc_spmv.argtypes = [_P(_CSR), _vp, _vp]
            L.oc_transpose.argtypes = [_P(_CSR), _P(_CSR)]
            L.oc_spgemm.argtypes = [_P(_CSR), _P(_CSR), _P(_CSR)]
            L.oc_strength.argtypes = [_P(_CSR), _d, _P(_CSR)]
            L.oc_square_graph.argtypes = [_P(_CSR), _P(_CSR)]
            L.oc_mix64.argtypes = [_u64]
            L.oc_mix64.restype = _u64
            L.oc_level_key.argtypes = [_u64, _i, _i]
            L.oc_level_key.restype = _u64
            L.oc_mis.argtypes = [_P(_CSR), _u64, _vp]
            L.oc_aggregate.argtypes = [_P(_CSR), _vp, _vp, _P(_i)]
            L.oc_ptent.argtypes = [_i, _vp, _i, _vp, _P(_CSR), _vp]
            L.oc_lambda_max.argtypes = [_P(_CSR), _i, _u64, _P(_d), _P(_i)]
            L.oc_tridiag_max_eig.argtypes = [_i, _vp, _vp]
            L.oc_tridiag_max_eig.restype = _d
            L.oc_smooth_p.argtypes = [_P(_CSR), _P(_CSR), _d, _P(_CSR)]
            L.oc_setup.argtypes = [_P(_CSR), _P(_Opts), _P(_vp)]
            L.oc_hier_free.argtypes = [_vp]
            L.oc_hier_nlevels.argtypes = [_vp]
            for nm in ("oc_hier_A", "oc_hier_P", "oc_hier_Pt"):
                getattr(L, nm).argtypes = [_vp, _i]
                getattr(L, nm).restype = _P(_CSR)
            L.oc_hier_agg.argtypes = [_vp, _i]
            L.oc_hier_agg.restype = _P(_i)
            L.oc_hier_mis.argtypes = [_vp, _i]
            L.oc_hier_mis.restype = _P(C.c_ubyte)
            L.oc_hier_nagg.argtypes = [_vp, _i]
            L.oc_hier_lambda.argtypes = [_vp, _i]
            L.oc_hier_lambda.restype = _d
            L.oc_hier_null.argtypes = [_vp, _i]
            L.oc_hier_null.restype = _P(_d)
            L.oc_chebyshev.argtypes = [_P(_CSR), _vp, _vp, _i, _i, _d, _d]
            L.oc_coarse_solve.argtypes = [_vp, _vp, _vp]
            L.oc_vcycle.argtypes = [_vp, _vp, _vp]
            L.oc_pcg.argtypes = [_vp, _vp, _vp, _i, _d, _i, _P(_i), _P(_d), _P(_d)]
            L.oc_bd_step.argtypes = [_vp, _vp, _i, _d, _d, _d, _P(_RM), _vp, _vp, _vp, _vp,
                                     _d, _i, _P(_i)]
            L.oc_elliptic_block.argtypes = [_P(_CSR), _P(_CSR), _P(_CSR)]
            L.oc_parabolic_cg.argtypes = [_P(_CSR), _vp, _d, _vp, _vp, _d, _i, _i, _P(_i), _P(_d)]
            L.oc_bd_step_decoupled.argtypes = [_vp, _P(_CSR), _vp, _i, _d, _d, _d, _P(_RM), _vp,
                                               _vp, _vp, _vp, _d, _i, _i, _P(_i), _P(_i)]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_vp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _In:
    """Borrowed view of a scipy CSR as an oc_csr (keeps the arrays alive)."""

    def __init__(self, m: sp.csr_matrix):
        m = sp.csr_matrix(m)
        m.sort_indices()
        self.rp = np.ascontiguousarray(m.indptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(m.indices, dtype=np.int32)
        self.v = _f64(m.data)
        self.s = _CSR(m.shape[0], m.shape[1], int(m.nnz),
                      self.rp.ctypes.data_as(_P(_i64)), self.ci.ctypes.data_as(_P(_i)),
                      self.v.ctypes.data_as(_P(_d)))


def _view(c: _CSR) -> sp.csr_matrix:
    n, m, nnz = c.nrows, c.ncols, c.nnz
    rp = np.ctypeslib.as_array(c.rp, shape=(n + 1,)).copy()
    if nnz:
        ci = np.ctypeslib.as_array(c.ci, shape=(nnz,)).copy()
        v = np.ctypeslib.as_array(c.v, shape=(nnz,)).copy()
    else:
        ci = np.zeros(0, np.int32)
        v = np.zeros(0)
    return sp.csr_matrix((v, ci, rp), shape=(n, m))


def _own(c: _CSR) -> sp.csr_matrix:
    out = _view(c)
    lib().oc_csr_free(C.byref(c))
    return out


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


# ---------------------------------------------------------------- primitives
def set_threads(n: int) -> None:
    """Threads of the oracle's solve phase (results do not depend on it)."""
    _check(lib().oc_set_threads(int(n)), "set_threads")


def get_threads() -> int:
    return lib().oc_get_threads()


def dot_exact(x, y) -> float:
    x, y = _f64(x), _f64(y)
    return lib().oc_dot_exact(x.size, _ptr(x), _ptr(y))


def sum_exact(x) -> float:
    x = _f64(x)
    return lib().oc_sum_exact(x.size, _ptr(x))


def mix64(z: int) -> int:
    return lib().oc_mix64(z & (2**64 - 1))


def level_key(seed: int, level: int, stream: int) -> int:
    return lib().oc_level_key(seed & (2**64 - 1), level, stream)


def assemble(mesh: dict, params: dict, fib: np.ndarray) -> dict:
    """a0: returns dict(Ki, Ke, M, A) (scipy CSR / numpy)."""
    nx, ny, nz = mesh["nx"], mesh["ny"], mesh["nz"]
    fib = _f64(fib).reshape(-1)
    if fib.size != nz * 6:
        raise ValueError("fibre table must hold nz*2*3 values")
    N = (nx + 1) * (ny + 1) * (nz + 1)
    Ki, Ke, A = _CSR(), _CSR(), _CSR()
    M = np.zeros(N)
    rc = lib().oc_assemble(nx, ny, nz, mesh["lx"], mesh["ly"], mesh["lz"], _ptr(fib),
                           params["sil"], params["sit"], params["sel"], params["set"],
                           params["chi"], params["cm"], params["dt"],
                           C.byref(Ki), C.byref(Ke), _ptr(M), C.byref(A))
    _check(rc, "assemble")
    return {"Ki": _own(Ki), "Ke": _own(Ke), "M": M, "A": _own(A)}


def spmv(A, x):
    a = _In(A)
    x = _f64(x)
    y = np.zeros(A.shape[0])
    lib().oc_spmv(C.byref(a.s), _ptr(x), _ptr(y))
    return y


def transpose(A):
    a, out = _In(A), _CSR()
    _check(lib().oc_transpose(C.byref(a.s), C.byref(out)), "transpose")
    return _own(out)


def spgemm(A, B):
    a, b, out = _In(A), _In(B), _CSR()
    _check(lib().oc_spgemm(C.byref(a.s), C.byref(b.s), C.byref(out)), "spgemm")
    return _own(out)


def strength(A, theta: float):
    a, out = _In(A), _CSR()
    _check(lib().oc_strength(C.byref(a.s), theta, C.byref(out)), "strength")
    return _own(out)


def square_graph(S):
    s, out = _In(S), _CSR()
    _check(lib().oc_square_graph(C.byref(s.s), C.byref(out)), "square_graph")
    return _own(out)


def mis(S, key: int) -> np.ndarray:
    s = _In(S)
    out = np.zeros(S.shape[0], np.uint8)
    _check(lib().oc_mis(C.byref(s.s), key & (2**64 - 1), _ptr(out)), "mis")
    return out


def aggregate(S, in_set):
    s = _In(S)
    in_set = np.ascontiguousarray(in_set, dtype=np.uint8)
    agg = np.zeros(S.shape[0], np.int32)
    na = C.c_int(0)
    _check(lib().oc_aggregate(C.byref(s.s), _ptr(in_set), _ptr(agg), C.byref(na)), "aggregate")
    return agg, na.value


def ptent(agg, n_agg: int, B):
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    B = _f64(B)
    out = _CSR()
    Bc = np.zeros(2 * n_agg)
    _check(lib().oc_ptent(agg.size, _ptr(agg), n_agg, _ptr(B), C.byref(out), _ptr(Bc)), "ptent")
    return _own(out), Bc


def lambda_max(A, steps: int, key: int):
    a = _In(A)
    lam = C.c_double(0.0)
    done = C.c_int(0)
    _check(lib().oc_lambda_max(C.byref(a.s), steps, key & (2**64 - 1), C.byref(lam),
                               C.byref(done)), "lambda_max")
    return lam.value, done.value


def tridiag_max_eig(d, e) -> float:
    d = _f64(d)
    e = _f64(e) if len(e) else np.zeros(1)
    return lib().oc_tridiag_max_eig(d.size, _ptr(d), _ptr(e))


def smooth_p(A, Pt, omega: float):
    a, p, out = _In(A), _In(Pt), _CSR()
    _check(lib().oc_smooth_p(C.byref(a.s), C.byref(p.s), omega, C.byref(out)), "smooth_p")
    return _own(out)


def elliptic_block(Ki, Ke):
    """f4: the elliptic operator Ai + Ae as the 2x2-block operator
    [I, 0; 0, Ai + Ae] on the node pattern (explicit zeros kept)."""
    a, b, out = _In(Ki), _In(Ke), _CSR()
    _check(lib().oc_elliptic_block(C.byref(a.s), C.byref(b.s), C.byref(out)), "elliptic_block")
    return _own(out)


def parabolic_cg(Ki, M, c: float, b, v0, rtol=1e-8, max_it=500, jacobi=True):
    """f4: (c M + Ai) v = b by (Jacobi-preconditioned) CG from v0."""
    k = _In(Ki)
    M, b = _f64(M), _f64(b)
    v = _f64(v0).copy()
    it, rr = C.c_int(0), C.c_double(0)
    rc = lib().oc_parabolic_cg(C.byref(k.s), _ptr(M), c, _ptr(b), _ptr(v), rtol, max_it,
                               int(bool(jacobi)), C.byref(it), C.byref(rr))
    return v, dict(status=rc, iters=it.value, rel_res=rr.value)


def chebyshev(A, f, x0, degree: int, lo: float, hi: float, x_is_zero: bool = False):
    a = _In(A)
    f = _f64(f)
    x = _f64(np.zeros(A.shape[0]) if x0 is None else x0).copy()
    _check(lib().oc_chebyshev(C.byref(a.s), _ptr(f), _ptr(x), int(x_is_zero), degree, lo, hi),
           "chebyshev")
    return x


DEFAULT_OPTS = dict(theta=0.06, coarse_eq_limit=100, max_levels=10, cheb_degree=2,
                    esteig_steps=10, eig_lo=0.05, eig_hi=1.05, seed=0, square_levels=16)

RM_PARAMS = dict(G=1.5, vth=13.0, vp=100.0, eta1=4.4, eta2=0.012, eta3=1.0)


class Hierarchy:
    """a1..a9: the oracle's AMG hierarchy (Algorithm 1)."""

    def __init__(self, A, **opts):
        o = dict(DEFAULT_OPTS)
        o.update(opts)
        self.opts = o
        a = _In(A)
        h = _vp()
        co = _Opts(o["theta"], o["coarse_eq_limit"], o["max_levels"], o["cheb_degree"],
                   o["esteig_steps"], o["eig_lo"], o["eig_hi"], o["seed"] & (2**64 - 1),
                   o["square_levels"])
        _check(lib().oc_setup(C.byref(a.s), C.byref(co), C.byref(h)), "setup")
        self._h = h
        self.n = A.shape[0]

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oc_hier_free(self._h)
            self._h = None

    @property
    def nlevels(self) -> int:
        return lib().oc_hier_nlevels(self._h)

    def A(self, l):
        return _view(lib().oc_hier_A(self._h, l).contents)

    def P(self, l):
        p = lib().oc_hier_P(self._h, l)
        return _view(p.contents) if p else None

    def Pt(self, l):
        p = lib().oc_hier_Pt(self._h, l)
        return _view(p.contents) if p else None

    def nagg(self, l) -> int:
        return lib().oc_hier_nagg(self._h, l)

    def agg(self, l):
        p = lib().oc_hier_agg(self._h, l)
        if not p:
            return None
        return np.ctypeslib.as_array(p, shape=(self.A(l).shape[0] // 2,)).copy()

    def mis(self, l):
        p = lib().oc_hier_mis(self._h, l)
        if not p:
            return None
        return np.ctypeslib.as_array(p, shape=(self.A(l).shape[0] // 2,)).copy()

    def lam(self, l) -> float:
        return lib().oc_hier_lambda(self._h, l)

    def null(self, l):
        p = lib().oc_hier_null(self._h, l)
        return np.ctypeslib.as_array(p, shape=(self.A(l).shape[0],)).copy()

    def coarse_solve(self, r):
        r = _f64(r)
        x = np.zeros_like(r)
        _check(lib().oc_coarse_solve(self._h, _ptr(r), _ptr(x)), "coarse_solve")
        return x

    def vcycle(self, r):
        r = _f64(r)
        z = np.zeros_like(r)
        _check(lib().oc_vcycle(self._h, _ptr(r), _ptr(z)), "vcycle")
        return z

    def pcg(self, f, x0=None, rtol=1e-8, max_it=500):
        f = _f64(f)
        x = np.zeros_like(f) if x0 is None else _f64(x0).copy()
        it, rr, tr = C.c_int(0), C.c_double(0), C.c_double(0)
        rc = lib().oc_pcg(self._h, _ptr(f), _ptr(x), int(x0 is not None), rtol, max_it,
                          C.byref(it), C.byref(rr), C.byref(tr))
        return x, dict(status=rc, iters=it.value, rel_res=rr.value, true_rel_res=tr.value)

    def bd_step(self, M, params: dict, Iapp, v, ue, w, rtol=1e-8, max_it=500, rm=None):
        rm = dict(RM_PARAMS if rm is None else rm)
        M = _f64(M)
        Iapp = _f64(Iapp)
        it = C.c_int(0)
        crm = _RM(rm["G"], rm["vth"], rm["vp"], rm["eta1"], rm["eta2"], rm["eta3"])
        rc = lib().oc_bd_step(self._h, _ptr(M), M.size, params["chi"], params["cm"], params["dt"],
                              C.byref(crm), _ptr(Iapp), _ptr(v), _ptr(ue), _ptr(w), rtol, max_it,
                              C.byref(it))
        return dict(status=rc, iters=it.value)

    def bd_step_decoupled(self, Ki, M, params: dict, Iapp, v, ue, w, rtol=1e-8, max_it=500,
                          jacobi=True, rm=None):
        """f4: one step of the paper's decoupled scheme; self is the hierarchy
        of elliptic_block(Ki, Ke).  v, ue, w updated in place."""
        rm = dict(RM_PARAMS if rm is None else rm)
        k = _In(Ki)
        M = _f64(M)
        Iapp = _f64(Iapp)
        ie, ip = C.c_int(0), C.c_int(0)
        crm = _RM(rm["G"], rm["vth"], rm["vp"], rm["eta1"], rm["eta2"], rm["eta3"])
        rc = lib().oc_bd_step_decoupled(self._h, C.byref(k.s), _ptr(M), M.size, params["chi"],
                                        params["cm"], params["dt"], C.byref(crm), _ptr(Iapp),
                                        _ptr(v), _ptr(ue), _ptr(w), rtol, max_it, int(bool(jacobi)),
                                        C.byref(ie), C.byref(ip))
        return dict(status=rc, iters_elliptic=ie.value, iters_parabolic=ip.value)
