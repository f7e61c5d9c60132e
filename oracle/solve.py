"""ctypes wrapper of the oracle's C core -- TEST INFRASTRUCTURE ONLY.

project()  : dense Newton-KKT projection (Appendix B) of a batch, per connected component.
adjoint()  : dense implicit-function adjoint K [a; b] = [gbar; 0] at the solution.
"""
import ctypes as C

import numpy as np

from . import build as _build
from . import problems

ORA_OK, ORA_MAXITER, ORA_LINESEARCH, ORA_NONFINITE, ORA_SINGULAR, ORA_NOT_MINIMUM = 0, 1, 2, 3, 6, 7


class OraOpts(C.Structure):
    _fields_ = [("tol_kkt", C.c_double), ("max_iter", C.c_int), ("max_backtracks", C.c_int),
                ("c1", C.c_double), ("delta0", C.c_double), ("max_corrections", C.c_int),
                ("split_components", C.c_int), ("w_keep", C.c_double), ("restore", C.c_int)]


class OraStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("backtracks", C.c_int), ("status", C.c_int),
                ("corrections", C.c_int), ("kkt_inf", C.c_double), ("phi", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        u8p = C.POINTER(C.c_uint8)
        _lib.ora_project_batch.argtypes = [C.c_int, C.c_int, ip, ip, dp, ip, ip, dp, u8p, C.c_int,
                                           dp, dp, dp, C.POINTER(OraOpts), C.c_int, dp, dp,
                                           C.POINTER(OraStats)]
        _lib.ora_adjoint_batch.argtypes = [C.c_int, C.c_int, ip, ip, dp, ip, ip, dp, u8p, C.c_int,
                                           dp, dp, dp, C.c_int, C.c_int, dp, dp]
        _lib.ora_components.argtypes = [C.c_int, C.c_int, ip, ip, ip, ip, u8p, C.c_int, ip, ip]
        _lib.ora_ldl_solve_dense.argtypes = [C.c_int, dp, dp, dp, ip]
        _lib.ora_max_threads.restype = C.c_int
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def default_opts(**kw):
    o = dict(tol_kkt=1e-10, max_iter=50, max_backtracks=30, c1=1e-4, delta0=1e-8,
             max_corrections=0, split_components=1, w_keep=0.01, restore=1)
    o.update(kw)
    return OraOpts(**o)


def project(S, b, u_hat, u0=None, nthreads=0, **opts):
    """Solve the projection of every sample.  Returns (u [B,n], lam [B,m], stats dict)."""
    L = lib()
    b = np.ascontiguousarray(np.atleast_2d(b), np.float64)
    u_hat = np.ascontiguousarray(np.atleast_2d(u_hat).reshape(b.shape[0], -1), np.float64)
    B = u_hat.shape[0]
    assert u_hat.shape[1] == S.n and b.shape == (B, S.m)
    u = np.zeros((B, S.n))
    lam = np.zeros((B, S.m))
    st = (OraStats * B)()
    u0p = None
    if u0 is not None:
        u0 = np.ascontiguousarray(np.atleast_2d(u0).reshape(B, -1), np.float64)
        u0p = _p(u0, C.c_double)
    # u kept stationary for the projection's own start u0 = u_hat; an explicit start point u0
    # takes the primal-dual iteration
    opts.setdefault("restore", 0 if u0 is not None else 1)
    o = default_opts(**opts)
    L.ora_project_batch(S.n, S.m, _p(S.a_ptr, C.c_int), _p(S.a_col, C.c_int),
                        _p(S.a_val, C.c_double), _p(S.q_ptr, C.c_int), _p(S.q_col, C.c_int),
                        _p(S.q_val, C.c_double), _p(S.active, C.c_uint8), B,
                        _p(b, C.c_double), _p(u_hat, C.c_double), u0p, C.byref(o), nthreads,
                        _p(u, C.c_double), _p(lam, C.c_double), st)
    stats = dict(iters=np.array([s.iters for s in st]), backtracks=np.array([s.backtracks for s in st]),
                 status=np.array([s.status for s in st]), corrections=np.array([s.corrections for s in st]),
                 kkt_inf=np.array([s.kkt_inf for s in st]), phi=np.array([s.phi for s in st]))
    return u, lam, stats


def adjoint(S, u, lam, gbar, split=1, nthreads=0):
    """K [a; b] = [gbar; 0] per component at (u, lam).  Returns (a [B,n], b [B,m])."""
    L = lib()
    u = np.ascontiguousarray(np.atleast_2d(u), np.float64)
    B = u.shape[0]
    lam = np.ascontiguousarray(np.atleast_2d(lam), np.float64)
    gbar = np.ascontiguousarray(np.atleast_2d(gbar).reshape(B, -1), np.float64)
    a = np.zeros((B, S.n))
    bl = np.zeros((B, S.m))
    rc = L.ora_adjoint_batch(S.n, S.m, _p(S.a_ptr, C.c_int), _p(S.a_col, C.c_int),
                             _p(S.a_val, C.c_double), _p(S.q_ptr, C.c_int), _p(S.q_col, C.c_int),
                             _p(S.q_val, C.c_double), _p(S.active, C.c_uint8), B,
                             _p(u, C.c_double), _p(lam, C.c_double), _p(gbar, C.c_double),
                             split, nthreads, _p(a, C.c_double), _p(bl, C.c_double))
    if rc != 0:
        raise RuntimeError("oracle adjoint: singular KKT matrix")
    return a, bl


def components(S, split=1):
    L = lib()
    cv = np.zeros(S.n, np.int32)
    cr = np.zeros(S.m, np.int32)
    nc = L.ora_components(S.n, S.m, _p(S.a_ptr, C.c_int), _p(S.a_col, C.c_int),
                          _p(S.q_ptr, C.c_int), _p(S.q_col, C.c_int), _p(S.active, C.c_uint8),
                          split, _p(cv, C.c_int), _p(cr, C.c_int))
    return nc, cv, cr


def ldl_solve_dense(A, rhs):
    """Bunch-Kaufman LDL^T solve of one dense symmetric system; returns (x, inertia)."""
    L = lib()
    A = np.ascontiguousarray(A, np.float64)
    rhs = np.ascontiguousarray(rhs, np.float64)
    x = np.zeros_like(rhs)
    inert = np.zeros(3, np.int32)
    rc = L.ora_ldl_solve_dense(A.shape[0], _p(A, C.c_double), _p(rhs, C.c_double),
                               _p(x, C.c_double), _p(inert, C.c_int))
    return x, tuple(int(v) for v in inert), rc


def max_threads():
    return int(lib().ora_max_threads())


# ----------------------------------------------------------------------------------------
# Family-level conveniences
# ----------------------------------------------------------------------------------------

def project_1d(family, nx, nt, params, u_hat, u0=None, energy_floor=0.05, nthreads=0, **opts):
    S = problems.structure_1d(family, nx, nt)
    b = problems.rhs_1d(family, nx, nt, params, energy_floor)
    u, lam, st = project(S, b, np.asarray(u_hat).reshape(b.shape[0], -1), u0, nthreads, **opts)
    h = problems.eval_h(S, u, b)
    st["h_inf"] = np.abs(h).max(axis=1)
    return u, lam, st, S, b


def adjoint_1d(family, nx, nt, params, u, lam, gbar, energy_floor=0.05, nthreads=0):
    S = problems.structure_1d(family, nx, nt)
    a, bl = adjoint(S, u, lam, gbar, nthreads=nthreads)
    gp = problems.grad_params_1d(family, nx, nt, params, bl, energy_floor)
    return a, gp, bl
