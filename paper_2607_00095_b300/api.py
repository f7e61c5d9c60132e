"""Python binding of libsnap: the C-ABI calls with torch tensors as device memory.

Every step of the projection runs in the CUDA kernels behind include/snap.h; this module only
allocates buffers (torch), passes pointers and decodes the per-sample statistics.  There is
no CPU path: calls on CPU tensors raise.
"""
import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import check, lib

STATS_DTYPE = np.dtype([("iters", "<i4"), ("backtracks", "<i4"), ("status", "<i4"),
                        ("corrections", "<i4"), ("h_inf", "<f8"), ("kkt_inf", "<f8"),
                        ("obj", "<f8")])
FAMILIES = {"A": _abi.FAMILY_A, "B": _abi.FAMILY_B, "C": _abi.FAMILY_C, "toy": _abi.FAMILY_TOY}
PATHS = {"auto": _abi.PATH_AUTO, "general": _abi.PATH_GENERAL, "moment": _abi.PATH_MOMENT,
         "mixed": _abi.PATH_MIXED}


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def options(**kw):
    o = _abi.Options()
    check(lib().snap_options_default(C.byref(o)))
    for k, v in kw.items():
        if k == "path" and isinstance(v, str):
            v = PATHS[v]
        setattr(o, k, v)
    return o


def decode_stats(st):
    """uint8 [B, 40] tensor of snap_stats -> numpy structured array."""
    raw = st.detach().cpu().numpy() if isinstance(st, torch.Tensor) else np.asarray(st)
    return np.frombuffer(raw.tobytes(), dtype=STATS_DTYPE)


class Problem:
    """One constraint family on one grid (snap_problem_create)."""

    def __init__(self, family, nx, nt, ny=None, rows=0, energy_floor=0.05, max_batch=0):
        L = lib()
        fam = FAMILIES[family] if isinstance(family, str) else int(family)
        d = _abi.ProblemDesc(fam, nx, ny if ny is not None else (nx if fam == _abi.FAMILY_C else 0),
                             nt, rows, energy_floor, max_batch)
        h = C.c_void_p()
        check(L.snap_problem_create(C.byref(d), C.byref(h)))
        self._h = h
        self.family = family
        self.nx, self.nt = nx, nt
        info = _abi.Info()
        check(L.snap_problem_info(h, C.byref(info)))
        self.n_vars = info.n_vars
        self.n_rows = info.n_rows_nominal
        self.n_rows_active = info.n_rows_active
        self.n_params = info.n_params
        self.pattern_nnz = info.pattern_nnz
        self.n_blocks = info.n_blocks
        self._ws = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _abi._lib is not None:
            _abi._lib.snap_problem_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    # ---- sizes and host-side structure -------------------------------------------------
    def workspace_bytes(self, B):
        n = C.c_size_t()
        check(lib().snap_workspace_size(self._h, B, C.byref(n)))
        return n.value

    def cache_bytes(self, B):
        n = C.c_size_t()
        check(lib().snap_adjoint_cache_size(self._h, B, C.byref(n)))
        return n.value

    def workspace(self, B, device):
        key = (B, str(device))
        ws = self._ws.get(key)
        if ws is None:
            ws = torch.empty(max(self.workspace_bytes(B), 256), dtype=torch.uint8, device=device)
            self._ws = {key: ws}
        return ws

    def pattern(self):
        rp = np.zeros(self.n_rows + 1, np.int32)
        ci = np.zeros(max(self.pattern_nnz, 1), np.int32)
        check(lib().snap_problem_pattern(self._h, rp.ctypes.data_as(C.POINTER(C.c_int)),
                                         ci.ctypes.data_as(C.POINTER(C.c_int))))
        return rp, ci[:self.pattern_nnz]

    def active_rows(self):
        a = np.zeros(self.n_rows, np.uint8)
        check(lib().snap_problem_active_rows(self._h, a.ctypes.data_as(C.POINTER(C.c_uint8))))
        return a

    # ---- compute -----------------------------------------------------------------------
    def _check_dev(self, *ts):
        for t in ts:
            if t is not None:
                if not t.is_cuda:
                    raise ValueError("snap needs CUDA tensors (no CPU path)")
                if t.dtype != torch.float64 or not t.is_contiguous():
                    raise ValueError("snap needs contiguous float64 tensors")

    def project(self, u_hat, params, u0=None, opts=None, cache=False, out=None, stream=None,
                workspace=None):
        """Returns (u [B, n_vars], lambda [B, n_rows], stats uint8 [B, 40], cache or None)."""
        B = u_hat.shape[0]
        u_hat = u_hat.reshape(B, self.n_vars)
        self._check_dev(u_hat, params, u0)
        dev = u_hat.device
        if out is None:
            u = torch.empty_like(u_hat)
            lam = torch.empty(B, self.n_rows, dtype=torch.float64, device=dev)
            st = torch.empty(B, 40, dtype=torch.uint8, device=dev)
        else:
            u, lam, st = out
        cb = None
        if cache:
            cb = torch.empty(max(self.cache_bytes(B), 8), dtype=torch.uint8, device=dev)
        ws = workspace if workspace is not None else self.workspace(B, dev)
        o = opts if opts is not None else options()
        check(lib().snap_project(self._h, B, _ptr(u_hat), _ptr(params),
                                 _ptr(u0.reshape(B, self.n_vars)) if u0 is not None else None,
                                 _ptr(u), _ptr(lam), _ptr(st), _ptr(cb), C.byref(o), _ptr(ws),
                                 ws.numel(), _stream(stream)))
        return u, lam, st, cb

    def project_noalloc(self, u_hat, params, u, lam, st, opts=None, stream=None):
        """snap_project_noalloc: the 1-D forward projection into caller-given outputs, with the
        scratch in the library's static device array (no workspace, nothing allocated by the
        call).  Calls that overlap on the GPU race on that array."""
        B = u_hat.shape[0]
        self._check_dev(u_hat, params, u, lam)
        if not st.is_cuda or st.dtype != torch.uint8 or st.numel() != 40 * B:
            raise ValueError("stats must be a CUDA uint8 tensor of 40 bytes per sample")
        o = opts if opts is not None else options()
        check(lib().snap_project_noalloc(self._h, B, _ptr(u_hat), _ptr(params), _ptr(u),
                                         _ptr(lam), _ptr(st), C.byref(o), _stream(stream)))
        return u, lam, st

    def backward(self, grad_u, u, lam, params, stats=None, cache=None, stream=None,
                 with_params=True):
        B = u.shape[0]
        grad_u = grad_u.reshape(B, self.n_vars).contiguous()
        self._check_dev(grad_u, u, lam, params)
        gh = torch.empty_like(u)
        gp = torch.empty(B, self.n_params, dtype=torch.float64, device=u.device) if with_params else None
        ws = self.workspace(B, u.device)
        check(lib().snap_project_backward(self._h, B, _ptr(grad_u), _ptr(u), _ptr(lam),
                                          _ptr(params), _ptr(stats), _ptr(cache), _ptr(gh),
                                          _ptr(gp), _ptr(ws), ws.numel(), _stream(stream)))
        return gh, gp

    def residual(self, u, params, want_rows=True, stream=None):
        B = u.shape[0]
        u = u.reshape(B, self.n_vars)
        self._check_dev(u, params)
        h = torch.empty(B, self.n_rows, dtype=torch.float64, device=u.device) if want_rows else None
        hinf = torch.empty(B, dtype=torch.float64, device=u.device)
        ws = self.workspace(B, u.device)
        check(lib().snap_constraint_residual(self._h, B, _ptr(u), _ptr(params), _ptr(h),
                                             _ptr(hinf), _ptr(ws), ws.numel(), _stream(stream)))
        return h, hinf


class SnapProject(torch.autograd.Function):
    """u = projection(u_hat; params) with the implicit-function adjoint as backward.

    store_factor: True keeps the per-block factors from the forward pass for the backward,
    False recomputes them from (u, lambda), "auto" stores them when they take less than a
    quarter of the free device memory.
    """

    @staticmethod
    def forward(ctx, u_hat, params, problem, store_factor="auto", opts=None):
        B = u_hat.shape[0]
        store = store_factor
        if store == "auto":
            free, _ = torch.cuda.mem_get_info(u_hat.device)
            store = problem.cache_bytes(B) < 0.25 * free
        u, lam, st, cb = problem.project(u_hat.detach().contiguous(), params.detach().contiguous(),
                                         opts=opts, cache=bool(store))
        ctx.problem = problem
        ctx.save_for_backward(u, lam, params.detach(), st, cb if cb is not None else torch.empty(0))
        ctx.has_cache = cb is not None
        ctx.shape = u_hat.shape
        return u.reshape(u_hat.shape)

    @staticmethod
    def backward(ctx, grad_u):
        u, lam, params, st, cb = ctx.saved_tensors
        gh, gp = ctx.problem.backward(grad_u.contiguous(), u, lam, params.contiguous(), stats=st,
                                      cache=cb if ctx.has_cache else None)
        return gh.reshape(ctx.shape), gp, None, None, None


def project(problem, u_hat, params, **kw):
    """Forward projection; returns (u, lambda, stats as numpy structured array)."""
    u, lam, st, _ = problem.project(u_hat, params, **kw)
    return u, lam, decode_stats(st)


def measure_fp64_rate(device=0):
    r = C.c_double()
    check(lib().snap_measure_fp64_rate(device, C.byref(r)))
    return r.value


def profile_enable(on=True):
    check(lib().snap_profile_enable(1 if on else 0))


def profile_reset():
    check(lib().snap_profile_reset())


def profile_read(name):
    """(total_ms, launches) of the event-timed launches of kernel `name`."""
    t = C.c_double()
    n = C.c_longlong()
    check(lib().snap_profile_read(name.encode(), C.byref(t), C.byref(n)))
    return t.value, n.value


def last_launch_count():
    return int(lib().snap_last_launch_count())
