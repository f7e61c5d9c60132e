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
FAMILIES = {"A": _abi.FAMILY_A, "B": _abi.FAMILY_B, "C": _abi.FAMILY_C, "toy": _abi.FAMILY_TOY,
            "D": _abi.FAMILY_D, "E": _abi.FAMILY_E, "F": _abi.FAMILY_F}
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

    def __init__(self, family, nx, nt, ny=None, rows=0, energy_floor=0.05, max_batch=0, n_flux=0):
        L = lib()
        fam = FAMILIES[family] if isinstance(family, str) else int(family)
        d = _abi.ProblemDesc(fam, nx, ny if ny is not None else (nx if fam == _abi.FAMILY_C else 0),
                             nt, rows, energy_floor, max_batch, n_flux)
        h = C.c_void_p()
        check(L.snap_problem_create(C.byref(d), C.byref(h)))
        self._h = h
        self.family = family
        self.nx, self.nt = nx, nt
        self.n_flux = n_flux
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

    def _check_sizes(self, B, u_hat=None, params=None, u=None, lam=None, st=None):
        """Every buffer the library reads or writes must hold exactly the problem's sizes
        for B samples: a short buffer would be written past its end on the device."""
        want = (("u_hat", u_hat, B * self.n_vars), ("params", params, B * self.n_params),
                ("u", u, B * self.n_vars), ("lambda", lam, B * self.n_rows),
                ("stats", st, 40 * B))
        for name, t, n in want:
            if t is not None and t.numel() != n:
                raise ValueError(f"{name} holds {t.numel()} elements; this problem needs {n} "
                                 f"for B = {B}")

    def project(self, u_hat, params, u0=None, opts=None, out=None, stream=None, workspace=None):
        """Returns (u [B, n_vars], lambda [B, n_rows], stats uint8 [B, 40])."""
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
            self._check_dev(u, lam)
        self._check_sizes(B, u_hat, params, u, lam, st)
        ws = workspace if workspace is not None else self.workspace(B, dev)
        o = opts if opts is not None else options()
        check(lib().snap_project(self._h, B, _ptr(u_hat), _ptr(params),
                                 _ptr(u0.reshape(B, self.n_vars)) if u0 is not None else None,
                                 _ptr(u), _ptr(lam), _ptr(st), C.byref(o), _ptr(ws),
                                 ws.numel(), _stream(stream)))
        return u, lam, st

    def project_noalloc(self, u_hat, params, u, lam, st, opts=None, stream=None):
        """snap_project_noalloc: the 1-D forward projection into caller-given outputs, with the
        scratch in the library's static device array (no workspace, nothing allocated by the
        call).  Calls that overlap on the GPU race on that array."""
        B = u_hat.shape[0]
        self._check_dev(u_hat, params, u, lam)
        if not st.is_cuda or st.dtype != torch.uint8 or not st.is_contiguous():
            raise ValueError("stats must be a contiguous CUDA uint8 tensor of 40 bytes per sample")
        self._check_sizes(B, u_hat, params, u, lam, st)
        if u.data_ptr() == u_hat.data_ptr() or lam.data_ptr() in (u.data_ptr(), u_hat.data_ptr()):
            raise ValueError("outputs may not alias inputs")
        o = opts if opts is not None else options()
        check(lib().snap_project_noalloc(self._h, B, _ptr(u_hat), _ptr(params), _ptr(u),
                                         _ptr(lam), _ptr(st), C.byref(o), _stream(stream)))
        return u, lam, st

    def pcfm_sample(self, u0, x1, xi, params, n_steps, sigma0=0.0, opts=None, out=None,
                    stream=None):
        """snap_pcfm_sample: one sampling pass of n_steps shoot / project / pull-back steps
        with the analytic velocity (x1 - u0) + sigma0 (1 - tau) xi.  Returns (u, lambda,
        stats) of the last projection."""
        B = u0.shape[0]
        self._check_dev(u0, x1, xi, params)
        dev = u0.device
        if out is None:
            u = torch.empty_like(u0)
            lam = torch.empty(B, self.n_rows, dtype=torch.float64, device=dev)
            st = torch.empty(B, 40, dtype=torch.uint8, device=dev)
        else:
            u, lam, st = out
        key = ("pcfm", B, str(dev))
        ws = self._ws.get(key)
        if ws is None:
            n = C.c_size_t()
            check(lib().snap_pcfm_workspace_size(self._h, B, C.byref(n)))
            ws = torch.empty(max(n.value, 8), dtype=torch.uint8, device=dev)
            self._ws[key] = ws
        o = opts if opts is not None else options()
        check(lib().snap_pcfm_sample(self._h, B, int(n_steps), float(sigma0), _ptr(u0), _ptr(x1),
                                     _ptr(xi), _ptr(params), _ptr(u), _ptr(lam), _ptr(st),
                                     C.byref(o), _ptr(ws), ws.numel(), _stream(stream)))
        return u, lam, st

    def backward(self, grad_u, u, lam, params, stats=None, stream=None, with_params=True):
        B = u.shape[0]
        grad_u = grad_u.reshape(B, self.n_vars).contiguous()
        self._check_dev(grad_u, u, lam, params)
        gh = torch.empty_like(u)
        gp = torch.empty(B, self.n_params, dtype=torch.float64, device=u.device) if with_params else None
        ws = self.workspace(B, u.device)
        check(lib().snap_project_backward(self._h, B, _ptr(grad_u), _ptr(u), _ptr(lam),
                                          _ptr(params), _ptr(stats), _ptr(gh),
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


# energy_floor that switches the floor of the energy targets off: E_k = E0 exp(-r t_k)
NO_ENERGY_FLOOR = -1e300


def vorticity_problem(N, nt, max_batch=0):
    """The 2-D vorticity constraints of the Navier-Stokes problem (Appendix A): per frame of the
    N x N periodic grid on [0, 1]^2, the IC frame w(., 0) = w_IC, total vorticity
    int w = int w_IC and enstrophy int w^2 = int w_IC^2.  With a frame flattened to N^2 values
    and dx dy = 1 / N^2 these are exactly the rows of family A with nx = N^2, rate 0 and no
    energy floor; params = [w_IC (N^2 values), 0.0]."""
    return Problem("A", N * N, nt, energy_floor=NO_ENERGY_FLOOR, max_batch=max_batch)


class SnapProject(torch.autograd.Function):
    """u = projection(u_hat; params) with the implicit-function adjoint as backward (the
    per-block factors are rebuilt from (u, lambda) in the backward pass)."""

    @staticmethod
    def forward(ctx, u_hat, params, problem, opts=None):
        u, lam, st = problem.project(u_hat.detach().contiguous(), params.detach().contiguous(),
                                     opts=opts)
        ctx.problem = problem
        ctx.save_for_backward(u, lam, params.detach(), st)
        ctx.shape = u_hat.shape
        return u.reshape(u_hat.shape)

    @staticmethod
    def backward(ctx, grad_u):
        u, lam, params, st = ctx.saved_tensors
        gh, gp = ctx.problem.backward(grad_u.contiguous(), u, lam, params.contiguous(), stats=st)
        return gh.reshape(ctx.shape), gp, None, None


def _schedule_dict(s):
    return dict(ctas_per_sm=s.ctas_per_sm, order=s.order, pack_1d=s.pack_1d, sort_1d=s.sort_1d,
                tile_1d=s.tile_1d, lanes_1d=s.lanes_1d)


class Batch:
    """Uneven batch (snap_batch_*): instances of several problems (1-D families A/B, 2-D
    family C) projected in one persistent kernel launch.  Instance i is one sample of
    problems[inst_problem[i]]."""

    def __init__(self, problems, inst_problem):
        self.problems = list(problems)
        self.inst_problem = np.ascontiguousarray(inst_problem, dtype=np.int32)
        n = int(self.inst_problem.size)
        arr = (C.c_void_p * len(self.problems))(*[p._h.value for p in self.problems])
        h = C.c_void_p()
        check(lib().snap_batch_create(len(self.problems), arr, n,
                                      self.inst_problem.ctypes.data_as(C.POINTER(C.c_int)),
                                      C.byref(h)))
        self._h = h
        self.n_inst = n
        self._keep = None
        self._ws = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _abi._lib is not None:
            _abi._lib.snap_batch_destroy(h)
            self._h = None

    def groups(self):
        """{problem index: instance ids of that problem, in instance order}."""
        return {int(pi): np.nonzero(self.inst_problem == pi)[0]
                for pi in np.unique(self.inst_problem)}

    def alloc(self, device):
        """Allocate contiguous per-group buffers (u_hat, params, u, lambda, stats), bind them and
        return {problem index: dict(ids, uh, pr, u, lam, st)} (row j = instance ids[j])."""
        out = {}
        per = [None] * self.n_inst
        for pi, ids in self.groups().items():
            p = self.problems[pi]
            n = len(ids)
            g = dict(ids=ids,
                     uh=torch.zeros(n, p.n_vars, dtype=torch.float64, device=device),
                     pr=torch.zeros(n, p.n_params, dtype=torch.float64, device=device),
                     u=torch.empty(n, p.n_vars, dtype=torch.float64, device=device),
                     lam=torch.empty(n, p.n_rows, dtype=torch.float64, device=device),
                     st=torch.empty(n, 40, dtype=torch.uint8, device=device))
            out[pi] = g
            for j, i in enumerate(ids):
                per[i] = (g["uh"][j], g["pr"][j], g["u"][j], g["lam"][j], g["st"][j])
        self.bind(*[[x[k] for x in per] for k in range(5)])
        return out

    def bind(self, u_hat, params, u, lam, stats):
        """Bind per-instance device tensors (lists of length n_inst)."""
        n = self.n_inst

        def tab(ts):
            return (C.c_void_p * max(n, 1))(*[t.data_ptr() for t in ts])

        tabs = [tab(t) for t in (u_hat, params, u, lam, stats)]
        check(lib().snap_batch_bind(self._h, *tabs))
        self._keep = (u_hat, params, u, lam, stats)

    def workspace_bytes(self):
        n = C.c_size_t()
        check(lib().snap_batch_workspace_size(self._h, C.byref(n)))
        return n.value

    def workspace(self, device):
        need = max(self.workspace_bytes(), 8)
        if self._ws is None or self._ws.numel() < need or self._ws.device != torch.device(device):
            self._ws = torch.empty(need, dtype=torch.uint8, device=device)
        return self._ws

    def _dev(self):
        return self._keep[0][0].device if self._keep and self.n_inst else torch.device("cuda:0")

    def project(self, opts=None, t_ns=None, stream=None):
        ws = self.workspace(self._dev())
        o = opts if opts is not None else options()
        check(lib().snap_batch_project(self._h, C.byref(o), _ptr(t_ns), _ptr(ws), ws.numel(),
                                       _stream(stream)))

    def project_grouped(self, opts=None, stream=None):
        ws = self.workspace(self._dev())
        o = opts if opts is not None else options()
        check(lib().snap_batch_project_grouped(self._h, C.byref(o), _ptr(ws), ws.numel(),
                                               _stream(stream)))

    def schedule(self):
        s = _abi.Schedule()
        check(lib().snap_batch_get_schedule(self._h, C.byref(s)))
        return _schedule_dict(s)

    def set_schedule(self, **kw):
        d = self.schedule()
        d.update(kw)
        s = _abi.Schedule(d["ctas_per_sm"], d["order"], d["pack_1d"], d["sort_1d"], d["tile_1d"],
                          d.get("lanes_1d", 0))
        check(lib().snap_batch_set_schedule(self._h, C.byref(s)))

    def group_lanes(self):
        """Lanes per slice of every group (problem order; 0 for 2-D groups)."""
        n = self.info()["groups"]
        a = np.zeros(max(n, 1), np.int32)
        check(lib().snap_batch_get_group_lanes(self._h, a.ctypes.data_as(C.POINTER(C.c_int))))
        return a[:n].tolist()

    def set_group_lanes(self, lanes):
        a = np.ascontiguousarray(lanes, dtype=np.int32)
        check(lib().snap_batch_set_group_lanes(self._h, a.ctypes.data_as(C.POINTER(C.c_int))))

    def autotune(self, opts=None, reps=3, stream=None):
        """Time every schedule, keep the fastest; returns (schedule dict, ms)."""
        ws = self.workspace(self._dev())
        o = opts if opts is not None else options()
        s = _abi.Schedule()
        ms = C.c_double()
        check(lib().snap_batch_autotune(self._h, C.byref(o), _ptr(ws), ws.numel(),
                                        _stream(stream), reps, C.byref(s), C.byref(ms)))
        return _schedule_dict(s), ms.value

    def capture_graph(self, opts=None, t_ns=None):
        ws = self.workspace(self._dev())
        o = opts if opts is not None else options()
        check(lib().snap_batch_capture_graph(self._h, C.byref(o), _ptr(t_ns), _ptr(ws),
                                             ws.numel()))

    def launch_graph(self, stream=None):
        check(lib().snap_batch_launch_graph(self._h, _stream(stream)))

    def alloc_backward(self, device, with_params=True):
        """Allocate contiguous per-group adjoint buffers (dL/du input, dL/du_hat and dL/dparams
        outputs), bind them and return {problem index: dict(ids, gu, gh, gp)} (row j = instance
        ids[j]); gp is None without parameter gradients."""
        out = {}
        per = [None] * self.n_inst
        for pi, ids in self.groups().items():
            p = self.problems[pi]
            n = len(ids)
            g = dict(ids=ids,
                     gu=torch.zeros(n, p.n_vars, dtype=torch.float64, device=device),
                     gh=torch.empty(n, p.n_vars, dtype=torch.float64, device=device),
                     gp=(torch.empty(n, p.n_params, dtype=torch.float64, device=device)
                         if with_params else None))
            out[pi] = g
            for j, i in enumerate(ids):
                per[i] = (g["gu"][j], g["gh"][j], g["gp"][j] if with_params else None)
        self.bind_backward(*[[x[k] for x in per] for k in range(3)])
        return out

    def bind_backward(self, grad_u, grad_u_hat, grad_params=None):
        """Bind per-instance adjoint tensors (lists of length n_inst; grad_params may be None,
        or hold None entries: no parameter gradient for those instances)."""
        n = self.n_inst

        def tab(ts):
            return (C.c_void_p * max(n, 1))(*[(t.data_ptr() if t is not None else None)
                                               for t in ts])

        gp = tab(grad_params) if grad_params is not None else None
        check(lib().snap_batch_bind_backward(self._h, tab(grad_u), tab(grad_u_hat), gp))
        self._keep_bwd = (grad_u, grad_u_hat, grad_params)

    def backward(self, stream=None):
        """The adjoint of every instance in one persistent launch (after project)."""
        ws = self.workspace(self._dev())
        check(lib().snap_batch_project_backward(self._h, _ptr(ws), ws.numel(), _stream(stream)))

    def backward_grouped(self, stream=None):
        ws = self.workspace(self._dev())
        check(lib().snap_batch_project_backward_grouped(self._h, _ptr(ws), ws.numel(),
                                                        _stream(stream)))

    def capture_graph_backward(self):
        ws = self.workspace(self._dev())
        check(lib().snap_batch_capture_graph_backward(self._h, _ptr(ws), ws.numel()))

    def launch_graph_backward(self, stream=None):
        check(lib().snap_batch_launch_graph_backward(self._h, _stream(stream)))

    def info(self):
        g, t, f = C.c_int(), C.c_int(), C.c_int()
        check(lib().snap_batch_info(self._h, C.byref(g), C.byref(t), C.byref(f)))
        return dict(groups=g.value, tiles_1d=t.value, frames_2d=f.value)


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
