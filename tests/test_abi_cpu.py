"""C-ABI checks that need no GPU: the library loads, exports every declared entry point,
and its host-side problem construction (row list, Jacobian pattern, implied rows) matches
the oracle's row builders and the printed Appendix C Jacobian bit for bit."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import problems
from paper_2607_00095_b300 import Problem, _abi, options
from paper_2607_00095_b300.api import STATS_DTYPE

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"SNAP_API[^;(]*?\b(snap_\w+)\s*\(", txt, flags=re.S))
    return names


def test_library_loads_and_exports_every_declared_symbol():
    L = _abi.lib()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    # the binding declares prototypes for exactly the header's entry points
    assert set(_abi.declared_symbols()) == declared
    assert b"sm_103a" in L.snap_version()


def _pattern_of(S):
    """CSR pattern of the oracle's rows (union of linear and quadratic parts)."""
    rp = [0]
    ci = []
    for r in range(S.m):
        cols = set(S.a_col[S.a_ptr[r]:S.a_ptr[r + 1]]) | set(S.q_col[S.q_ptr[r]:S.q_ptr[r + 1]])
        ci.extend(sorted(int(c) for c in cols))
        rp.append(len(ci))
    return np.array(rp), np.array(ci)


@pytest.mark.parametrize("family,nx,nt", [("A", 32, 32), ("B", 128, 100), ("B", 4, 2), ("A", 6, 3)])
def test_pattern_1d_matches_oracle(family, nx, nt):
    p = Problem(family, nx, nt)
    S = problems.structure_1d(family, nx, nt)
    rp, ci = p.pattern()
    orp, oci = _pattern_of(S)
    assert p.n_rows == S.m and p.n_vars == S.n
    assert p.n_params == problems.n_params_1d(family, nx, nt)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    np.testing.assert_array_equal(p.active_rows(), S.active)
    assert p.n_rows_active == int(S.active.sum())


@pytest.mark.parametrize("N,nt", [(4, 2), (8, 3), (64, 2), (6, 2), (12, 3)])
def test_pattern_2d_matches_oracle(N, nt):
    p = Problem("C", N, nt)
    S = problems.structure_2d(N, nt)
    rp, ci = p.pattern()
    orp, oci = _pattern_of(S)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    np.testing.assert_array_equal(p.active_rows(), S.active)


def test_toy_pattern_matches_printed_jacobian():
    ref = np.loadtxt(os.path.join(ROOT, "tests", "golden", "toy_jacobian_appC.txt"))
    p = Problem("toy", 3, 3)
    rp, ci = p.pattern()
    dense = np.zeros_like(ref)
    for r in range(len(rp) - 1):
        dense[r, ci[rp[r]:rp[r + 1]]] = 1
    np.testing.assert_array_equal(dense, (ref != 0).astype(float))


def test_row_mask_layout():
    p = Problem("A", 16, 5, rows=_abi.ROW_IC | _abi.ROW_MASS)
    assert p.n_rows == 16 + 5 and p.n_rows_active == 16 + 4
    with pytest.raises(_abi.SnapError):
        Problem("A", 16, 5, rows=_abi.ROW_IC | _abi.ROW_BOUNDARY)   # boundary needs family B
    with pytest.raises(_abi.SnapError):
        Problem("B", 16, 5, rows=_abi.ROW_MASS)                      # IC rows required


@pytest.mark.parametrize("kw", [dict(family="B", nx=5, nt=4), dict(family="B", nx=2, nt=4),
                                dict(family="A", nx=16, nt=1), dict(family="C", nx=8, nt=2, ny=6),
                                dict(family=9, nx=8, nt=4)])
def test_bad_descriptors_rejected(kw):
    with pytest.raises(_abi.SnapError) as ei:
        Problem(**kw)
    assert ei.value.code == 1


def test_null_and_size_errors_without_gpu():
    L = _abi.lib()
    assert L.snap_problem_create(None, None) == 1
    assert b"null" in L.snap_last_error()
    p = Problem("B", 16, 4, max_batch=8)
    n = C.c_size_t()
    assert L.snap_workspace_size(p.handle, 9, C.byref(n)) == 1       # above max_batch
    assert L.snap_workspace_size(p.handle, -1, C.byref(n)) == 1
    o = options()
    # B = 0 is a no-op even with null buffers
    assert L.snap_project(p.handle, 0, None, None, None, None, None, None, C.byref(o), None, 0, None) == 0
    # missing workspace is reported before any launch
    fake = C.c_void_p(1 << 20)
    rc = L.snap_project(p.handle, 2, fake, fake, None, C.c_void_p(2 << 20), C.c_void_p(3 << 20), None,
                        C.byref(o), None, 0, None)
    assert rc == 5
    bad = options(tol_kkt=-1.0)
    rc = L.snap_project(p.handle, 2, fake, fake, None, fake, fake, None, C.byref(bad), None, 0, None)
    assert rc == 1
    # the adjoint refuses outputs that alias its inputs, before any launch
    g1, g2 = C.c_void_p(4 << 20), C.c_void_p(5 << 20)
    for gu, uu, gh in ((g1, g2, g1), (g1, g2, g2)):
        rc = L.snap_project_backward(p.handle, 2, gu, uu, fake, fake, None, gh, None, None, 0, None)
        assert rc == 1 and b"alias" in L.snap_last_error()
    t = Problem("toy", 3, 3)
    rc = L.snap_project(t.handle, 1, fake, fake, None, fake, fake, None, C.byref(o), None, 0, None)
    assert rc == 2


def test_options_defaults_and_stats_layout():
    o = options()
    assert o.tol_kkt == 1e-10 and o.tol_h == 1e-8 and o.max_iter == 50 and o.max_backtracks == 30
    assert o.armijo_c1 == 1e-4 and o.max_corrections == 0 and o.w_keep == 0.01
    assert STATS_DTYPE.itemsize == C.sizeof(_abi.Stats) == 40


def test_workspace_sizes():
    p = Problem("B", 128, 100)
    assert p.workspace_bytes(512) > p.workspace_bytes(1) > 0


@pytest.mark.parametrize("nx,nt,K", [(5, 4, 1), (12, 7, 3), (9, 3, 2)])
def test_pattern_flux_matches_oracle(nx, nt, K):
    """Family E: the pattern covers every entry of the oracle's Jacobian at a generic point,
    with one row per nominal row, and the active mask leaves out mass rows 0..K."""
    from oracle import flux
    p = Problem("E", nx, nt, n_flux=K)
    n, m = flux.sizes(nx, nt, K)
    assert (p.n_vars, p.n_rows, p.n_params) == (n, m, nx)
    rp, ci = p.pattern()
    u = np.random.default_rng(5).uniform(-1, 1, size=n)
    J = flux.full_jacobian(nx, nt, K, u)
    P = np.zeros((m, n), bool)
    for r in range(m):
        P[r, ci[rp[r]:rp[r + 1]]] = True
    assert not (np.abs(J) > 0)[~P].any()
    np.testing.assert_array_equal(p.active_rows(), flux.active_rows(nx, nt, K))
    assert p.n_rows_active == int(flux.active_rows(nx, nt, K).sum())


@pytest.mark.parametrize("kw", [dict(nx=2, nt=4, n_flux=1), dict(nx=8, nt=4, n_flux=0),
                                dict(nx=8, nt=4, n_flux=4), dict(nx=600, nt=4, n_flux=1),
                                dict(nx=8, nt=4, n_flux=1, rows=1)])
def test_flux_bad_descriptors_rejected(kw):
    with pytest.raises(_abi.SnapError):
        Problem("E", **kw)
    with pytest.raises(_abi.SnapError):
        Problem("D", 8, 4, n_flux=1)


def test_noalloc_rejects_aliased_outputs_without_a_device():
    """snap_project_noalloc returns INVALID_ARG for in-place calls (u == u_hat, lambda == u)
    before it touches the device: the addresses below are never dereferenced."""
    L = _abi.lib()
    p = Problem("B", 128, 100)
    o = options()
    a, b, c = C.c_void_p(0x10000), C.c_void_p(0x20000), C.c_void_p(0x30000)
    for uh, u, lam in [(a, a, c), (a, b, b), (a, b, a)]:
        rc = L.snap_project_noalloc(p.handle, 2, uh, c, u, lam, None, C.byref(o), None)
        assert rc == 1
        assert "alias" in L.snap_last_error().decode()
    # families outside A and B are refused with a message that names them
    e = Problem("E", 9, 5, n_flux=1)
    rc = L.snap_project_noalloc(e.handle, 2, a, c, b, C.c_void_p(0x40000), None, C.byref(o), None)
    assert rc == 2 and "families A and B" in L.snap_last_error().decode()


def test_binding_rejects_short_buffers_without_launching():
    """The binding compares every buffer with the problem's sizes before any call: a short
    tensor would otherwise be written past its end on the device."""
    import torch
    p = Problem("B", 16, 6)
    B = 3
    uh = torch.zeros(B, p.n_vars, dtype=torch.float64)
    pr = torch.zeros(B, p.n_params, dtype=torch.float64)
    lam = torch.zeros(B, p.n_rows, dtype=torch.float64)
    st = torch.zeros(B, 40, dtype=torch.uint8)
    p._check_sizes(B, uh, pr, uh, lam, st)
    for bad in [dict(params=pr[:, :-1]), dict(u=uh[:, :-1]), dict(lam=lam[:2]),
                dict(st=st[:, :39]), dict(u_hat=uh[:2])]:
        kw = dict(u_hat=uh, params=pr, u=uh, lam=lam, st=st)
        kw.update(bad)
        with pytest.raises(ValueError):
            p._check_sizes(B, **kw)


def test_batch_rejects_2d_sides_it_does_not_hold_without_a_device():
    """The uneven batch holds the frame code of the power-of-two sides only: a family C
    problem of another side is refused when the batch is created (before any device work)."""
    from paper_2607_00095_b300.api import Batch
    with pytest.raises(_abi.SnapError) as ei:
        Batch([Problem("C", 12, 2)], [0])
    assert ei.value.code == 2
    assert b"4, 8, 16, 32 and 64" in _abi.lib().snap_last_error()
