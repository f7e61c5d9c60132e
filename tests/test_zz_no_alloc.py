"""snap_project_noalloc (forward projection with the library's static device scratch) against
snap_project on the same seeded inputs, within the parity tolerances of the other GPU tests.

Collected last on purpose: it must pass after every other test has used the library (and the
static scratch then holds whatever the previous calls left), as well as alone."""
import numpy as np
import pytest
import torch

from paper_2607_00095_b300 import Problem, _abi, decode_stats, options, synthetic
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _noalloc(p, uh, pr, **opt):
    B = uh.shape[0]
    u = torch.full_like(uh, np.nan)
    lam = torch.full((B, p.n_rows), np.nan, dtype=torch.float64, device=uh.device)
    st = torch.full((B, 40), 255, dtype=torch.uint8, device=uh.device)
    p.project_noalloc(uh, pr, u, lam, st, opts=options(**opt))
    torch.cuda.synchronize()
    return u.cpu().numpy(), lam.cpu().numpy(), decode_stats(st)


def _compare(p, uh, pr, **opt):
    u1, l1, s1 = _noalloc(p, uh, pr, **opt)
    u0, l0, s0 = p.project(uh, pr, opts=options(**opt))
    torch.cuda.synchronize()
    s0 = decode_stats(s0)
    np.testing.assert_array_equal(s1["status"], s0["status"])
    ok = s0["status"] == 0
    assert ok.any()
    H.assert_u_close(u1[ok], u0.cpu().numpy()[ok])
    lam0 = l0.cpu().numpy()[ok]
    for s in range(lam0.shape[0]):
        den = max(np.abs(lam0[s]).max(), 1e-12)
        assert np.abs(l1[ok][s] - lam0[s]).max() / den <= H.LAM_RTOL
    assert s1["h_inf"][ok].max() <= H.H_TOL
    return s1


@pytest.mark.parametrize("family,nx,nt,B,seed", [("B", 128, 100, 512, 9001), ("A", 32, 32, 8, 9002)])
def test_noalloc_matches_project_twice(family, nx, nt, B, seed):
    p = Problem(family, nx, nt)
    for call, (bb, sd) in enumerate([(B, seed), (max(1, B // 2 - 3), seed + 1)]):
        uh, pr = synthetic.gen_1d(sd, bb, nx, nt, family=family)
        uh = H.to_dev(uh.reshape(bb, -1))
        pr = H.to_dev(pr)
        st = _compare(p, uh, pr)
        assert (st["status"] == 0).all(), f"call {call}"


def test_noalloc_limits():
    p = Problem("B", 128, 100)
    B = 2048                                      # 204,800 slices: above the static scratch
    assert p.workspace_bytes(B) > _abi.NOALLOC_SCRATCH_BYTES
    uh = torch.zeros(B, p.n_vars, dtype=torch.float64, device="cuda:0")
    pr = torch.zeros(B, p.n_params, dtype=torch.float64, device="cuda:0")
    u = torch.empty_like(uh)
    lam = torch.empty(B, p.n_rows, dtype=torch.float64, device="cuda:0")
    st = torch.empty(B, 40, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(_abi.SnapError) as ei:
        p.project_noalloc(uh, pr, u, lam, st)
    assert ei.value.code == 5
    assert "static array" in str(ei.value)
    q = Problem("C", 8, 2)
    with pytest.raises(_abi.SnapError) as ei:
        q.project_noalloc(uh[:1, :q.n_vars].contiguous(), pr[:1, :q.n_params].contiguous(),
                          u[:1, :q.n_vars].contiguous(), lam[:1, :q.n_rows].contiguous(), st[:1])
    assert ei.value.code == 2
