"""GPU parity of the PCFM sampling pass (snap_pcfm_sample: shoot / project / pull-back
steps with the analytic velocity) against the oracle's loop on the same seeded inputs."""
import numpy as np
import pytest
import torch

from oracle import closed_form, pcfm, problems, solve
from paper_2607_00095_b300 import Problem, _abi, decode_stats, options, synthetic
from tests import gpu_helpers as H
from tests import pins_1d

pytestmark = pytest.mark.gpu


def _run(p, u0, x1, xi, pr, n_steps, sigma0, **opt):
    d = [H.to_dev(a) for a in (u0, x1, xi, pr)]
    u, lam, st = p.pcfm_sample(*d, n_steps=n_steps, sigma0=sigma0, opts=options(**opt))
    torch.cuda.synchronize()
    return u.cpu().numpy(), lam.cpu().numpy(), decode_stats(st), d


@pytest.mark.parametrize("family,nx,nt,B,N,s0,seed", [("B", 16, 5, 3, 4, 0.3, 51),
                                                       ("B", 128, 33, 4, 10, 0.3, 52),
                                                       ("A", 32, 6, 2, 3, 0.8, 53)])
def test_pcfm_1d_against_oracle_loop(family, nx, nt, B, N, s0, seed):
    u0, x1, xi, pr = synthetic.gen_pcfm(seed, B, nx, nt, family)
    p = Problem(family, nx, nt)
    u, lam, st, _ = _run(p, u0, x1, xi, pr, N, s0)
    assert (st["status"] == 0).all() and st["h_inf"].max() <= H.H_TOL
    proj = lambda y: solve.project_1d(family, nx, nt, pr, y)[:3]
    ue, le, so = pcfm.sample(proj, u0, x1, xi, N, s0)
    assert (so["status"] == 0).all()
    H.assert_u_close(u, ue)
    H.assert_lam_close(problems.structure_1d(family, nx, nt), lam, le)


def test_pcfm_no_perturbation_equals_projection_of_data():
    nx, nt, B = 32, 8, 3
    u0, x1, xi, pr = synthetic.gen_pcfm(54, B, nx, nt, "A")
    p = Problem("A", nx, nt)
    u, lam, st, _ = _run(p, u0, x1, xi, pr, 6, 0.0, tol_kkt=1e-13)
    ue, le = pins_1d.family_a_closed_form(nx, nt, pr, x1)
    H.assert_u_close(u, ue)


def test_pcfm_2d_against_closed_form_loop():
    N, nt, B, steps = 16, 2, 2, 3
    x1, pr = synthetic.gen_2d(55, B, N, nt, kmax=7)
    rng = np.random.default_rng(56)
    u0 = rng.normal(size=(B, x1[0].size))
    xi = rng.normal(size=(B, x1[0].size))
    x1 = x1.reshape(B, -1)
    p = Problem("C", N, nt)
    u, lam, st, _ = _run(p, u0, x1, xi, pr, steps, 0.2)
    assert (st["status"] == 0).all()
    def proj(y):
        wc, lc = closed_form.project_2d(y.reshape(B, nt, 2, N, N), pr)
        return wc.reshape(B, -1), lc, None

    ue, le, _ = pcfm.sample(proj, u0, x1, xi, steps, 0.2)
    H.assert_u_close(u, ue)
    H.assert_lam_close(problems.structure_2d(N, nt), lam, le)


def test_pcfm_full_size_sampled_and_graph():
    """The sampling workload: B = 512 Burgers samples, 10 steps; a captured pass replays to
    the same bits; sampled samples against the oracle loop."""
    w = synthetic.WORKLOADS["pcfm_1d"]
    B, nx, nt, N, s0 = w["B"], w["nx"], w["nt"], w["n_steps"], w["sigma0"]
    u0, x1, xi, pr = synthetic.gen_pcfm(w["seed"], B, nx, nt, w["family"])
    p = Problem("B", nx, nt)
    u, lam, st, d = _run(p, u0, x1, xi, pr, N, s0)
    ok = st["status"] == 0
    assert ok.sum() >= B - 2 and st["h_inf"][ok].max() <= H.H_TOL
    out = (torch.empty_like(d[0]), torch.empty(B, p.n_rows, dtype=torch.float64, device="cuda"),
           torch.empty(B, 40, dtype=torch.uint8, device="cuda"))
    p.pcfm_sample(*d, n_steps=N, sigma0=s0, out=out)        # warm-up outside the capture
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            p.pcfm_sample(*d, n_steps=N, sigma0=s0, out=out, stream=s)
    out[0].zero_()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out[0].cpu().numpy(), u)
    pick = [int(i) for i in np.nonzero(ok)[0][[0, 7, 300]]]
    proj = lambda y: solve.project_1d("B", nx, nt, pr[pick], y)[:3]
    ue, le, so = pcfm.sample(proj, u0[pick], x1[pick], xi[pick], N, s0)
    assert (so["status"] == 0).all()
    H.assert_u_close(u[pick], ue)
    H.assert_lam_close(problems.structure_1d("B", nx, nt), lam[pick], le)


def test_pcfm_errors():
    p = Problem("B", 16, 3)
    u0, x1, xi, pr = synthetic.gen_pcfm(57, 1, 16, 3)
    d = [H.to_dev(a) for a in (u0, x1, xi, pr)]
    with pytest.raises(_abi.SnapError):
        p.pcfm_sample(*d, n_steps=0)
    with pytest.raises(_abi.SnapError):
        p.pcfm_sample(*d, n_steps=2, sigma0=float("nan"))


def test_pcfm_family_d_against_oracle_loop():
    """The sampling pass on the Burgers boundary-condition rows (family D, odd nx)."""
    nx, nt, B, N, s0 = 21, 5, 3, 4, 0.2
    x1, pr = synthetic.gen_burgers_bc(58, B, nx, nt)
    x1 = x1.reshape(B, -1)
    rng = np.random.default_rng(59)
    u0 = rng.normal(size=x1.shape)
    xi = rng.normal(size=x1.shape)
    p = Problem("D", nx, nt)
    u, lam, st, _ = _run(p, u0, x1, xi, pr, N, s0)
    assert (st["status"] == 0).all()
    S = problems.structure_bc(nx, nt)
    b = problems.rhs_bc(nx, nt, pr)
    ue, le, so = pcfm.sample(lambda y: solve.project(S, b, y), u0, x1, xi, N, s0)
    assert (so["status"] == 0).all()
    H.assert_u_close(u, ue)
    H.assert_lam_close(S, lam, le)


def test_pcfm_family_e_against_oracle_loop():
    """The sampling pass on the Burgers IC + mass + Godunov flux rows (family E)."""
    from types import SimpleNamespace

    from oracle import flux
    nx, nt, K, B, N, s0 = 17, 20, 3, 3, 4, 0.2
    x1, g = synthetic.gen_burgers_flux(60, B, nx, nt)
    x1 = x1.reshape(B, -1)
    rng = np.random.default_rng(61)
    u0 = rng.normal(size=x1.shape)
    xi = rng.normal(size=x1.shape)
    p = Problem("E", nx, nt, n_flux=K)
    u, lam, st, _ = _run(p, u0, x1, xi, g, N, s0)
    assert (st["status"] == 0).all() and st["h_inf"].max() <= H.H_TOL
    ue, le, _ = pcfm.sample(lambda y: flux.project(nx, nt, K, g, y), u0, x1, xi, N, s0)
    H.assert_u_close(u, ue)
    H.assert_lam_close(SimpleNamespace(row_type=flux.row_types(nx, nt, K)), lam, le)
