"""Pins of the family-E oracle (Burgers IC + mass + Godunov flux rows) against facts that do
not come from the oracle itself: the exact Riemann solution of Burgers' equation sampled at
the interface, the upwind scheme it reduces to for one-signed data, conservation of the
periodic update, the Rankine-Hugoniot shock speed, a finite-difference Jacobian, the
Newton-KKT iteration of Appendix B and finite differences of the solution map."""
import numpy as np
import pytest

from oracle import flux
from paper_2607_00095_b300 import synthetic


def riemann_state_at_interface(a, b):
    """Entropy solution of u_t + (u^2/2)_x = 0 with data a | b, sampled on x/t = 0: a shock
    of speed (a + b)/2 when a > b, a rarefaction fan with speeds in [a, b] when a <= b."""
    if a > b:
        return a if (a + b) / 2 > 0 else b
    if a >= 0:
        return a
    if b <= 0:
        return b
    return 0.0


def test_flux_textbook_values():
    cases = [((1.0, 0.0), 0.5),      # right-moving shock: upwind state 1
             ((0.0, 1.0), 0.0),      # rarefaction from 0
             ((-1.0, 1.0), 0.0),     # transonic rarefaction: sonic point 0
             ((1.0, -1.0), 0.5),     # stationary shock
             ((-1.0, -2.0), 2.0),    # left-moving shock: upwind state -2
             ((2.0, 3.0), 2.0),      # right-moving rarefaction: upwind state 2
             ((-3.0, -2.0), 2.0)]    # left-moving rarefaction: upwind state -2
    for (a, b), want in cases:
        assert flux.godunov_flux(a, b) == want, (a, b)


def test_flux_is_f_of_riemann_state():
    rng = np.random.default_rng(7)
    ab = rng.uniform(-2, 2, size=(4000, 2))
    ab[:200, 1] = -ab[:200, 0]                   # stationary shocks / symmetric fans
    ab[200:300, 1] = ab[200:300, 0]              # constant states
    for a, b in ab:
        w = riemann_state_at_interface(a, b)
        assert abs(flux.godunov_flux(a, b) - 0.5 * w * w) <= 1e-15 * (1 + w * w), (a, b)


def test_flux_branch_derivatives_match_differences():
    rng = np.random.default_rng(8)
    ab = rng.uniform(-2, 2, size=(2000, 2))
    ia, ib = flux.flux_branch(ab[:, 0], ab[:, 1])
    e = 1e-7
    da = (flux.godunov_flux(ab[:, 0] + e, ab[:, 1]) - flux.godunov_flux(ab[:, 0] - e, ab[:, 1])) / (2 * e)
    db = (flux.godunov_flux(ab[:, 0], ab[:, 1] + e) - flux.godunov_flux(ab[:, 0], ab[:, 1] - e)) / (2 * e)
    far = np.minimum.reduce([np.abs(ab[:, 0]), np.abs(ab[:, 1]), np.abs(ab[:, 0] - ab[:, 1]),
                             np.abs(ab[:, 0] + ab[:, 1])]) > 1e-5
    np.testing.assert_allclose((ia * ab[:, 0])[far], da[far], atol=1e-7)
    np.testing.assert_allclose((ib * ab[:, 1])[far], db[far], atol=1e-7)


def test_step_conserves_and_reduces_to_upwind():
    rng = np.random.default_rng(9)
    c = 0.8
    v = rng.normal(size=(16, 37))
    np.testing.assert_allclose(flux.godunov_step(v, c).sum(axis=1), v.sum(axis=1), atol=1e-12)
    pos = rng.uniform(0.1, 1.0, size=(8, 29))
    up = pos - c * (0.5 * pos ** 2 - 0.5 * np.roll(pos, 1, axis=1) ** 2)
    np.testing.assert_allclose(flux.godunov_step(pos, c), up, rtol=0, atol=1e-15)
    neg = -pos
    upn = neg - c * (0.5 * np.roll(neg, -1, axis=1) ** 2 - 0.5 * neg ** 2)
    np.testing.assert_allclose(flux.godunov_step(neg, c), upn, rtol=0, atol=1e-15)


def test_shock_moves_mass_at_rankine_hugoniot_speed():
    # states 1 | 0: the shock speed is 1/2, so the mass right of the jump grows by dt/2 a step
    nx, nt = 101, 101
    dx, dt, c = flux.grid(nx, nt)
    j = 50
    v = np.where(np.arange(nx) < j, 1.0, 0.0)
    m0 = dx * v[j:].sum()
    for n in range(1, 21):
        v = flux.godunov_step(v, c)
        assert abs(dx * v[j:].sum() - m0 - n * dt / 2) < 1e-13, n


def small_case(seed, B, nx, nt):
    uh, g = synthetic.gen_burgers_flux(seed, B, nx, nt)
    return uh.reshape(B, -1), g


def fd_jacobian(nx, nt, K, g, u, e=1e-6):
    n = u.size
    m = flux.sizes(nx, nt, K)[1]
    J = np.zeros((m, n))
    for j in range(n):
        up, um = u.copy(), u.copy()
        up[j] += e
        um[j] -= e
        J[:, j] = (flux.eval_h(nx, nt, K, g[None], up[None])[0]
                   - flux.eval_h(nx, nt, K, g[None], um[None])[0]) / (2 * e)
    return J


def kink_distance(nx, nt, K, u):
    """Smallest distance of the chain's flux arguments to a branch switch of F."""
    U = u.reshape(-1, nt, nx)[:, :K]
    a, b = U, np.roll(U, -1, axis=-1)
    return min(np.abs(a).min(), np.abs(b).min(), np.abs(a + b).min())


@pytest.mark.parametrize("K,signed", [(1, False), (3, False), (3, True)])
def test_definition_is_a_kkt_point(K, signed):
    # finite differences need the flux arguments away from the switches of F: the front's
    # tail (g ~ 1e-10) is lifted by 0.05, or g is drawn with both signs
    nx, nt = 10, 12                          # dt/dx = 9/11 (CFL <= 1 for |u| <= 1)
    uh, g = small_case(11, 3, nx, nt)
    g = np.random.default_rng(21).uniform(-1, 1, size=g.shape) if signed else g + 0.05
    u, lam, st = flux.project(nx, nt, K, g, uh)
    assert kink_distance(nx, nt, K, u) > 1e-4
    act = flux.active_rows(nx, nt, K).astype(bool)
    assert np.all(lam[:, ~act] == 0)
    assert st["h_inf"].max() < 1e-14          # every nominal row, the implied mass rows too
    for b in range(3):
        J = fd_jacobian(nx, nt, K, g[b], u[b])
        gl = u[b] - uh[b] + J[act].T @ lam[b, act]
        assert np.abs(gl).max() < 1e-8 * max(1.0, np.abs(lam[b]).max())
        np.testing.assert_allclose(J, flux.full_jacobian(nx, nt, K, u[b]), atol=1e-8)


def test_mass_slices_are_the_nearest_feasible_points():
    nx, nt, K = 10, 6, 2
    uh, g = small_case(12, 2, nx, nt)
    u, _, _ = flux.project(nx, nt, K, g, uh)
    U, Uh = u.reshape(2, nt, nx), uh.reshape(2, nt, nx)
    rng = np.random.default_rng(3)
    for b in range(2):
        for k in range(K + 1, nt):
            d = U[b, k] - Uh[b, k]
            assert np.ptp(d) < 1e-14        # a uniform shift: orthogonal to the feasible plane
            for _ in range(20):
                z = rng.normal(size=nx)
                z -= z.mean()
                assert 0.5 * ((U[b, k] + 0.1 * z - Uh[b, k]) ** 2).sum() > 0.5 * (d ** 2).sum()


@pytest.mark.parametrize("K", [1, 2, 4])
def test_newton_kkt_reaches_the_definition(K):
    nx, nt = 8, 6
    uh, g = small_case(13, 2, nx, nt)
    u, lam, _ = flux.project(nx, nt, K, g, uh)
    for b in range(2):
        un, ln, it, ok = flux.newton_kkt(nx, nt, K, g[b], uh[b])
        assert ok and it >= 2
        np.testing.assert_allclose(un, u[b], rtol=0, atol=1e-12)
        np.testing.assert_allclose(ln, lam[b], rtol=0, atol=1e-9 * max(1.0, np.abs(lam[b]).max()))


def test_adjoint_matches_finite_differences():
    nx, nt, K = 12, 7, 3
    uh, g = small_case(14, 2, nx, nt)
    g = g + 0.05
    rng = np.random.default_rng(15)
    gbar = rng.normal(size=uh.shape)
    u, _, _ = flux.project(nx, nt, K, g, uh)
    assert kink_distance(nx, nt, K, u) > 1e-4
    a, gg, _ = flux.adjoint(nx, nt, K, g, u, gbar)

    def loss(uh_, g_):
        return (flux.project(nx, nt, K, g_, uh_)[0] * gbar).sum(axis=1)

    e = 1e-6
    for _ in range(4):
        d = rng.normal(size=uh.shape)
        fd = (loss(uh + e * d, g) - loss(uh - e * d, g)) / (2 * e)
        np.testing.assert_allclose((a * d).sum(axis=1), fd, rtol=1e-6, atol=1e-8)
    for i in range(nx):
        dg = np.zeros_like(g)
        dg[:, i] = e
        fd = (loss(uh, g + dg) - loss(uh, g - dg)) / (2 * e)
        np.testing.assert_allclose(gg[:, i], fd, rtol=1e-5, atol=1e-7)


# ---- the pins are sensitive: each plausible slip planted in the oracle fails one of them ----

def _mut_step_sign(v, c):
    v = np.asarray(v, np.float64)
    Fr = flux.godunov_flux(v, np.roll(v, -1, axis=-1))
    return v + c * (Fr - np.roll(Fr, 1, axis=-1))


def _mut_flux_shock_branch(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    fa, fb = 0.5 * a * a, 0.5 * b * b
    lo = np.where(a > 0, fa, np.where(b < 0, fb, 0.0))
    return np.where(a <= b, lo, np.minimum(fa, fb))


def _mut_branch_swapped(a, b):
    ia, ib = ORIG_BRANCH(a, b)
    return ib, ia


def _mut_lambda_transposed(nx, nt, K, u_chain):
    return ORIG_CHAIN(nx, nt, K, u_chain).T


ORIG_BRANCH = flux.flux_branch
ORIG_CHAIN = flux.chain_jacobian
PINS = [test_flux_textbook_values, test_flux_is_f_of_riemann_state,
        test_flux_branch_derivatives_match_differences, test_step_conserves_and_reduces_to_upwind,
        test_shock_moves_mass_at_rankine_hugoniot_speed,
        lambda: test_definition_is_a_kkt_point(3, True),
        lambda: test_newton_kkt_reaches_the_definition(2), test_adjoint_matches_finite_differences]


@pytest.mark.parametrize("name,attr,mutant", [
    ("step_sign", "godunov_step", _mut_step_sign),
    ("shock_takes_min", "godunov_flux", _mut_flux_shock_branch),
    ("branch_swapped", "flux_branch", _mut_branch_swapped),
    ("multiplier_solve_transposed", "chain_jacobian", _mut_lambda_transposed)])
def test_pins_catch_mutant(monkeypatch, name, attr, mutant):
    monkeypatch.setattr(flux, attr, mutant)
    failed = 0
    for pin in PINS:
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError):
            failed += 1
    assert failed >= 1, name
