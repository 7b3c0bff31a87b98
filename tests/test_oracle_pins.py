"""Pins of the FP64 CPU oracle against facts fixed outside the oracle itself.

Each test pins a part of the method to something other than the oracle's own
formula: finite-difference stencils and explicit DFT matrices, closed-form
solutions, brute-force dense solves of the converged problem, and invariants.
"""
import numpy as np
import pytest

from oracle import acm_oracle as O
from paper_2312_15554_gb300 import inputs as I
from tests import dense_ops as DO

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# --------------------------------------------------------------------------
# symbols and transforms (Eq. 13, Eq. 21)
# --------------------------------------------------------------------------
def test_forward_dft_convention_direct_sum():
    shape = (4, 6, 8)
    f = I.random_field(shape, 1)
    fh = O.fft3(f)
    j = [np.arange(n) for n in shape]
    for m in [(0, 0, 0), (1, 2, 3), (3, 5, 7), (2, 3, 4)]:
        ph = (np.exp(-2j * np.pi * m[0] * j[0] / shape[0])[:, None, None]
              * np.exp(-2j * np.pi * m[1] * j[1] / shape[1])[None, :, None]
              * np.exp(-2j * np.pi * m[2] * j[2] / shape[2])[None, None, :])
        assert abs(fh[m] - np.sum(f * ph)) < 1e-12 * np.sum(np.abs(f))


def test_central_symbols_are_the_central_difference_stencils():
    shape = (8, 6, 10)
    f = I.random_field(shape, 2)
    d, L = O.symbols(shape, O.CENTRAL)
    g_spec = O.spectral_grad(f, d)
    np.testing.assert_allclose(g_spec, DO.grad_fd(f), atol=1e-11 * np.abs(g_spec).max())
    lap_spec = O.ifft3(L * O.fft3(f))
    np.testing.assert_allclose(lap_spec, DO.lap_neg_fd(f), atol=1e-11 * np.abs(lap_spec).max())


def test_exact_symbols_differentiate_single_modes_exactly():
    shape = (8, 8, 16)
    x = [(np.arange(n) + 0.5) / n for n in shape]
    X = np.meshgrid(*x, indexing="ij")
    d, L = O.symbols(shape, O.EXACT)
    for m in [(1, 0, 0), (0, 3, 0), (2, -1, 7), (3, 3, -5)]:
        ph = 2 * np.pi * sum(m[c] * X[c] for c in range(3))
        f = np.cos(ph)
        gr = O.spectral_grad(f, d)
        for c in range(3):
            np.testing.assert_allclose(gr[c], -2 * np.pi * m[c] * np.sin(ph), atol=1e-10)
        lap = O.ifft3(L * O.fft3(f))
        np.testing.assert_allclose(lap, (2 * np.pi) ** 2 * sum(mc * mc for mc in m) * f, atol=1e-8)


# --------------------------------------------------------------------------
# one ADMM iteration satisfies Eq. 7, 8, 9 (stencils, not FFTs)
# --------------------------------------------------------------------------
def _random_state(shape, seed):
    r = lambda s, k: I.random_field(s, seed + k)
    return O.StokesState(u=r((3,) + shape, 1), ut=r((3,) + shape, 2), q=r(shape, 3),
                         a=r((3,) + shape, 4), lam=r((3,) + shape, 5))


@pytest.mark.parametrize("shape", [(6, 8, 4), (8, 8, 8)])
def test_one_admm_iteration_satisfies_steps_1_to_3_central(shape):
    H = I.random_indicator(shape, 0.4, 11)
    Hf = H.astype(float)
    X0 = _random_state(shape, 20)
    g = np.array([0.7, -0.2, 1.3])
    nu, alpha, beta, b = 1.7, 40.0, 25.0, 60.0
    P = O.StokesParams(nu=nu, eps=0.0, alpha0=alpha, beta0=beta, b0=b, adaptive=False,
                       max_iter=1, deriv=O.CENTRAL)
    R = O.stokes(H, g, P, init=X0)
    X1 = R.state
    # Eq. 7 with central-difference operators
    res = (nu * np.stack([DO.lap_neg_fd(X1.u[c]) for c in range(3)])
           - g[:, None, None, None] + DO.grad_fd(X0.q)
           - beta * DO.grad_fd(DO.div_fd(X1.u)) + X0.a + b * (X1.u - X0.ut))
    scale = np.abs(X0.a).max() + b * np.abs(X0.ut).max()
    assert np.abs(res).max() < 1e-10 * scale
    # Eq. 8
    res8 = -X0.a - b * (X1.u - X1.ut) + Hf * X0.lam + alpha * Hf * X1.ut
    assert np.abs(res8).max() < 1e-10 * scale
    # Eq. 9
    np.testing.assert_allclose(X1.q, X0.q - beta * DO.div_fd(X1.u), atol=1e-10 * scale)
    np.testing.assert_allclose(X1.a, X0.a + b * (X1.u - X1.ut), atol=1e-10 * scale)
    np.testing.assert_allclose(X1.lam, X0.lam + alpha * Hf * X1.ut, atol=1e-10 * scale)
    # Eq. 10 residuals of that iteration
    rp = R.residuals[0]
    assert rp[0] == pytest.approx(np.linalg.norm(Hf * X1.ut))
    assert rp[3] == pytest.approx(beta * np.linalg.norm(DO.div_fd(X1.u) - DO.div_fd(X0.u)), rel=1e-9)
    assert rp[5] == pytest.approx(b * np.linalg.norm(X1.u - X0.u))


def test_one_admm_iteration_satisfies_step_1_exact_dft_matrices():
    shape = (4, 6, 4)
    H = I.random_indicator(shape, 0.4, 12)
    X0 = _random_state(shape, 40)
    g = np.array([1.0, 0.5, -0.25])
    nu, alpha, beta, b = 1.0, 30.0, 20.0, 50.0
    P = O.StokesParams(nu=nu, eps=0.0, alpha0=alpha, beta0=beta, b0=b, adaptive=False,
                       max_iter=1, deriv=O.EXACT)
    X1 = O.stokes(H, g, P, init=X0).state
    D, Lneg = DO.exact_ops(shape)
    V = H.size
    u = X1.u.reshape(3, V)
    divu = sum(D[c] @ u[c] for c in range(3))
    for c in range(3):
        res = (nu * Lneg @ u[c] - g[c] + D[c] @ X0.q.ravel() - beta * D[c] @ divu
               + X0.a[c].ravel() + b * (u[c] - X0.ut[c].ravel()))
        assert np.abs(res).max() < 1e-9 * (b * np.abs(X0.ut).max())


# --------------------------------------------------------------------------
# converged ADMM = dense KKT solve of the discrete Stokes problem
# --------------------------------------------------------------------------
@pytest.mark.parametrize("deriv", [O.CENTRAL, O.EXACT])
@pytest.mark.parametrize("shape,seed", [((4, 4, 4), 3), ((6, 4, 6), 5), ((1, 8, 6), 7)])
def test_converged_stokes_matches_dense_kkt(deriv, shape, seed):
    H = I.random_indicator(shape, 0.35, seed)
    if H.sum() == 0:
        H[0, 0, 0] = 1
    g = np.array([1.0, -0.3, 0.6])
    D, Lneg = (DO.central_ops(shape) if deriv == O.CENTRAL else DO.exact_ops(shape))
    u_kkt = DO.stokes_kkt(H, g, D, Lneg)
    P = O.StokesParams(eps=1e-13, alpha0=300, beta0=300, b0=300, adaptive=False,
                       max_iter=40000, deriv=deriv)
    R = O.stokes(H, g, P)
    assert R.converged
    np.testing.assert_allclose(R.state.u, u_kkt, atol=1e-9 * np.abs(u_kkt).max())


def test_converged_result_is_penalty_independent():
    shape = (6, 6, 6)
    H = I.random_indicator(shape, 0.3, 9)
    g = [0.0, 1.0, 0.0]
    Ra = O.stokes(H, g, O.StokesParams(eps=1e-12, alpha0=300, beta0=300, b0=300, adaptive=False))
    Rb = O.stokes(H, g, O.StokesParams(eps=1e-12, alpha0=50, beta0=900, b0=150, adaptive=True))
    assert Ra.converged and Rb.converged
    np.testing.assert_allclose(Ra.state.u, Rb.state.u, atol=1e-8 * np.abs(Ra.state.u).max())


def test_consistent_pressure_of_a_gradient_force_is_minus_its_potential():
    # a = grad(phi) is balanced by q = -phi (Eq. 7 with u = 0); phi in the band
    # of the exact symbols, its gradient written out by hand
    shape = (8, 12, 16)
    x = [(np.arange(n) + 0.5) / n for n in shape]
    X0, X1, X2 = np.meshgrid(*x, indexing="ij")
    tp = 2 * np.pi
    phi = np.sin(tp * X0) * np.cos(tp * 2 * X1) + 0.5 * np.cos(tp * 3 * X2)
    a = np.stack([tp * np.cos(tp * X0) * np.cos(tp * 2 * X1),
                  -2 * tp * np.sin(tp * X0) * np.sin(tp * 2 * X1),
                  -1.5 * tp * np.sin(tp * 3 * X2)])
    d, _ = O.symbols(shape, O.EXACT)
    q = O.consistent_pressure(a, d)
    np.testing.assert_allclose(q, -(phi - phi.mean()), atol=1e-12)


@pytest.mark.parametrize("deriv", [O.EXACT, O.CENTRAL])
def test_converged_pressure_is_the_consistent_pressure_of_the_multiplier(deriv):
    shape = (8, 8, 8)
    H = I.random_indicator(shape, 0.3, 4)
    R = O.stokes(H, [0.3, 1.0, -0.5], O.StokesParams(eps=1e-12, alpha0=300, beta0=300, b0=300, adaptive=False,
                                                     max_iter=40000, deriv=deriv))
    assert R.converged
    d, _ = O.symbols(shape, deriv)
    q = O.consistent_pressure(R.state.a, d)
    np.testing.assert_allclose(q, R.p, atol=1e-7 * np.abs(R.p).max())


def test_restart_from_a_converged_velocity_and_multiplier_stops_at_once():
    shape = (8, 8, 8)
    H = I.random_indicator(shape, 0.3, 5)
    P = O.StokesParams(eps=1e-9, alpha0=300, beta0=300, b0=300, adaptive=False, max_iter=40000)
    R = O.stokes(H, [1.0, 0.0, 0.0], P)
    assert R.converged and R.iters > 50
    init = O.warm_state(H, R.state.u, R.state.lam)
    R2 = O.stokes(H, [1.0, 0.0, 0.0], P, init=init)
    assert R2.converged and R2.iters <= 8
    # without the consistent pressure the restart is far from done
    init.q[...] = 0.0
    R3 = O.stokes(H, [1.0, 0.0, 0.0], P, init=init)
    assert R3.iters > 10 * R2.iters


# --------------------------------------------------------------------------
# plane Poiseuille flow (closed forms)
# --------------------------------------------------------------------------
def test_plane_poiseuille_central_discrete_closed_form():
    n, s = 16, 5                       # s solid layers normal to axis 1, m = n - s fluid layers
    H = I.slab((4, n, 4), s, normal_axis=1)
    m = n - s
    h = 1.0 / n
    P = O.StokesParams(eps=1e-12, alpha0=300, beta0=300, b0=300, adaptive=False,
                       max_iter=60000, deriv=O.CENTRAL)
    R = O.stokes(H, [1.0, 0.0, 0.0], P)
    assert R.converged
    j = np.arange(1, m + 1)
    profile = np.zeros(n)
    profile[s:] = h * h * j * (m + 1 - j) / 2.0       # -u'' = 1 discretely, u = 0 on the walls
    np.testing.assert_allclose(R.state.u[0, 1, :, 2], profile, atol=1e-9 * profile.max())
    assert np.abs(R.state.u[1:]).max() < 1e-9 * profile.max()
    K = h * h * m * (m + 1) * (m + 2) / (12.0 * n)
    assert R.K_col[0] == pytest.approx(K, rel=1e-8)


def test_plane_poiseuille_exact_symbol_bracketed_and_converging():
    errs = []
    for n in (8, 16, 32):
        s = n // 4
        m = n - s
        h = 1.0 / n
        H = I.slab((2, n, 2), s, normal_axis=1)
        R = O.stokes(H, [1.0, 0.0, 0.0], O.StokesParams(eps=1e-10, alpha0=300, beta0=300, b0=300,
                                                        adaptive=False, max_iter=60000))
        assert R.converged
        K = R.K_col[0]
        assert (m * h) ** 3 / 12 < K < ((m + 1) * h) ** 3 / 12
        errs.append(abs(K - (0.75) ** 3 / 12))   # wall midway between the last solid and first fluid centre
    assert errs[2] < errs[1] < errs[0]


# --------------------------------------------------------------------------
# Eq. 2 literally: K_ij = integral over Y_p of grad u^i : grad u^j
# --------------------------------------------------------------------------
def _poiseuille_profile(n, s):
    """Discrete central-symbol Poiseuille profile of a slab (s solid layers at
    the start of axis 1, m = n - s fluid layers), g = nu = 1: u_j = h^2 j (m + 1 - j) / 2."""
    m = n - s
    h = 1.0 / n
    prof = np.zeros(n)
    j = np.arange(1, m + 1)
    prof[s:] = h * h * j * (m + 1 - j) / 2.0
    return prof


def test_gradient_form_of_the_discrete_poiseuille_profile():
    """With the central symbol the gradient of u_j = h^2 j (m + 1 - j)/2 at fluid
    layer j is the central difference (u_{j+1} - u_{j-1}) / 2h = h (m + 1 - 2j)/2
    (u = 0 in the walls), so over the pore Eq. 2 gives
    h^3 N^2 sum_j h^2 (m + 1 - 2j)^2 / 4 = h^3 m (m^2 - 1) / 12 (unit cube)."""
    n, s = 16, 5
    m, h = n - s, 1.0 / n
    H = I.slab((4, n, 4), s, normal_axis=1)
    u = np.zeros((3,) + H.shape)
    u[0] = _poiseuille_profile(n, s)[None, :, None]
    Kg = O.permeability_grad_form(H, [u], O.CENTRAL)
    closed = h**3 * m * (m * m - 1) / 12.0
    assert Kg[0, 0] == pytest.approx(closed, rel=1e-12)
    # the same sum with the stencils written out (pore voxels only)
    grad = np.stack([DO.grad_fd(u[c]) for c in range(3)])
    pore = H == 0
    assert np.sum((grad * grad)[:, :, pore]) / H.size == pytest.approx(closed, rel=1e-12)
    # the integral over all of Y (walls included) is a different number: the
    # central difference at the wall layers next to the fluid is not zero
    assert np.sum(grad * grad) / H.size > closed * (1 + 1e-2)
    # and so is the exact symbol's gradient of the same field
    assert abs(O.permeability_grad_form(H, [u], O.EXACT)[0, 0] / closed - 1) > 1e-2


def test_gradient_form_of_a_single_mode_over_half_the_cell():
    """u = (cos 2 pi m x1, 0, 0) with the exact symbols has |grad u|^2 =
    (2 pi m)^2 sin^2(2 pi m x1); over a pore that is the half x0 < 1/2 of the
    cell Eq. 2 gives (2 pi m)^2 / 4. The cross term of two loads follows the
    product of their gradients."""
    shape = (8, 16, 4)
    m = 3
    x1 = (np.arange(shape[1]) + 0.5) / shape[1]
    H = np.zeros(shape, np.uint8)
    H[shape[0] // 2:] = 1
    u = np.zeros((3,) + shape)
    u[0] = np.cos(2 * np.pi * m * x1)[None, :, None]
    v = np.zeros((3,) + shape)
    v[0] = np.sin(2 * np.pi * m * x1)[None, :, None]
    K = O.permeability_grad_form(H, [u, v], O.EXACT)
    k2 = (2 * np.pi * m) ** 2
    assert K[0, 0] == pytest.approx(k2 / 4, rel=1e-12)
    assert K[1, 1] == pytest.approx(k2 / 4, rel=1e-12)
    assert abs(K[0, 1]) < 1e-12 * k2       # sin cos integrates to zero over whole periods
    Kall = O.permeability_grad_form(np.zeros(shape, np.uint8), [u], O.EXACT)
    assert Kall[0, 0] == pytest.approx(k2 / 2, rel=1e-12)


def test_converged_slab_flow_gives_the_gradient_form_closed_form():
    """The oracle's converged central-symbol slab flow, through
    permeability_tensor, reproduces h^3 m (m^2 - 1)/12 for K_grad[0, 0]."""
    n, s = 16, 5
    m, h = n - s, 1.0 / n
    H = I.slab((4, n, 4), s, normal_axis=1)
    P = O.StokesParams(eps=1e-12, alpha0=300, beta0=300, b0=300, adaptive=False, max_iter=60000,
                       deriv=O.CENTRAL)
    R = O.stokes(H, [1.0, 0.0, 0.0], P)
    assert R.converged
    Kg = O.permeability_grad_form(H, [R.state.u], O.CENTRAL)
    assert Kg[0, 0] == pytest.approx(h**3 * m * (m * m - 1) / 12.0, rel=1e-7)


# --------------------------------------------------------------------------
# Eq. 22: adaptive penalties
# --------------------------------------------------------------------------
def test_adaptive_penalty_rule_on_hand_built_residuals():
    """Each case is Eq. 22 read off its text: psi_k grows by phi_k when
    r_p / r_d > tau_k, shrinks by phi_k but not below psi_min when
    r_d / r_p > tau_k, and stays otherwise; pair k drives (alpha, beta, b)[k]."""
    psi = [10.0, 20.0, 30.0]
    phi = (1.1, 1.2, 1.5)
    tau = (5.0, 10.0, 5.0)
    psi_min = [1.0, 1.0, 29.0]
    # pair 1: r_p / r_d = 6 > 5 -> 11; pair 2: r_d / r_p = 11 > 10 -> 20 / 1.2;
    # pair 3: r_d / r_p = 10 > 5 -> max(30 / 1.5, 29) = 29
    out = O.adapt_penalties(psi, [60.0, 10.0, 1.0, 11.0, 1.0, 10.0], phi, tau, psi_min)
    np.testing.assert_allclose(out, [11.0, 20.0 / 1.2, 29.0], rtol=1e-15)
    # ratios at or inside the band leave every penalty alone
    out = O.adapt_penalties(psi, [5.0, 1.0, 1.0, 9.0, 1.0, 4.0], phi, tau, psi_min)
    np.testing.assert_allclose(out, psi, rtol=0)
    # zero residuals: 0 > tau * 0 is false, a positive primal over a zero dual grows,
    # a positive dual over a zero primal shrinks
    out = O.adapt_penalties(psi, [0.0, 0.0, 1e-3, 0.0, 0.0, 1e-3], phi, tau, psi_min)
    np.testing.assert_allclose(out, [10.0, 24.0, 29.0], rtol=1e-15)
    # shrinking stops at psi_min exactly
    out = O.adapt_penalties([1.05, 20.0, 30.0], [1.0, 100.0, 1.0, 1.0, 1.0, 1.0], phi, tau, psi_min)
    np.testing.assert_allclose(out, [1.0, 20.0, 30.0], rtol=0)


def test_admm_takes_the_next_penalties_from_this_iterations_residuals():
    """In an adaptive run the penalties of iteration n + 1 are Eq. 22 applied to
    the penalties and residuals of iteration n, and both directions occur."""
    H = I.sphere_pack((8, 8, 8), 0.5, 2.0, 3)[0]
    P = O.StokesParams(eps=0.0, adaptive=True, max_iter=40, alpha0=1.0, beta0=2000.0, b0=300.0)
    R = O.stokes(H, [1.0, 0.0, 0.0], P)
    psi_min = [P.psi_min_frac * x for x in (1.0, 2000.0, 300.0)]
    for n in range(R.iters - 1):
        nxt = O.adapt_penalties(list(R.penalties[n]), R.residuals[n], P.phi, P.tau, psi_min)
        np.testing.assert_allclose(R.penalties[n + 1], nxt, rtol=0)
    steps = np.diff(np.log(R.penalties), axis=0)
    assert (steps > 0).any() and (steps < 0).any()


# --------------------------------------------------------------------------
# periodic simple-cubic sphere array (Hasimoto 1959; Sangani & Acrivos 1982)
# --------------------------------------------------------------------------
def hasimoto_sangani_acrivos(c):
    a = (3 * c / (4 * np.pi)) ** (1 / 3)
    x = c ** (1 / 3)
    series = 1 - 1.7601 * x + c - 1.5593 * c**2 + 3.9799 * c ** (8 / 3) - 3.0734 * c ** (10 / 3)
    return series / (6 * np.pi * a)


def test_sphere_array_permeability_hasimoto():
    """Dilute simple-cubic array, central symbols: K within 10% at 32^3 and improving with N."""
    errs = []
    for n in (16, 32):
        H = I.single_sphere((n, n, n), 0.3)
        c = H.mean()
        R = O.stokes(H, [1.0, 0.0, 0.0], O.StokesParams(eps=1e-7, alpha0=300, beta0=300, b0=300,
                                                        adaptive=False, max_iter=20000,
                                                        deriv=O.CENTRAL))
        assert R.converged
        errs.append(abs(R.K_col[0] / hasimoto_sangani_acrivos(c) - 1))
    assert errs[1] < 0.10
    assert errs[1] < errs[0]


# --------------------------------------------------------------------------
# the two-dimensional cell (one plane, n0 = 1): the paper's own setting
# --------------------------------------------------------------------------
def square_cylinder_array(c):
    """Permeability of a square array of cylinders at solid fraction c (unit
    cell, nu = 1, flow across the cylinders): the dilute expansion of the drag
    of Sangani & Acrivos (1982) and Drummond & Tahir (1984),
    K = (-ln c - 1.476 + 2 c - 1.774 c^2 + 4.076 c^3) / (8 pi)."""
    return (-np.log(c) - 1.476 + 2 * c - 1.774 * c**2 + 4.076 * c**3) / (8 * np.pi)


def test_square_cylinder_array_permeability_2d():
    """One disk of radius 0.2 (c about 0.125) in a plane cell, central symbols:
    within 3% of the array formula at 64^2 and closer than at 32^2 (the grid
    converges towards it: 1.1% at 128^2); no transverse flow."""
    errs = []
    for n in (32, 64):
        H = I.single_cylinder((1, n, n), 0.2)
        R = O.stokes(H, [0.0, 0.0, 1.0], O.StokesParams(eps=1e-9, alpha0=300, beta0=300, b0=300,
                                                        adaptive=False, max_iter=60000, deriv=O.CENTRAL))
        assert R.converged
        errs.append(abs(R.K_col[2] / square_cylinder_array(H.mean()) - 1))
        assert abs(R.K_col[1]) < 1e-12 and abs(R.K_col[0]) < 1e-12
    assert errs[1] < 0.03 and errs[1] < errs[0]


def test_plane_poiseuille_in_a_plane_cell_central_closed_form():
    """A channel in the plane (walls normal to axis 1, flow along axis 2) has
    the discrete profile u_j = h^2 j (m + 1 - j) / 2 of the 3D slab."""
    n, s = 16, 5
    m, h = n - s, 1.0 / n
    H = I.slab((1, n, n), s, normal_axis=1)
    R = O.stokes(H, [0.0, 0.0, 1.0], O.StokesParams(eps=1e-12, alpha0=300, beta0=300, b0=300, adaptive=False,
                                                    max_iter=60000, deriv=O.CENTRAL))
    assert R.converged
    assert R.K_col[2] == pytest.approx(h * h * m * (m + 1) * (m + 2) / (12.0 * n), rel=1e-8)


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------
def test_admm_invariants():
    shape = (8, 8, 8)
    H = I.random_indicator(shape, 0.3, 21)
    Hf = H.astype(float)
    g = np.array([1.0, 0.0, 0.0])
    P1 = O.StokesParams(eps=0, alpha0=200, beta0=100, b0=150, adaptive=False, max_iter=1)
    X1 = O.stokes(H, g, P1).state
    np.testing.assert_allclose(X1.a, Hf * X1.lam, atol=1e-13)        # a = H lambda after step 3
    P = O.StokesParams(eps=1e-11, alpha0=300, beta0=300, b0=300, adaptive=False, max_iter=40000)
    R = O.stokes(H, g, P)
    assert R.converged
    X = R.state
    # force balance: the solid carries the whole body force
    np.testing.assert_allclose((Hf * X.lam).reshape(3, -1).mean(axis=1), g, atol=1e-8)
    # energy identity nu <grad u : grad u> = <u . g> (Parseval with L)
    assert O.energy_form(X.u, O.EXACT) == pytest.approx(R.K_col[0], rel=1e-7)
    # no flow in the solid, divergence free
    assert np.abs(Hf * X.u).max() < 1e-8
    d, _ = O.symbols(shape, O.EXACT)
    assert np.abs(O.spectral_div(X.u, d)).max() < 1e-7


def test_permeability_tensor_symmetries():
    shape = (8, 8, 8)
    H = I.random_indicator(shape, 0.3, 33)
    P = O.StokesParams(eps=1e-11, alpha0=300, beta0=300, b0=300, adaptive=False, max_iter=40000)
    K, Kg, _ = O.permeability_tensor(H, P)
    np.testing.assert_allclose(K, K.T, atol=1e-9 * np.abs(K).max())
    assert np.all(np.linalg.eigvalsh(0.5 * (K + K.T)) > 0)
    # an integer roll of H leaves K unchanged
    K2, _, _ = O.permeability_tensor(np.roll(H, (3, -2, 5), axis=(0, 1, 2)), P)
    np.testing.assert_allclose(K2, K, atol=1e-9 * np.abs(K).max())
    # an axis permutation of H permutes K
    perm = (2, 0, 1)
    K3, _, _ = O.permeability_tensor(np.transpose(H, perm), P)
    np.testing.assert_allclose(K3, K[np.ix_(perm, perm)], atol=1e-9 * np.abs(K).max())
    # a mirror image flips the sign of the off-diagonals that involve the mirrored axis
    Hm = np.roll(H[::-1], 1, axis=0)
    K4, _, _ = O.permeability_tensor(Hm, P)
    S = np.diag([-1.0, 1.0, 1.0])
    np.testing.assert_allclose(K4, S @ K @ S, atol=1e-9 * np.abs(K).max())


def test_centred_sphere_permeability_is_isotropic():
    n = 8
    H = I.single_sphere((n, n, n), 0.3)
    P = O.StokesParams(eps=1e-11, alpha0=300, beta0=300, b0=300, adaptive=False, max_iter=40000,
                       deriv=O.CENTRAL)
    K, _, _ = O.permeability_tensor(H, P)
    k = K[0, 0]
    np.testing.assert_allclose(K, k * np.eye(3), atol=1e-9 * k)


# --------------------------------------------------------------------------
# solute transport (Eq. 16-21)
# --------------------------------------------------------------------------
def test_one_ls_iteration_satisfies_eq17_with_stencils():
    shape = (6, 8, 4)
    H = I.random_indicator(shape, 0.4, 51)
    Hf = H.astype(float)
    u = I.random_field((3,) + shape, 52)
    Pe, eta, A0 = 3.0, 0.05, 0.7
    B0 = np.array([0.3, -0.2, 0.1])
    g = np.array([0.2, 1.0, -0.4])
    R = O.advdiff(H, u, Pe, g, O.AdvDiffParams(eta=eta, A0=A0, B0=B0, eps=0, max_iter=1,
                                                deriv=O.CENTRAL))
    chi1 = R.chi
    A = (1 - Hf) + eta * Hf
    pore = H == 0
    ubar = np.array([u[c][pore].mean() for c in range(3)])
    B = Pe * (1 - Hf)[None] * u
    F = Pe * (1 - Hf) * (ubar @ g)
    e0 = np.broadcast_to(g[:, None, None, None], (3,) + shape)     # grad chi^0 = 0
    F0 = F + DO.div_fd((A - A0)[None] * e0) - np.sum((B - B0[:, None, None, None]) * e0, axis=0)
    lhs = A0 * DO.lap_neg_fd(chi1) + sum(B0[c] * DO.d_fd(chi1, c) for c in range(3))
    rhs = F0 - F0.mean()
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(rhs).max()
    assert abs(chi1.mean()) < 1e-12
    np.testing.assert_allclose(R.grad_chi, DO.grad_fd(chi1), atol=1e-10 * np.abs(R.grad_chi).max())


@pytest.mark.parametrize("shape,seed", [((4, 4, 4), 61), ((6, 4, 6), 62), ((1, 8, 6), 63)])
def test_converged_ls_matches_dense_fixed_point(shape, seed):
    H = I.random_indicator(shape, 0.4, seed)
    u = 0.2 * I.random_field((3,) + shape, seed + 1)
    Pe, eta, A0 = 2.0, 0.1, 0.7
    B0 = np.array([0.1, 0.0, -0.1])
    g = np.array([1.0, 0.3, 0.0])
    R = O.advdiff(H, u, Pe, g, O.AdvDiffParams(eta=eta, A0=A0, B0=B0, eps=1e-14, max_iter=5000,
                                                deriv=O.CENTRAL))
    assert R.converged
    D, Lneg = DO.central_ops(shape)
    chi = DO.advdiff_fixed_point(H, u, Pe, g, D, Lneg, A0, B0, eta)
    np.testing.assert_allclose(R.chi, chi, atol=1e-10 * np.abs(chi).max())


def test_central_ls_fixed_point_depends_on_a0_as_the_dense_solve_says():
    """With the Eq. 21 symbols L != |d|^2, so the converged chi keeps an
    A0 (L - |d|^2) term; two comparison media give two fixed points, each the
    dense stencil solve for its own A0."""
    shape = (6, 4, 6)
    H = I.random_indicator(shape, 0.4, 63)
    u = 0.2 * I.random_field((3,) + shape, 64)
    Pe, eta = 2.0, 0.1
    B0 = np.array([0.1, 0.0, -0.1])
    g = np.array([1.0, 0.3, 0.0])
    D, Lneg = DO.central_ops(shape)
    chis = []
    for A0 in (0.7, 1.3):
        R = O.advdiff(H, u, Pe, g, O.AdvDiffParams(eta=eta, A0=A0, B0=B0, eps=1e-14, max_iter=8000,
                                                    deriv=O.CENTRAL))
        assert R.converged
        ref = DO.advdiff_fixed_point(H, u, Pe, g, D, Lneg, A0, B0, eta)
        np.testing.assert_allclose(R.chi, ref, atol=1e-10 * np.abs(ref).max())
        chis.append(R.chi)
    assert np.abs(chis[0] - chis[1]).max() > 1e-4 * np.abs(chis[0]).max()


@pytest.mark.parametrize("deriv", [O.EXACT, O.CENTRAL])
def test_laminate_diffusivity_parallel_is_pore_fraction(deriv):
    n, s = 16, 6                              # solid layers normal to axis 0
    H = I.laminate((n, 2, 4), s, normal_axis=0)
    phi = 1 - s / n
    u = np.zeros((3,) + H.shape)
    P = O.AdvDiffParams(eta=0.01, A0=0.55, eps=1e-12, max_iter=20000, deriv=deriv)
    for j in (1, 2):                          # g along the layers: chi = 0, D = pore fraction
        R = O.advdiff(H, u, 0.0, np.eye(3)[j], P)
        assert R.converged
        assert R.Dg[j] == pytest.approx(phi, abs=1e-12)
        assert np.abs(R.chi).max() < 1e-12


def test_laminate_diffusivity_series_is_harmonic_mean_exact_symbol():
    """Across two equal layers the flux is the harmonic mean of the diffusivities.

    With the exact symbol and equal layer thicknesses the discrete 1D solution
    reproduces the continuum flux to rounding.
    """
    eta = 0.01
    for n, s in ((8, 4), (16, 8), (32, 16)):
        H = I.laminate((n, 2, 2), s, normal_axis=0)
        phi = 1 - s / n
        u = np.zeros((3,) + H.shape)
        R = O.advdiff(H, u, 0.0, [1.0, 0.0, 0.0],
                      O.AdvDiffParams(eta=eta, A0=0.55, eps=1e-13, max_iter=20000, deriv=O.EXACT))
        assert R.converged
        harm = eta / (phi * eta + 1 - phi)
        assert R.Dg_ext[0] == pytest.approx(harm, rel=1e-9)
        assert R.Dg[0] == pytest.approx(phi * harm, rel=1e-9)     # Eq. 3: pore part of the flux


def test_laminate_diffusivity_series_central_symbol_converges_first_order():
    eta = 0.01
    errs = []
    for n in (16, 32, 64):
        H = I.laminate((n, 2, 2), n // 2, normal_axis=0)
        u = np.zeros((3,) + H.shape)
        R = O.advdiff(H, u, 0.0, [1.0, 0.0, 0.0],
                      O.AdvDiffParams(eta=eta, A0=0.55, eps=1e-12, max_iter=20000, deriv=O.CENTRAL))
        assert R.converged
        errs.append(abs(R.Dg_ext[0] / (eta / (0.5 * eta + 0.5)) - 1))
    assert errs[2] < errs[1] < errs[0]
    assert 1.5 < errs[0] / errs[1] < 3.5 and 1.5 < errs[1] / errs[2] < 3.5


def test_no_solid_no_flow_gives_identity_diffusivity():
    shape = (4, 6, 8)
    H = np.zeros(shape, np.uint8)
    u = np.zeros((3,) + shape)
    D, Dx, res = O.diffusivity_tensor(H, u, 10.0, O.AdvDiffParams(eps=1e-12))
    assert all(r.converged for r in res)
    np.testing.assert_allclose(D, np.eye(3), atol=1e-13)
    assert max(np.abs(r.chi).max() for r in res) < 1e-13


def test_taylor_dispersion_in_plane_poiseuille_flow():
    """Pe term of Eq. 3 and of the iteration: Taylor-Aris dispersion between plates.

    For the plane Poiseuille profile u = y (w - y) / 2 (pore width w, mean w^2/12)
    and g_chi along the flow, the exact cell solution gives
    D_xx = w (1 + (Pe u_mean w)^2 / 210). With the central symbols the discrete
    result converges to it at second order.
    """
    Pe = 300.0
    errs = []
    for n in (16, 32, 64):
        s = n // 4
        H = I.slab((2, n, 2), s, normal_axis=1)
        h = 1.0 / n
        y = (np.arange(n) + 0.5) * h - s * h
        w = 1 - s * h
        u = np.zeros((3,) + H.shape)
        u[0] = np.where(H[0, :, 0] == 0, 0.5 * y * (w - y), 0.0)[None, :, None]
        R = O.advdiff(H, u, Pe, [1.0, 0.0, 0.0],
                      O.AdvDiffParams(eta=1e-3, A0=0.55, eps=1e-12, max_iter=20000, deriv=O.CENTRAL))
        assert R.converged
        D = w * (1 + (Pe * (w * w / 12) * w) ** 2 / 210)
        errs.append(abs(R.Dg[0] / D - 1))
        assert abs(R.Dg[1]) < 1e-10 and abs(R.Dg[2]) < 1e-10
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 2e-3


def test_shear_flow_manufactured_solution_and_dispersion_closed_form():
    """No solid, shear flow u = (0, U sin 2 pi x0, 0) (divergence free, zero
    pore mean), composition gradient e_1. The fixed point of Eq. 17 (with A = 1,
    B = Pe u, F = 0) reduces to chi'' = Pe U sin 2 pi x0, so
    chi = -Pe U sin(2 pi x0) / (2 pi)^2 (a single Fourier mode: exact with the
    exact symbols), and Eq. 3 gives D_11 = 1 + Pe^2 U^2 / (8 pi^2), D_01 = 0."""
    shape = (16, 8, 8)
    n0 = shape[0]
    x0 = (np.arange(n0) + 0.5) / n0
    U, Pe = 1.0, 3.0
    H = np.zeros(shape, dtype=np.uint8)
    u = np.zeros((3,) + shape)
    u[1] = U * np.sin(2 * np.pi * x0)[:, None, None]
    R = O.advdiff(H, u, Pe, [0.0, 1.0, 0.0], O.AdvDiffParams(eps=1e-13, max_iter=20000, deriv=O.EXACT))
    assert R.converged
    chi = -Pe * U * np.sin(2 * np.pi * x0)[:, None, None] / (2 * np.pi) ** 2 * np.ones(shape)
    np.testing.assert_allclose(R.chi, chi, atol=1e-10 * np.abs(chi).max())
    assert R.Dg[1] == pytest.approx(1 + Pe ** 2 * U ** 2 / (8 * np.pi ** 2), rel=1e-10)
    assert abs(R.Dg[0]) < 1e-10 and abs(R.Dg[2]) < 1e-10
