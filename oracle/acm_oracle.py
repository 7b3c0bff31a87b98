"""Plain FP64 CPU oracle of the ACM method (Karimi & Bhattacharya, arXiv 2312.15554).

TEST INFRASTRUCTURE ONLY. Nothing in the product library imports, links or calls
this module; only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` use it. It shares no code with the CUDA path.

It is a slow, literal restatement of the paper in numpy (double precision,
full complex spectra from the oracle's own radix-2 FFT in `oracle/fft.py`), in
the order and notation of the paper:

* Stokes flow, Section 3.1: ADMM steps 1-4 (Eq. 7-13) with the adaptive
  penalties of Eq. 22, i.e. Problem 1 of Algorithm 1.
* Solute transport, Section 3.2: the Lippmann-Schwinger iteration (Eq. 16-21),
  Problem 2 of Algorithm 1.
* The effective properties of Eq. 2 (permeability) and Eq. 3 (diffusivity),
  and the pore-averaged velocity defined below Eq. 1.

Conventions (unit cube, grid (n0, n1, n2), h_c = 1/n_c, component c of a vector
field is along array axis c):

* forward DFT  f^(m) = sum_x f(x) exp(-2 pi i m.x), unnormalised (oracle/fft.py);
* wavenumber k_c = 2 pi m_c;
* first-derivative symbol d_c (d/dx_c <-> i d_c), Laplacian symbol L (-Laplacian <-> L):
  EXACT    d_c = k_c (0 on the Nyquist plane of axis c), L = |k|^2;
  CENTRAL  d_c = sin(h k_c)/h, L = sum_c 4 sin^2(h k_c / 2)/h^2  (Eq. 21, second
           line read as the compact three-point Laplacian).

Readings where the paper is garbled or silent (each is listed in the design notes):
* Eq. 13: the gradient of q is i d q^ and -beta grad(div u) is +beta d (d.u^).
* The Fourier transform of the constant body force g is g * (number of voxels) at k = 0.
* Tolerances of constraint pairs 2 and 3 follow the pattern Eq. 11-12 give for pair 1.
* Algorithm 1 stops when every constraint pair passes its primal and dual test.
* Norms are plain Euclidean norms over all voxels and components.
* Eq. 22 compares r_p > tau r_d (increase) and r_d > tau r_p (decrease).
* The solute iteration sets chi^(0) = 0 (the mean of chi is free).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from oracle import fft as FFT

EXACT = 0
CENTRAL = 1

_FFT_AX = (1, 2, 3)


# ----------------------------------------------------------------------------
# Spectral symbols (Section 3.1 Eq. 13; Section 3.2 Eq. 21)
# ----------------------------------------------------------------------------
def axis_symbols(n: int, deriv: int):
    """First-derivative and second-derivative symbols on one axis of n points.

    Returns (d, l) with d/dx <-> i*d and -d^2/dx^2 <-> l, for integer
    frequencies m in DFT order (0..n/2-1, -n/2..-1).
    """
    if n == 1:
        # a single plane (two-dimensional cell): the only mode is m = 0
        return np.zeros(1), np.zeros(1)
    if n < 2 or n % 2:
        raise ValueError("axis length must be 1, or even and >= 2")
    h = 1.0 / n
    m = np.concatenate([np.arange(0, n // 2), np.arange(-(n // 2), 0)]).astype(np.float64)
    k = 2.0 * np.pi * m
    if deriv == EXACT:
        d = k.copy()
        d[n // 2] = 0.0          # odd derivative has no real Nyquist mode
        l = k * k
    elif deriv == CENTRAL:
        d = np.sin(h * k) / h                      # Eq. 21, first line
        l = 4.0 * np.sin(0.5 * h * k) ** 2 / h**2  # Eq. 21, second line (compact 3-point)
    else:
        raise ValueError("deriv must be EXACT or CENTRAL")
    return d, l


def symbols(shape, deriv: int):
    """Symbols on the full 3D spectrum: list d[c] (broadcast to shape) and L."""
    d, L = [], np.zeros(tuple(shape))
    for c in range(3):
        dc, lc = axis_symbols(shape[c], deriv)
        bshape = [1, 1, 1]
        bshape[c] = shape[c]
        d.append(np.broadcast_to(dc.reshape(bshape), tuple(shape)))
        L = L + lc.reshape(bshape)
    return d, L


def fft3(f):
    """Forward DFT over the three grid axes (the last three array axes)."""
    return FFT.fftn(f, axes=(-3, -2, -1))


def ifft3(fh):
    """Inverse DFT over the three grid axes; the real part (every field of the method is real)."""
    return FFT.ifftn(fh, axes=(-3, -2, -1)).real


def spectral_grad(f, d):
    """Gradient of a scalar field with symbol d: returns (3, ...) real field."""
    fh = fft3(f)
    return np.stack([ifft3(1j * d[c] * fh) for c in range(3)])


def spectral_div(v, d):
    """Divergence of a vector field with symbol d."""
    vh = fft3(v)
    return ifft3(1j * (d[0] * vh[0] + d[1] * vh[1] + d[2] * vh[2]))


def _norm(x) -> float:
    return float(np.sqrt(np.sum(np.square(x))))


# ----------------------------------------------------------------------------
# Stokes flow: ADMM (Section 3.1, Eq. 5-13, Eq. 22; Algorithm 1 Problem 1)
# ----------------------------------------------------------------------------
@dataclass
class StokesParams:
    nu: float = 1.0
    eps: float = 1e-8
    alpha0: float = 0.0          # 0 selects the default (see default_penalty)
    beta0: float = 0.0
    b0: float = 0.0
    phi: tuple = (1.1, 1.1, 1.1)  # Eq. 22 (Section 4.1)
    tau: tuple = (5.0, 10.0, 5.0)  # Eq. 22, random-geometry values (Section 4.1 footnote)
    psi_min_frac: float = 1e-3
    adaptive: bool = True
    max_iter: int = 20000
    deriv: int = EXACT


def default_penalty(shape, nu: float) -> float:
    """Initial penalty when none is given: nu times the squared wavenumber of the
    geometric mean grid spacing (the stiffness of a voxel-scale mode); the mean
    is taken over the axes longer than one voxel (the plane of a 2D cell)."""
    ax = [n for n in shape if n > 1]
    n = float(np.prod(ax)) ** (1.0 / len(ax))
    return nu * (np.pi * n) ** 2 / 8.0


@dataclass
class StokesState:
    """ADMM state X^n = {u, u~, q, a, lambda} (Section 3.1)."""
    u: np.ndarray
    ut: np.ndarray
    q: np.ndarray
    a: np.ndarray
    lam: np.ndarray


@dataclass
class StokesResult:
    state: StokesState
    p: np.ndarray
    iters: int
    converged: bool
    residuals: np.ndarray      # (iters, 6): r_p1, r_d1, r_p2, r_d2, r_p3, r_d3
    tolerances: np.ndarray     # (iters, 6)
    penalties: np.ndarray      # (iters, 3): alpha, beta, b used in iteration n
    K_col: np.ndarray          # mean_Y(u): K g for nu = 1 (volume-average form of Eq. 2)
    mean_u_hist: np.ndarray = field(default=None)


def zero_state(shape) -> StokesState:
    z3 = np.zeros((3,) + tuple(shape))
    return StokesState(u=z3.copy(), ut=z3.copy(), q=np.zeros(tuple(shape)), a=z3.copy(), lam=z3.copy())


def consistent_pressure(a, d):
    """The pressure q (mean zero) of an ADMM fixed point with multiplier field a.

    At a fixed point of Section 3.1, u = u~ and div u = 0, so the divergence of
    the Step 1 equation (Eq. 7 in Fourier space, Eq. 13) leaves
    |d|^2 q^ = i d . a^ at every k != 0 (the uniform body force has no k != 0
    part); q^ is 0 where |d|^2 = 0. A warm start given u and lambda starts from
    this q with a = H lambda.
    """
    ah = fft3(a)
    dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
    num = 1j * (d[0] * ah[0] + d[1] * ah[1] + d[2] * ah[2])
    qh = np.where(dd > 0, num / np.where(dd > 0, dd, 1.0), 0.0)
    return ifft3(qh)


def warm_state(H, u, lam, deriv=EXACT) -> StokesState:
    """Warm-start state from a velocity and a multiplier: u~ = u, lambda and a
    masked by H, q the consistent pressure of a."""
    Hf = np.asarray(H).astype(np.float64)
    lam = np.asarray(lam, dtype=np.float64) * Hf[None]
    d, _ = symbols(np.asarray(H).shape, deriv)
    u = np.asarray(u, dtype=np.float64)
    return StokesState(u=u.copy(), ut=u.copy(), q=consistent_pressure(lam, d), a=lam.copy(), lam=lam.copy())


def stokes_step1(state: StokesState, g, nu, beta, b, d, L):
    """Step 1 (Eq. 7), solved in Fourier space (Eq. 13).

    Per wavevector: (nu L + b) u^ + beta d (d . u^) = g^ - i d q^ - a^ + b u~^,
    a 3x3 linear system whose matrix is a rank-one update of a multiple of the
    identity, inverted in closed form. Returns u^{n+1} and div u^{n+1} in real space.
    """
    shape = state.q.shape
    V = state.q.size
    ut_h = fft3(state.ut)
    q_h = fft3(state.q)
    a_h = fft3(state.a)
    rhs = np.empty((3,) + shape, dtype=np.complex128)
    for c in range(3):
        rhs[c] = -1j * d[c] * q_h - a_h[c] + b * ut_h[c]
        rhs[c][0, 0, 0] += g[c] * V          # transform of the uniform body force
    # (c I + beta d d^T)^{-1} r = [r - beta d (d.r)/(c + beta |d|^2)] / c,  c = nu L + b
    # (inverse of a rank-one update of a multiple of the identity)
    c0 = nu * L + b
    dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
    dr = d[0] * rhs[0] + d[1] * rhs[1] + d[2] * rhs[2]
    f = beta * dr / (c0 + beta * dd)
    u_h = np.stack([(rhs[c] - d[c] * f) / c0 for c in range(3)])
    u_new = ifft3(u_h)
    div_new = ifft3(1j * (d[0] * u_h[0] + d[1] * u_h[1] + d[2] * u_h[2]))
    return u_new, div_new, u_h


def adapt_penalties(psi, r, phi, tau, psi_min):
    """Eq. 22: the penalties of the next iteration from this iteration's residuals.

    Constraint pair k = 0, 1, 2 (primal r[2k], dual r[2k + 1]) drives psi[k] =
    alpha, beta, b. The penalty grows by phi_k when the primal residual exceeds
    tau_k times the dual one, shrinks by phi_k (not below psi_min[k]) when the
    dual residual exceeds tau_k times the primal one, and stays otherwise. The
    ratios are compared as products (r_p > tau r_d), so a zero residual needs no
    division.
    """
    out = list(psi)
    for k in range(3):
        rp, rd = r[2 * k], r[2 * k + 1]
        if rp > tau[k] * rd:
            out[k] = phi[k] * psi[k]
        elif rd > tau[k] * rp:
            out[k] = max(psi[k] / phi[k], psi_min[k])
    return out


def stokes(H, g, params: StokesParams = None, init: StokesState = None,
           record_mean_u: bool = False) -> StokesResult:
    """Algorithm 1, Problem 1: ADMM for Stokes flow in the periodic cell.

    H: uint8 indicator (1 = solid, Eq. 4). g: body force (the average pressure
    gradient -g_p of Eq. 1 enters as +g). Returns the state after the last
    iteration, the pressure p = q - mean(q), residual/penalty histories and the
    volume average of u.
    """
    P = params or StokesParams()
    H = np.asarray(H)
    shape = H.shape
    V = H.size
    Hf = H.astype(np.float64)
    g = np.asarray(g, dtype=np.float64)
    d, L = symbols(shape, P.deriv)
    st = zero_state(shape) if init is None else StokesState(
        init.u.copy(), init.ut.copy(), init.q.copy(), init.a.copy(), init.lam.copy())
    div_u = spectral_div(st.u, d)
    p0 = default_penalty(shape, P.nu)
    psi = [P.alpha0 or p0, P.beta0 or p0, P.b0 or p0]
    psi_min = [P.psi_min_frac * x for x in psi]
    n1 = n3 = 3 * V
    n2 = V
    eps = P.eps
    res_h, tol_h, pen_h, mu_h = [], [], [], []
    converged = False
    it = 0
    for it in range(1, P.max_iter + 1):
        alpha, beta, b = psi
        pen_h.append((alpha, beta, b))
        # Step 1: stationarity in u (Eq. 7 / Eq. 13)
        u_new, div_new, u_h = stokes_step1(st, g, P.nu, beta, b, d, L)
        if record_mean_u:
            mu_h.append(u_h[:, 0, 0, 0].real / V)
        # Step 2: stationarity in u~, pointwise (Eq. 8)
        ut_new = (b * u_new + st.a - Hf * st.lam) / (b + alpha * Hf)
        # Step 3: multiplier updates (Eq. 9)
        q_new = st.q - beta * div_new
        a_new = st.a + b * (u_new - ut_new)
        lam_new = st.lam + alpha * (Hf * ut_new)
        # Step 4: primal and dual residuals (Eq. 10)
        r = np.array([
            _norm(Hf * ut_new), alpha * _norm(Hf * (ut_new - st.ut)),
            _norm(div_new), beta * _norm(div_new - div_u),
            _norm(u_new - ut_new), b * _norm(u_new - st.u),
        ])
        # tolerances (Eq. 11-12 for pair 1, same pattern for pairs 2 and 3)
        nl, nq, na = _norm(lam_new), _norm(q_new), _norm(a_new)
        tol = np.array([
            np.sqrt(n1) * eps + eps * max(r[0], nl), np.sqrt(n1) * eps + eps * nl,
            np.sqrt(n2) * eps + eps * max(r[2], nq), np.sqrt(n2) * eps + eps * nq,
            np.sqrt(n3) * eps + eps * max(r[4], na), np.sqrt(n3) * eps + eps * na,
        ])
        res_h.append(r)
        tol_h.append(tol)
        st = StokesState(u_new, ut_new, q_new, a_new, lam_new)
        div_u = div_new
        if np.all(r <= tol):
            converged = True
            break
        if P.adaptive:
            psi = adapt_penalties(psi, r, P.phi, P.tau, psi_min)
    p = st.q - st.q.mean()
    return StokesResult(state=st, p=p, iters=it, converged=converged,
                        residuals=np.array(res_h), tolerances=np.array(tol_h),
                        penalties=np.array(pen_h), K_col=st.u.reshape(3, -1).mean(axis=1),
                        mean_u_hist=np.array(mu_h) if record_mean_u else None)


def permeability_tensor(H, params: StokesParams = None, init=None):
    """Three unit loads e_j (Section 2, superposition below Eq. 1).

    Returns (K_mean, K_grad, results): K_mean[i, j] = mean_Y(u^j_i) (volume
    average, nu = 1), K_grad = Eq. 2 over the pore voxels with the spectral
    gradient of the same symbol.
    """
    P = params or StokesParams()
    res = [stokes(H, np.eye(3)[j], P, init) for j in range(3)]
    Km = np.stack([r.K_col for r in res], axis=1)
    Kg = permeability_grad_form(H, [r.state.u for r in res], P.deriv)
    return Km, Kg, res


def permeability_grad_form(H, us, deriv):
    """Eq. 2: K_ij = integral over Y_p of grad u^i : grad u^j (h^3 per voxel)."""
    H = np.asarray(H)
    shape = H.shape
    V = H.size
    d, _ = symbols(shape, deriv)
    pore = (H == 0)
    n = len(us)
    grads = [np.stack([spectral_grad(u[c], d) for c in range(3)]) for u in us]  # (3 comp, 3 dir, ...)
    K = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            K[i, j] = np.sum((grads[i] * grads[j])[:, :, pore]) / V
    return K


def energy_form(u, deriv, nu: float = 1.0):
    """nu * sum_x grad u : grad u / V computed in Fourier space with L (Parseval)."""
    shape = u.shape[1:]
    V = float(np.prod(shape))
    _, L = symbols(shape, deriv)
    uh = fft3(u)
    return nu * float(np.sum(L * np.sum(np.abs(uh) ** 2, axis=0))) / V**2


# ----------------------------------------------------------------------------
# Solute transport: Lippmann-Schwinger (Section 3.2, Eq. 14-21; Algorithm 1 Problem 2)
# ----------------------------------------------------------------------------
@dataclass
class AdvDiffParams:
    eta: float = 0.01            # fictitious solid diffusivity (Section 4.2)
    A0: float = 0.55             # comparison medium (Section 4.2)
    B0: tuple = None             # None: mean over Y of B (see advdiff)
    eps: float = 1e-8
    max_iter: int = 20000
    deriv: int = CENTRAL         # Eq. 21 filter is the solute default


@dataclass
class AdvDiffResult:
    chi: np.ndarray
    grad_chi: np.ndarray
    iters: int
    converged: bool
    residuals: np.ndarray        # (iters, 2): r1, r2
    Dg: np.ndarray               # D g_chi (Eq. 3)
    Dg_ext: np.ndarray           # extended-domain average of A (g + grad chi) + Pe term
    ubar: np.ndarray
    B0: np.ndarray


def pore_average(H, u):
    """u-bar = (1/|Y_p|) integral over Y_p of u (definition below Eq. 1)."""
    pore = (np.asarray(H) == 0)
    return np.array([u[c][pore].mean() for c in range(3)])


def advdiff(H, u, Pe: float, g_chi, params: AdvDiffParams = None) -> AdvDiffResult:
    """Algorithm 1, Problem 2 for one composition gradient g_chi and one velocity u."""
    P = params or AdvDiffParams()
    H = np.asarray(H)
    shape = H.shape
    V = H.size
    Hf = H.astype(np.float64)
    g = np.asarray(g_chi, dtype=np.float64)
    d, L = symbols(shape, P.deriv)
    # coefficients of the penalised equation (Eq. 14) in the form of Eq. 16
    A = (1.0 - Hf) + P.eta * Hf
    ubar = pore_average(H, u)
    B = Pe * (1.0 - Hf)[None] * u
    Fsrc = Pe * (1.0 - Hf) * float(ubar @ g)
    B0 = np.array([B[c].mean() for c in range(3)]) if P.B0 is None else np.asarray(P.B0, float)
    A0 = P.A0
    g_h = np.zeros((3,) + shape, dtype=np.complex128)
    for c in range(3):
        g_h[c][0, 0, 0] = g[c] * V                           # transform of a uniform field
    denom = 1j * (B0[0] * d[0] + B0[1] * d[1] + B0[2] * d[2]) + A0 * L
    k0 = np.zeros(shape, dtype=bool)
    k0[0, 0, 0] = True
    chi = np.zeros(shape)
    grad = np.zeros((3,) + shape)
    res_h = []
    converged = False
    tol1 = np.sqrt(V) * P.eps
    tol2 = np.sqrt(3 * V) * P.eps
    it = 0
    for it in range(1, P.max_iter + 1):
        # Step 1: residual F^n in real space (Eq. 18)
        e = grad + g[:, None, None, None]
        tau = (A - A0)[None] * e
        Fn = Fsrc + spectral_div(tau, d) - np.sum((B - B0[:, None, None, None]) * e, axis=0)
        # Step 2: solve Eq. 17 in Fourier space (Eq. 20); the k = 0 mode of chi is 0
        F_h = fft3(Fn)
        num = F_h - (B0[0] * g_h[0] + B0[1] * g_h[1] + B0[2] * g_h[2])
        chi_h = np.where(k0, 0.0, num / np.where(k0, 1.0, denom))
        chi_new = ifft3(chi_h)
        grad_new = np.stack([ifft3(1j * d[c] * chi_h) for c in range(3)])
        # Step 3: convergence (Eq. 19)
        r1 = _norm(chi_new - chi)
        r2 = _norm(grad_new - grad)
        res_h.append((r1, r2))
        chi, grad = chi_new, grad_new
        if r1 <= tol1 and r2 <= tol2:
            converged = True
            break
    Dg, Dg_ext = diffusivity_column(H, u, Pe, g, chi, grad, ubar, P.eta)
    return AdvDiffResult(chi=chi, grad_chi=grad, iters=it, converged=converged,
                         residuals=np.array(res_h), Dg=Dg, Dg_ext=Dg_ext, ubar=ubar, B0=B0)


def diffusivity_column(H, u, Pe, g, chi, grad, ubar, eta):
    """Eq. 3 contracted with g: (D g)_i = (1/V) sum over pore of [g_i + Pe (ubar - u)_i chi + d_i chi].

    Also the extended-domain form (1/V) sum over Y of A (g + grad chi)_i plus the same Pe term.
    """
    H = np.asarray(H)
    V = H.size
    pore = (H == 0)
    Hf = H.astype(np.float64)
    A = (1.0 - Hf) + eta * Hf
    Dg = np.zeros(3)
    Dx = np.zeros(3)
    for i in range(3):
        pe_term = Pe * np.sum(((ubar[i] - u[i]) * chi)[pore])
        Dg[i] = (g[i] * np.count_nonzero(pore) + pe_term + np.sum(grad[i][pore])) / V
        Dx[i] = (np.sum(A * (g[i] + grad[i])) + pe_term) / V
    return Dg, Dx


def diffusivity_tensor(H, u, Pe, params: AdvDiffParams = None):
    """D_ij for the three composition loads g_chi = e_j (columns), one velocity field u."""
    res = [advdiff(H, u, Pe, np.eye(3)[j], params) for j in range(3)]
    return np.stack([r.Dg for r in res], axis=1), np.stack([r.Dg_ext for r in res], axis=1), res
