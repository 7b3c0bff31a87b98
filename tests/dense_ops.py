"""Dense finite-difference / explicit-DFT operators for pinning the oracle.

These are independent of numpy.fft: the CENTRAL operators are the stencils
that the Eq. 21 symbols stand for (periodic shifts), and the EXACT operators
are built from explicit DFT matrices exp(-2 pi i m j / n).
"""
import numpy as np


def lap_neg_fd(f, shape=None):
    """-Laplacian, compact three-point stencil per axis (unit cube, h_c = 1/n_c)."""
    out = np.zeros_like(f)
    for c in range(3):
        h = 1.0 / f.shape[c]
        out -= (np.roll(f, -1, axis=c) + np.roll(f, 1, axis=c) - 2.0 * f) / h**2
    return out


def d_fd(f, c):
    """Central first difference along axis c: (f(x + h e_c) - f(x - h e_c)) / 2h."""
    h = 1.0 / f.shape[c]
    return (np.roll(f, -1, axis=c) - np.roll(f, 1, axis=c)) / (2.0 * h)


def grad_fd(f):
    return np.stack([d_fd(f, c) for c in range(3)])


def div_fd(v):
    return d_fd(v[0], 0) + d_fd(v[1], 1) + d_fd(v[2], 2)


def op_matrix(fun, shape):
    """Dense matrix of a linear map on scalar fields of the given shape."""
    V = int(np.prod(shape))
    M = np.zeros((V, V))
    for i in range(V):
        e = np.zeros(V)
        e[i] = 1.0
        M[:, i] = fun(e.reshape(shape)).ravel()
    return M


def dft_matrix(n):
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n)


def exact_ops(shape):
    """Dense EXACT-symbol operators (D_0, D_1, D_2, -Laplacian) from explicit DFT matrices."""
    F = np.kron(np.kron(dft_matrix(shape[0]), dft_matrix(shape[1])), dft_matrix(shape[2]))
    Finv = np.conj(F).T / F.shape[0]
    ms = []
    for c, n in enumerate(shape):
        m = np.arange(n).astype(float)
        m[m > n / 2] -= n
        ms.append(m)
    M0, M1, M2 = np.meshgrid(ms[0], ms[1], ms[2], indexing="ij")
    D = []
    for c, Mc in enumerate((M0, M1, M2)):
        n = shape[c]
        k = 2 * np.pi * Mc.ravel()
        dk = np.where(np.abs(Mc.ravel()) == n / 2, 0.0, k)
        D.append((Finv @ np.diag(1j * dk) @ F).real)
    L = (2 * np.pi) ** 2 * (M0**2 + M1**2 + M2**2).ravel()
    Lneg = (Finv @ np.diag(L) @ F).real
    return D, Lneg


def central_ops(shape):
    D = [op_matrix(lambda f, c=c: d_fd(f, c), shape) for c in range(3)]
    Lneg = op_matrix(lap_neg_fd, shape)
    return D, Lneg


def stokes_kkt(H, g, D, Lneg, nu=1.0):
    """Solve nu L u + D q + H lambda = g, D.u = 0, u = 0 on solid (dense least squares)."""
    V = H.size
    solid = np.flatnonzero(H.ravel())
    ns = solid.size
    S = np.zeros((ns, V))
    S[np.arange(ns), solid] = 1.0
    nu_ = 3 * V + V + 3 * ns
    rows = []
    rhs = []
    for c in range(3):
        r = np.zeros((V, nu_))
        r[:, c * V:(c + 1) * V] = nu * Lneg
        r[:, 3 * V:4 * V] = D[c]
        r[:, 4 * V + c * ns:4 * V + (c + 1) * ns] = S.T
        rows.append(r)
        rhs.append(np.full(V, g[c]))
    r = np.zeros((V, nu_))
    for c in range(3):
        r[:, c * V:(c + 1) * V] = D[c]
    rows.append(r)
    rhs.append(np.zeros(V))
    for c in range(3):
        r = np.zeros((ns, nu_))
        r[:, c * V:(c + 1) * V] = S
        rows.append(r)
        rhs.append(np.zeros(ns))
    A = np.vstack(rows)
    b = np.concatenate(rhs)
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    return x[:3 * V].reshape((3,) + H.shape)


def advdiff_fixed_point(H, u, Pe, g, D, Lneg, A0, B0, eta):
    """Dense solve of the Lippmann-Schwinger fixed point (Eq. 16 with the k = 0 row removed).

    A0 Lneg chi + B0.D chi = P[ F + D.((A - A0)(D chi + g)) - (B - B0).(D chi + g) ],  mean(chi) = 0,
    P = removal of the mean.
    """
    V = H.size
    Hf = H.ravel().astype(float)
    A = (1 - Hf) + eta * Hf
    pore = Hf == 0
    ubar = np.array([u[c].ravel()[pore].mean() for c in range(3)])
    B = [Pe * (1 - Hf) * u[c].ravel() for c in range(3)]
    F = Pe * (1 - Hf) * (ubar @ g)
    P = np.eye(V) - np.full((V, V), 1.0 / V)
    M = A0 * Lneg + sum(B0[c] * D[c] for c in range(3))
    M = M - P @ sum(D[c] @ np.diag(A - A0) @ D[c] for c in range(3))
    M = M + P @ sum(np.diag(B[c] - B0[c]) @ D[c] for c in range(3))
    rhs = F + sum(D[c] @ ((A - A0) * g[c]) for c in range(3)) - sum((B[c] - B0[c]) * g[c] for c in range(3))
    rhs = P @ rhs
    Ab = np.vstack([M, np.full((1, V), 1.0 / V)])
    bb = np.concatenate([rhs, [0.0]])
    chi = np.linalg.lstsq(Ab, bb, rcond=None)[0]
    return chi.reshape(H.shape)
