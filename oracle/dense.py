"""Tier 1 of the oracle: the collocation system written out as dense matrices.

Test infrastructure only (see the package docstring).  Tiny grids only
(2-D N <= 27, 3-D N <= 9): memory is O((d |N|)^2).

Two independent formulations of the same discrete problem:

1. ``assemble_A`` / ``solve_lu``: Eq. (mtrx_B) assembled factor by factor from
   the Vandermonde matrices of Eq. (DFT_def).  Nodes use the paper's centred
   indices m in Z^N and frequencies k in Z^N enumerated from their definition
   (-N/2 < k <= N/2, ascending), not FFT bin order, and the Green operator is
   evaluated from its closed form at those k.  ``I + B`` is then solved by
   LU with partial pivoting (LAPACK ``gesv``).

2. ``solve_potential``: no reference medium, no Green operator.  The field is
   written as ``e = E + D phi`` where ``D_a = F^-1 diag(i xi_a) F`` is the
   trigonometric gradient (curl-free by construction, zero mean), and the
   nodal current ``j = L e`` is made divergence-free in the same spectral
   sense, ``D^T j = 0`` (Eq. problem_def_1 in collocation form).  That is the
   symmetric positive semi-definite system ``D^T L D phi = -D^T L E``; the
   constant null space is removed by adding ``1 1^T / |N|`` and it is solved by
   Cholesky.

The collocation solution satisfies both characterisations (for k != 0
Eq. (LS_Fourier) gives ``e^(k)`` parallel to xi and ``xi . j^(k) = 0``), and
``I + B`` is nonsingular, so the two must agree to round-off.  That agreement
pins the Green operator and the operator assembly against an L0-free
formulation.

Storage order equals centred order: storage index i holds the node with
centred index m = i + min Z^N, and ``centred_indices`` lists m ascending, so a
flattened storage-order field is already in centred order; only the centred m
enters the DFT exponent (a constant shift of the node indices commutes with
the operator).

Even axes (the paper's grids are odd): the Green operator and the gradient
leave out the frequencies with a Nyquist component, the reading under which
both formulations are real and agree.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def centred_indices(n: int) -> np.ndarray:
    """The index set Z^N of Section 2.2 for one axis, ascending: -N/2 < k <= N/2."""
    lo = -(n // 2) + (1 if n % 2 == 0 else 0)
    return np.arange(lo, n // 2 + 1)


def dft_matrices(N, Y):
    """Forward and inverse Vandermonde matrices of Eq. (DFT_def), multi-index.

    F^{k m} = |Y|^{-1/2} exp(-2 pi i sum_a k_a m_a / N_a)
    (F^-1)^{k m} = |Y|^{1/2} |N|^{-1} exp(+2 pi i sum_a k_a m_a / N_a)

    Rows/columns follow C-order over the centred indices of each axis.  The
    exponential of a sum over axes is the Kronecker product of per-axis
    matrices.
    """
    vol = float(np.prod(2.0 * np.asarray(Y, dtype=np.float64)))
    size = int(np.prod(N))
    F = np.ones((1, 1), dtype=np.complex128)
    Fi = np.ones((1, 1), dtype=np.complex128)
    for n in N:
        k = centred_indices(n)
        ph = 2.0 * np.pi * np.outer(k, k) / n
        F = np.kron(F, np.exp(-1j * ph))
        Fi = np.kron(Fi, np.exp(1j * ph))
    return vol ** -0.5 * F, vol ** 0.5 / size * Fi


def _frequency_grid(N, Y):
    """xi_a = k_a / Y_a for every k in Z^N (C-order), shape (d, |N|)."""
    ks = np.meshgrid(*[centred_indices(n) for n in N], indexing="ij")
    return np.stack([k.ravel().astype(np.float64) / Y[a] for a, k in enumerate(ks)])


def _nyquist(N):
    """True for the k in Z^N (C-order) with a component k_a = N_a / 2 on an even axis."""
    ks = np.meshgrid(*[centred_indices(n) for n in N], indexing="ij")
    out = np.zeros(int(np.prod(N)), bool)
    for a, n in enumerate(N):
        if n % 2 == 0:
            out |= ks[a].ravel() == n // 2
    return out


def assemble_B(phase, L, L0, Y=None) -> np.ndarray:
    """Dense real matrix B of Eq. (mtrx_B) in centred node order, (d|N|, d|N|).

    B = diag(F^-1) [Gamma0_ab] diag(F) [dL_ab], each bracket a d x d array of
    |N| x |N| diagonal blocks (Gamma0 over frequencies, dL over nodes).
    """
    phase = np.asarray(phase)
    N = phase.shape
    d = len(N)
    Y = np.ones(d) if Y is None else np.asarray(Y, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    L0 = np.asarray(L0, dtype=np.float64)
    size = int(np.prod(N))
    F, Fi = dft_matrices(N, Y)

    xi = _frequency_grid(N, Y)
    q = np.einsum("ak,ab,bk->k", xi, L0, xi)
    G = np.zeros((d * size, d * size), dtype=np.complex128)
    nz = (q != 0.0) & ~_nyquist(N)  # even axes: no Nyquist modes (see oracle.operator.gamma_hat)
    for a in range(d):
        for b in range(d):
            g = np.zeros(size)
            g[nz] = xi[a, nz] * xi[b, nz] / q[nz]
            G[a * size:(a + 1) * size, b * size:(b + 1) * size] = np.diag(g)

    ph = phase.ravel()
    dL = L[ph] - L0  # (|N|, d, d)
    DL = np.zeros((d * size, d * size))
    for a in range(d):
        for b in range(d):
            DL[a * size:(a + 1) * size, b * size:(b + 1) * size] = np.diag(dL[:, a, b])

    Fd = scipy.linalg.block_diag(*([F] * d))
    Fid = scipy.linalg.block_diag(*([Fi] * d))
    B = Fid @ G @ Fd @ DL
    if np.max(np.abs(B.imag)) > 1e-9 * max(1.0, np.max(np.abs(B.real))):
        raise ValueError("B is not real: non-symmetric frequency set")
    return B.real


def apply_dense(e, phase, L, L0, Y=None, transpose: bool = False) -> np.ndarray:
    """(I + B) e (or (I + B^T) e) through the dense matrix, storage-order field."""
    e = np.asarray(e, dtype=np.float64)
    B = assemble_B(phase, L, L0, Y)
    ev = e.ravel()
    out = ev + (B.T @ ev if transpose else B @ ev)
    return out.reshape(e.shape)


def solve_lu(phase, L, L0, E, Y=None) -> np.ndarray:
    """Solve Eq. (linear_system) (I + B) e = e^0 by dense LU; storage-order field."""
    phase = np.asarray(phase)
    N = phase.shape
    d = len(N)
    size = int(np.prod(N))
    B = assemble_B(phase, L, L0, Y)
    rhs = np.repeat(np.asarray(E, dtype=np.float64), size)
    e = np.linalg.solve(np.eye(d * size) + B, rhs)
    return e.reshape((d,) + tuple(N))


def solve_potential(phase, L, E, Y=None) -> np.ndarray:
    """Equilibrium form: e = E + D phi with D^T L (E + D phi) = 0 (see module doc)."""
    phase = np.asarray(phase)
    N = phase.shape
    d = len(N)
    Y = np.ones(d) if Y is None else np.asarray(Y, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    size = int(np.prod(N))
    F, Fi = dft_matrices(N, Y)
    xi = _frequency_grid(N, Y)
    nyq = _nyquist(N)
    D = []
    for a in range(d):
        # the trigonometric gradient on the modes without a Nyquist component
        Da = Fi @ np.diag(1j * xi[a] * ~nyq) @ F
        if np.max(np.abs(Da.imag)) > 1e-9 * max(1.0, np.max(np.abs(Da.real))):
            raise ValueError("gradient is not real")
        D.append(Da.real)
    Dst = np.vstack(D)  # (d|N|, |N|)
    ph = phase.ravel()
    Ln = L[ph]
    Lmat = np.zeros((d * size, d * size))
    for a in range(d):
        for b in range(d):
            Lmat[a * size:(a + 1) * size, b * size:(b + 1) * size] = np.diag(Ln[:, a, b])
    Efield = np.repeat(np.asarray(E, dtype=np.float64), size)
    # null space of D: the constant and (even axes) the Nyquist modes; add the
    # orthogonal projector onto it, built from the inverse-DFT columns
    null = np.nonzero(nyq | (np.abs(xi).sum(axis=0) == 0.0))[0]
    P = np.zeros((size, size))
    for j in null:
        v = Fi[:, j] / np.linalg.norm(Fi[:, j])
        P += np.outer(v, v.conj()).real
    K = Dst.T @ Lmat @ Dst + P
    rhs = -Dst.T @ (Lmat @ Efield)
    phi = scipy.linalg.cho_solve(scipy.linalg.cho_factor(K), rhs)
    e = Efield + Dst @ phi
    return e.reshape((d,) + tuple(N))
