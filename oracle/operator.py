"""The collocation operator A = I + B, matrix-free, float64, a library FFT as DFT.

Test infrastructure only (see the package docstring).

Notation (Section 2): a field ``e`` has shape ``(d, N_0, ..., N_{d-1})``
(component planes, C-order).  ``phase`` is an integer image of shape ``N``;
``L`` is the per-phase tensor table ``(nphase, d, d)``; ``L0`` is the
reference conductivity ``(d, d)``; ``Y`` holds the half side lengths of the
cell ``Y = prod (-Y_a, Y_a)`` (Section 2.1).

The operator follows Eq. (mtrx_B) factor by factor, right to left (the DFT
step is a library FFT, scipy.fft on every host core):

    B e = F^-1 [ Gamma0(k) . F( dL . e ) ]

with ``dL(x) = L(x) - L0`` (Eq. current_decomp), ``F`` / ``F^-1`` the DFT pair
of Eq. (DFT_def) (the |Y|^{+-1/2} factors cancel; numpy's unnormalised forward
/ 1/|N| inverse is the same product) and ``Gamma0`` the Green operator of
Section 2.1:  Gamma0(0) = 0,  Gamma0(k) = xi (x) xi / (xi . L0 . xi).

Readings (the paper leaves these open):
* the frequency of FFT bin ``j`` on an axis of length ``n`` is the signed
  ``k = j`` for ``j <= (n-1)/2`` and ``k = j - n`` otherwise, i.e. the set Z^N
  of Section 2.2 for odd n;
* the wave vector entering Gamma0 is ``xi_a = k_a / Y_a`` (the scaling of the
  basis functions in Eq. fourier_coeff_def); Gamma0 is 0-homogeneous, so for
  a cube cell this is the same as integer k.

Pinned by: the dense assembly of Eq. (mtrx_B) from written-out DFT matrices
(``tests/test_oracle_operator.py``), the projection identities of Gamma0 L0,
and the adjoint identity <A u, v> = <u, A^T v>.
"""
from __future__ import annotations

import os

import numpy as np
from scipy import fft as _fft

# The DFT step runs on every host core (scipy.fft's pocketfft with worker
# threads computes the same unnormalised forward / 1/|N| inverse DFT as
# numpy.fft); ORACLE_FFT_WORKERS caps the thread count.
FFT_WORKERS = int(os.environ.get("ORACLE_FFT_WORKERS", str(os.cpu_count() or 1)))


def fftn(x, axes):
    """Forward DFT of Eq. (DFT_def) over ``axes`` (unnormalised)."""
    return _fft.fftn(x, axes=axes, workers=FFT_WORKERS)


def ifftn(x, axes):
    """Inverse DFT of Eq. (DFT_def) over ``axes`` (with the 1/|N| factor)."""
    return _fft.ifftn(x, axes=axes, workers=FFT_WORKERS)


def signed_frequencies(n: int) -> np.ndarray:
    """Signed frequency of each FFT bin on an axis of length ``n``: the set
    Z^N of Section 2.2, -n/2 < k <= n/2 (for even n the Nyquist bin is +n/2)."""
    j = np.arange(n)
    return np.where(j <= n // 2, j, j - n)


def nyquist_mask(N) -> np.ndarray:
    """True at the frequencies with a Nyquist component (k_a = N_a / 2 on an
    even axis), on the full FFT grid."""
    d = len(N)
    masks = [np.arange(n) == n // 2 if n % 2 == 0 else np.zeros(n, bool) for n in N]
    grids = np.meshgrid(*masks, indexing="ij") if d > 1 else masks
    out = np.zeros(tuple(N), bool)
    for m in grids:
        out |= m
    return out


def reference_medium(L: np.ndarray) -> np.ndarray:
    """Optimal isotropic reference medium of Eq. (opt_ref).

    ``L0 = (lambda_min + lambda_max)/2 I`` where the extremes run over every
    eigenvalue of every phase tensor (the eigenvalues of L(x) over the cell).
    """
    L = np.asarray(L, dtype=np.float64)
    lam = np.concatenate([np.linalg.eigvalsh(0.5 * (Lp + Lp.T)) for Lp in L])
    d = L.shape[-1]
    return 0.5 * (lam.min() + lam.max()) * np.eye(d)


def wave_vectors(N, Y) -> list[np.ndarray]:
    """xi_a = k_a / Y_a on the full frequency grid, one array per axis."""
    d = len(N)
    ks = [signed_frequencies(n).astype(np.float64) / Y[a] for a, n in enumerate(N)]
    return list(np.meshgrid(*ks, indexing="ij")) if d > 1 else ks


def gamma_hat(N, Y, L0) -> np.ndarray:
    """Green operator Gamma0(k) of Section 2.1 on the grid: shape (d, d, *N).

    Gamma0(0) = 0 and Gamma0(k) = xi (x) xi / (xi . L0 . xi) otherwise.
    Reading for an even axis (the paper uses odd grids): Gamma0 is zero at
    every frequency with a Nyquist component.  The collocation operator is
    then real, and its solution is the equilibrium solution on the
    trigonometric polynomials without Nyquist modes (``oracle.dense`` checks
    both characterisations against each other).
    """
    d = len(N)
    xi = wave_vectors(N, Y)
    denom = np.zeros(tuple(N))
    for a in range(d):
        for b in range(d):
            denom += xi[a] * L0[a, b] * xi[b]
    G = np.zeros((d, d) + tuple(N))
    nz = (denom != 0.0) & ~nyquist_mask(N)
    for a in range(d):
        for b in range(d):
            G[a, b][nz] = xi[a][nz] * xi[b][nz] / denom[nz]
    return G


def polarisation(e: np.ndarray, phase: np.ndarray, L: np.ndarray, L0: np.ndarray) -> np.ndarray:
    """tau(x) = dL(x) . e(x) with dL = L(x) - L0 (Eq. current_decomp)."""
    dL = np.asarray(L, dtype=np.float64)[phase] - L0  # (*N, d, d)
    return np.einsum("...ab,b...->a...", dL, e)


def _spatial_axes(e: np.ndarray) -> tuple[int, ...]:
    return tuple(range(1, e.ndim))


def green_apply(t: np.ndarray, N, Y, L0) -> np.ndarray:
    """F^-1 Gamma0 F t: the three leftmost factors of Eq. (mtrx_B)."""
    axes = _spatial_axes(t)
    th = fftn(t, axes=axes)
    G = gamma_hat(N, Y, L0)
    yh = np.einsum("ab...,b...->a...", G, th)
    return np.real(ifftn(yh, axes=axes))


def apply_B(e, phase, L, L0, Y=None) -> np.ndarray:
    """B e = F^-1 Gamma0 F dL e (Eq. mtrx_B)."""
    e = np.asarray(e, dtype=np.float64)
    N = e.shape[1:]
    Y = np.ones(len(N)) if Y is None else np.asarray(Y, dtype=np.float64)
    return green_apply(polarisation(e, phase, L, L0), N, Y, L0)


def apply_A(e, phase, L, L0, Y=None) -> np.ndarray:
    """(I + B) e, the left-hand side of Eq. (linear_system)."""
    e = np.asarray(e, dtype=np.float64)
    return e + apply_B(e, phase, L, L0, Y)


def apply_AT(v, phase, L, L0, Y=None) -> np.ndarray:
    """(I + B^T) v = v + dL . F^-1 Gamma0 F v.

    For odd N the matrix F^-1 Gamma0 F is real and symmetric (Gamma0 is real,
    symmetric and even in k, and Z^N is symmetric under k -> -k), and each dL
    block is symmetric, so B^T is the same factors in reverse order.  BiCG
    needs this product (Section 3).
    """
    v = np.asarray(v, dtype=np.float64)
    N = v.shape[1:]
    Y = np.ones(len(N)) if Y is None else np.asarray(Y, dtype=np.float64)
    return v + polarisation(green_apply(v, N, Y, L0), phase, L, L0)


def macroscopic_field(E, N) -> np.ndarray:
    """The right-hand side e^0 of Eq. (linear_system): E at every node."""
    E = np.asarray(E, dtype=np.float64)
    return np.broadcast_to(E.reshape((-1,) + (1,) * len(N)), (E.size,) + tuple(N)).copy()
