"""Iterative solvers and derived quantities, float64, plain numpy.

Test infrastructure only (see the package docstring).

* ``cg``          conjugate gradients in the order of Saad, Alg. 6.18, applied
                  to the non-symmetric system Eq. (linear_system) (Section 2.3).
* ``bicg``        biconjugate gradients in the order of Saad, Alg. 7.3, with
                  products by A and A^T (Section 3).
* ``fixed_point`` the FFTH / Moulinec-Suquet Neumann series Eq. (orig_fft),
                  e^(m+1) = e^0 - B e^(m), started from e^0.
* ``eta_e``       the equilibrium norm of Eq. (errE_def).
* ``effective_tensor``  L_eff[:, b] = <L e^(b)> (nodal mean), load b = unit E_b.

Readings of points the paper leaves open:

* Stopping: every solver stops when the relative residual
  ||e^0 - A e^(m)||_2 / ||e^0||_2 <= tol.  For CG/BiCG this is the recursively
  updated residual; the returned ``rel_res_true`` is recomputed from scratch.
  For the fixed point the residual of iterate m is e^(m+1) - e^(m), so the test
  is the printed Eq. (errR_def) divided by the reference conductivity.
* ``eta_r`` in the returned info is Eq. (errR_def) as printed:
  ||L0 (e^(m+1) - e^(m))||_2 / ||e^0||_2, where for CG/BiCG the increment
  e^(m+1) - e^(m) is alpha p; ``eta_r_history[m]`` holds it for every step m.
* The initial guess is e = E (x0 = e^0) unless one is passed.
* BiCG's shadow residual is r0* = r0.
* Breakdown ((A p, p) <= 0 for CG, a zero denominator for BiCG, or a
  non-finite scalar) stops the solver with status "breakdown"; reaching the
  iteration cap returns status "not_converged".

Pinned by: the homogeneous and laminate closed forms, agreement with the
dense LU and with the potential formulation (``oracle.dense``), the rate
bounds of Eq. (conv_rate), CG == BiCG iterates (Section 3.1), and
Voigt/Reuss ordering of the effective tensor (``tests/test_oracle_solvers.py``).
"""
from __future__ import annotations

import numpy as np

from .operator import apply_A, apply_AT, fftn, macroscopic_field, nyquist_mask, signed_frequencies


def _dot(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.vdot(a.ravel(), b.ravel()))


def _setup(phase, L, L0, E, Y):
    phase = np.asarray(phase)
    N = phase.shape
    L = np.asarray(L, dtype=np.float64)
    L0 = np.asarray(L0, dtype=np.float64)
    Y = np.ones(len(N)) if Y is None else np.asarray(Y, dtype=np.float64)
    b = macroscopic_field(E, N)
    return phase, N, L, L0, Y, b


def _info(status, iters, hist, res_true, eta_r, matvecs, eta_hist):
    return {
        "status": status,
        "iters": iters,
        "history": np.asarray(hist),
        "rel_res_true": res_true,
        "eta_r": eta_r,
        "eta_r_history": np.asarray(eta_hist),
        "matvecs": matvecs,
    }


def cg(phase, L, L0, E, tol=1e-8, max_iter=10000, Y=None, x0=None):
    """Conjugate gradients, Saad Alg. 6.18, on (I + B) e = e^0.

    r0 = b - A x0, p0 = r0; for j = 0, 1, ...:
      alpha = (r_j, r_j) / (A p_j, p_j);  x += alpha p_j;  r_(j+1) = r_j - alpha A p_j;
      beta = (r_(j+1), r_(j+1)) / (r_j, r_j);  p_(j+1) = r_(j+1) + beta p_j.
    Returns (e, info); ``info['history']`` holds the relative recursive
    residual after each iteration, starting with the initial one.
    """
    phase, N, L, L0, Y, b = _setup(phase, L, L0, E, Y)
    x = b.copy() if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    r = b - apply_A(x, phase, L, L0, Y)
    nb = np.sqrt(_dot(b, b))
    p = r.copy()
    rr = _dot(r, r)
    hist = [np.sqrt(rr) / nb]
    eta_hist = []
    status, it, eta_r, mv = "not_converged", 0, np.nan, 1
    if hist[-1] <= tol:
        status = "converged"
    else:
        for it in range(1, max_iter + 1):
            Ap = apply_A(p, phase, L, L0, Y)
            mv += 1
            pAp = _dot(Ap, p)
            if not np.isfinite(pAp) or pAp <= 0.0:
                status = "breakdown"
                break
            alpha = rr / pAp
            x += alpha * p
            r -= alpha * Ap
            eta_r = np.linalg.norm(np.einsum("ab,b...->a...", L0, alpha * p)) / nb
            eta_hist.append(eta_r)
            rr_new = _dot(r, r)
            hist.append(np.sqrt(rr_new) / nb)
            if not np.isfinite(rr_new):
                status = "breakdown"
                break
            if hist[-1] <= tol:
                status = "converged"
                break
            beta = rr_new / rr
            rr = rr_new
            p = r + beta * p
    res = b - apply_A(x, phase, L, L0, Y)
    return x, _info(status, len(hist) - 1, hist, np.sqrt(_dot(res, res)) / nb, eta_r, mv + 1, eta_hist)


def bicg(phase, L, L0, E, tol=1e-8, max_iter=10000, Y=None, x0=None, record=None):
    """Biconjugate gradients, Saad Alg. 7.3, with shadow residual r0* = r0.

    ``record``, if a list, receives a copy of (r_j, r*_j) for every j.

    alpha = (r_j, r*_j) / (A p_j, p*_j);  x += alpha p_j;
    r_(j+1) = r_j - alpha A p_j;  r*_(j+1) = r*_j - alpha A^T p*_j;
    beta = (r_(j+1), r*_(j+1)) / (r_j, r*_j);
    p_(j+1) = r_(j+1) + beta p_j;  p*_(j+1) = r*_(j+1) + beta p*_j.
    """
    phase, N, L, L0, Y, b = _setup(phase, L, L0, E, Y)
    x = b.copy() if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    r = b - apply_A(x, phase, L, L0, Y)
    nb = np.sqrt(_dot(b, b))
    rs = r.copy()
    p, ps = r.copy(), rs.copy()
    rho = _dot(r, rs)
    hist = [np.sqrt(_dot(r, r)) / nb]
    if record is not None:
        record.append((r.copy(), rs.copy()))
    eta_hist = []
    status, it, eta_r, mv = "not_converged", 0, np.nan, 1
    if hist[-1] <= tol:
        status = "converged"
    else:
        for it in range(1, max_iter + 1):
            Ap = apply_A(p, phase, L, L0, Y)
            ATps = apply_AT(ps, phase, L, L0, Y)
            mv += 2
            den = _dot(Ap, ps)
            if not np.isfinite(den) or den == 0.0:
                status = "breakdown"
                break
            alpha = rho / den
            x += alpha * p
            r -= alpha * Ap
            rs -= alpha * ATps
            if record is not None:
                record.append((r.copy(), rs.copy()))
            eta_r = np.linalg.norm(np.einsum("ab,b...->a...", L0, alpha * p)) / nb
            eta_hist.append(eta_r)
            hist.append(np.sqrt(_dot(r, r)) / nb)
            if hist[-1] <= tol:
                status = "converged"
                break
            rho_new = _dot(r, rs)
            if not np.isfinite(rho_new) or rho_new == 0.0:
                status = "breakdown"
                break
            beta = rho_new / rho
            rho = rho_new
            p = r + beta * p
            ps = rs + beta * ps
    res = b - apply_A(x, phase, L, L0, Y)
    return x, _info(status, len(hist) - 1, hist, np.sqrt(_dot(res, res)) / nb, eta_r, mv + 1, eta_hist)


def fixed_point(phase, L, L0, E, tol=1e-8, max_iter=100000, Y=None, x0=None):
    """FFTH Neumann iteration Eq. (orig_fft): e^(m+1) = e^0 - B e^(m), e^(0) = e^0.

    Written as e^(m+1) = e^(m) + r^(m) with r^(m) = e^0 - A e^(m), which is the
    same recurrence; the residual of iterate m is its increment.  Returns the
    last iterate e^(m+1) once ||r^(m)|| / ||e^0|| <= tol.
    """
    phase, N, L, L0, Y, b = _setup(phase, L, L0, E, Y)
    e = b.copy() if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    nb = np.sqrt(_dot(b, b))
    hist = []
    eta_hist = []
    status, it, eta_r = "not_converged", 0, np.nan
    for it in range(0, max_iter + 1):
        r = b - apply_A(e, phase, L, L0, Y)
        rel = np.sqrt(_dot(r, r)) / nb
        hist.append(rel)
        eta_r = np.linalg.norm(np.einsum("ab,b...->a...", L0, r)) / nb
        eta_hist.append(eta_r)
        if not np.isfinite(rel):
            status = "breakdown"
            break
        e = e + r
        if rel <= tol:
            status = "converged"
            break
    res = b - apply_A(e, phase, L, L0, Y)
    return e, _info(status, it, hist, np.sqrt(_dot(res, res)) / nb, eta_r, it + 2, eta_hist)


def solve(phase, L, L0, E, method="cg", tol=1e-8, max_iter=10000, Y=None, x0=None):
    """Dispatch to ``cg``, ``bicg`` or ``fixed_point``."""
    fn = {"cg": cg, "bicg": bicg, "fixed_point": fixed_point, "ffth": fixed_point}[method]
    return fn(phase, L, L0, E, tol=tol, max_iter=max_iter, Y=Y, x0=x0)


def current(e, phase, L) -> np.ndarray:
    """Nodal current j(x) = L(x) e(x) (Eq. problem_def_1)."""
    return np.einsum("...ab,b...->a...", np.asarray(L, dtype=np.float64)[np.asarray(phase)], e)


def effective_tensor(fields, phase, L) -> np.ndarray:
    """L_eff[:, b] = nodal mean of L(x) e^(b)(x), one solved field per unit load.

    The paper does not define the effective tensor in formulas; this is the
    macroscopic current <j> = L_eff E over the nodes (k = 0 Fourier
    coefficient up to normalisation), load b = e_b giving column b.
    """
    cols = [current(e, phase, L).reshape(len(fields[0]), -1).mean(axis=1) for e in fields]
    return np.stack(cols, axis=1)


def eta_e(e, phase, L, Y=None) -> float:
    """Equilibrium norm of Eq. (errE_def).

    eta_e^2 = sum_k |xi . j^(k)|^2 / |j^(0)|_2^2 with j = L e, xi_a = k_a / Y_a
    over every k in Z^N (k = 0 contributes zero); the DFT normalisation cancels.
    On an even axis the frequencies with a Nyquist component are left out
    (the reading of ``oracle.operator.gamma_hat``: equilibrium is not imposed
    there).
    """
    e = np.asarray(e, dtype=np.float64)
    N = e.shape[1:]
    Y = np.ones(len(N)) if Y is None else np.asarray(Y, dtype=np.float64)
    jh = fftn(current(e, phase, L), axes=tuple(range(1, e.ndim)))
    ks = np.meshgrid(*[signed_frequencies(n) / Y[a] for a, n in enumerate(N)], indexing="ij")
    div = sum(ks[a] * jh[a] for a in range(len(N)))
    div = np.where(nyquist_mask(N), 0.0, div)
    j0 = jh[(slice(None),) + (0,) * len(N)]
    return float(np.sqrt(np.sum(np.abs(div) ** 2) / np.sum(np.abs(j0) ** 2)))
