"""Pins for the oracle's collocation operator (CPU only).

Each test ties ``oracle.operator`` to something other than itself:
the dense assembly of Eq. (mtrx_B) from written-out DFT matrices, closed-form
identities of the Green operator (Section 2.1), the homogeneous-medium special
case, the adjoint identity, and the spectrum of I + B.
"""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1004_1122_gb300 import microstructure as micro


def _spd(rng, d, lo=0.5, hi=5.0):
    q, _ = np.linalg.qr(rng.normal(size=(d, d)))
    return q @ np.diag(rng.uniform(lo, hi, size=d)) @ q.T


@pytest.mark.parametrize("N,Y", [((9, 15), (1.0, 2.5)), ((11, 7), (1.0, 1.0)),
                                 ((5, 7, 3), (1.0, 0.5, 2.0)),
                                 ((6, 8), (1.0, 1.5)), ((4, 7), (1.0, 1.0)),   # even axes
                                 ((4, 5, 6), (1.0, 1.0, 0.5))])
@pytest.mark.parametrize("transpose", [False, True])
def test_apply_matches_dense_definition(N, Y, transpose):
    """FFT-based (I+B)e equals the dense product built from Eq. (DFT_def) / (mtrx_B).

    Anisotropic phase tensors and an anisotropic L0 exercise every d x d entry;
    a non-cubic cell exercises xi = k / Y.
    """
    rng = np.random.default_rng(7)
    d = len(N)
    phase = rng.integers(0, 3, size=N).astype(np.uint8)
    L = np.stack([_spd(rng, d) for _ in range(3)])
    L0 = _spd(rng, d, 1.0, 3.0)
    e = rng.normal(size=(d,) + N)
    fast = (oracle.apply_AT if transpose else oracle.apply_A)(e, phase, L, L0, Y)
    ref = dense.apply_dense(e, phase, L, L0, Y, transpose=transpose)
    assert np.max(np.abs(fast - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_dense_dft_pair_is_inverse_and_matches_numpy():
    """The written-out Vandermonde matrices are mutually inverse, and on
    storage-ordered data they reproduce numpy's FFT up to the node phase factor
    of the centred indexing."""
    N, Y = (5, 9), (1.0, 1.0)
    F, Fi = dense.dft_matrices(N, Y)
    assert np.allclose(Fi @ F, np.eye(45), atol=1e-13)
    rng = np.random.default_rng(1)
    x = rng.normal(size=N)
    # centred node m = i - (n-1)/2, centred frequency k ascending
    got = (F @ x.ravel()).reshape(N) * np.prod(2.0 * np.asarray(Y)) ** 0.5
    ref = np.fft.fftshift(np.fft.fftn(x))
    for a, n in enumerate(N):
        k = dense.centred_indices(n)
        shape = [1, 1]
        shape[a] = n
        ref = ref * np.exp(2j * np.pi * k * ((n - 1) // 2) / n).reshape(shape)
    assert np.allclose(got, ref, atol=1e-11)


def test_green_operator_closed_form_identities():
    """Gamma0(k) L0 is the L0-orthogonal projection onto span(xi) (Section 2.1):
    (Gamma0 L0)^2 = Gamma0 L0, Gamma0 L0 xi = xi, Gamma0(0) = 0, Gamma0 symmetric
    and even in k."""
    rng = np.random.default_rng(3)
    N, Y = (7, 9, 5), (1.0, 2.0, 0.75)
    L0 = _spd(rng, 3)
    G = oracle.gamma_hat(N, Y, L0)
    assert np.all(G[:, :, 0, 0, 0] == 0.0)
    ks = np.meshgrid(*[oracle.signed_frequencies(n) / Y[a] for a, n in enumerate(N)],
                     indexing="ij")
    xi = np.stack(ks)
    P = np.einsum("ab...,bc->ac...", G, L0)
    PP = np.einsum("ab...,bc...->ac...", P, P)
    mask = np.ones(N, dtype=bool)
    mask[0, 0, 0] = False
    assert np.allclose(PP[..., mask], P[..., mask], atol=1e-12)
    assert np.allclose(np.einsum("ab...,b...->a...", P, xi)[..., mask], xi[..., mask], atol=1e-12)
    assert np.allclose(G, np.swapaxes(G, 0, 1))
    Gneg = G[:, :, (-np.arange(7)) % 7][:, :, :, (-np.arange(9)) % 9][:, :, :, :, (-np.arange(5)) % 5]
    assert np.allclose(G, Gneg)


def test_signed_frequencies_are_Z_N():
    """FFT bin j maps onto the set -N/2 < k <= N/2 of Section 2.2 exactly once."""
    for n in (3, 9, 81, 135, 255, 2187):
        k = oracle.signed_frequencies(n)
        assert sorted(k.tolist()) == list(range(-(n - 1) // 2, (n - 1) // 2 + 1))
        assert np.all(np.mod(k, n) == np.arange(n))


def test_reference_medium_eq_opt_ref():
    """L0 = (lambda_min + lambda_max)/2 I over all phase eigenvalues (Eq. opt_ref)."""
    L = micro.isotropic_table([1.0, 10.0], 2)
    assert np.allclose(oracle.reference_medium(L), 5.5 * np.eye(2))
    L = np.array([np.diag([2.0, 3.0, 4.0]), np.diag([0.5, 7.0, 1.0])])
    assert np.allclose(oracle.reference_medium(L), 3.75 * np.eye(3))


def test_homogeneous_medium_B_of_constant_is_zero():
    """Constant L: dL e^0 is constant, its spectrum sits at k = 0 where
    Gamma0 vanishes, so B e^0 = 0 and A e^0 = e^0 exactly (up to FFT round-off)."""
    N = (15, 21)
    phase = np.zeros(N, dtype=np.uint8)
    L = np.array([[[3.0, 0.4], [0.4, 2.0]]])
    L0 = 7.0 * np.eye(2)
    e0 = oracle.operator.macroscopic_field([0.3, -1.2], N)
    assert np.max(np.abs(oracle.apply_B(e0, phase, L, L0))) < 1e-14


def test_adjoint_identity():
    """<A u, v> = <u, A^T v> (B^T = dL F^-1 Gamma0 F for odd N)."""
    rng = np.random.default_rng(11)
    phase = micro.rsa_disks(45, 0.3, 3, 6, seed=5)
    L = micro.isotropic_table([1.0, 50.0], 2)
    L0 = oracle.reference_medium(L)
    u, v = rng.normal(size=(2, 2, 45, 45))
    lhs = np.vdot(oracle.apply_A(u, phase, L, L0), v)
    rhs = np.vdot(u, oracle.apply_AT(v, phase, L, L0))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_spectrum_of_I_plus_B():
    """Isotropic L0 = l0 I: I + B has real spectrum in [lambda_min/l0, lambda_max/l0]
    together with the eigenvalue 1 (the constant / incompatible part), so CG
    applies (derived from Eq. (mtrx_B); the paper conjectures it in Section 4)."""
    phase = micro.centred_disk(9, 0.3)
    L = micro.isotropic_table([1.0, 10.0], 2)
    for l0 in (5.5, 2.0, 20.0):
        A = np.eye(162) + dense.assemble_B(phase, L, l0 * np.eye(2))
        ev = np.linalg.eigvals(A)
        assert np.max(np.abs(ev.imag)) < 1e-9
        lo, hi = min(1.0, 1.0 / l0) - 1e-9, max(1.0, 10.0 / l0) + 1e-9
        assert ev.real.min() >= lo and ev.real.max() <= hi
