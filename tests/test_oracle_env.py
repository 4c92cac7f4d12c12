"""Pin of the oracle's environment square roots (Sec. 2.5 step 1, Fig. 1
step 1: sqrt(M) absorbed, M^{-1/2} in the deabsorb) and of their
pseudo-inverse cut: eigenvalues below pinv_rel times the largest are treated
as zero.

The messages are built by hand from a known spectrum in a random orthonormal
basis, so every expected value is the spectrum itself: the square root
squares back to M with the cut eigenvalues removed, the inverse root times
the root is the projector onto the kept eigenvectors, the cut is relative
(invariant under scaling M), negative rounding eigenvalues count as zero,
and the Hermitian part is what is factored (Eq. 13 messages are Hermitian;
an antisymmetric rounding part is dropped).
"""
import numpy as np

from oracle.pepo import env_sqrt


def basis(n, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return q


def message(eigs, seed=0):
    V = basis(len(eigs), seed)
    return (V * np.asarray(eigs, dtype=float)) @ V.T, V


def test_full_rank_root_and_inverse_root():
    M, V = message([1.0, 0.3, 2e-3, 5e-7])
    S, Si = env_sqrt(M, 1e-12)
    assert np.allclose(S @ S, M, atol=1e-14)
    assert np.allclose(S @ Si, np.eye(4), atol=1e-9)
    assert np.allclose(S, S.T.conj(), atol=1e-15)


def test_rank_deficient_message_is_cut_relative_to_the_largest_eigenvalue():
    # pinv_rel 1e-5 (well above the rounding of M, so the kept eigenvectors
    # are exact to ~1e-11): kept 1, 0.5, 3e-5; cut 5e-6, 0 and a negative one
    eigs = [1.0, 0.5, 3e-5, 5e-6, 0.0, -1e-16]
    M, V = message(eigs, seed=1)
    S, Si = env_sqrt(M, 1e-5)
    keep = np.array([e > 1e-5 for e in eigs])
    P = V[:, keep] @ V[:, keep].T
    Mk = (V[:, keep] * np.array(eigs)[keep]) @ V[:, keep].T
    assert np.allclose(S @ S, Mk, atol=1e-13)
    assert np.allclose(S @ Si, P, atol=1e-8)            # the projector onto the kept space
    assert np.allclose(Si @ S, P, atol=1e-8)
    # the cut directions are annihilated by both factors
    for j in np.flatnonzero(~keep):
        assert np.linalg.norm(S @ V[:, j]) < 1e-10
        assert np.linalg.norm(Si @ V[:, j]) < 1e-8
    # the cut is relative: scaling M moves no eigenvalue across it
    S2, Si2 = env_sqrt(1e6 * M, 1e-5)
    assert np.allclose(S2, 1e3 * S, rtol=0, atol=1e-9)
    assert np.allclose(Si2 @ S2, P, atol=1e-8)


def test_threshold_boundary_and_hermitian_part():
    eigs = [2.0, 4.1e-4, 3.9e-4]                        # pinv_rel 2e-4: the cut is at 4e-4
    M, V = message(eigs, seed=2)
    A = np.array([[0, 1e-3, 0], [-1e-3, 0, 0], [0, 0, 0]])   # antisymmetric part, dropped
    S, Si = env_sqrt(M + A, 2e-4)
    P = V[:, :2] @ V[:, :2].T
    assert np.allclose(Si @ S, P, atol=1e-10)
    assert np.allclose(S @ S, (V[:, :2] * eigs[:2]) @ V[:, :2].T, atol=1e-13)
