"""Pins of the oracle's iterative refinement (krylov.refine), the outer loop of the
mixed-precision coarse solve: x += solve_inner(r), r = b - A x with the accurate operator.

Expected behaviour comes from closed forms, not from the routine itself: with an exact inner
solver one pass gives A^{-1} b; with an inner solver for a perturbed matrix A + E the residual
obeys r_{k+1} = E (A + E)^{-1} r_k, so every pass shrinks it by at most ||E (A + E)^{-1}||_2.
"""
import numpy as np
import pytest

from oracle import krylov


def _system(n, seed, cond_shift=4.0):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)) + cond_shift * np.sqrt(n) * np.eye(n)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    return A, b, rng


def test_exact_inner_solver_converges_in_one_pass():
    A, b, _ = _system(40, 1)
    x, hist = krylov.refine(lambda v: A @ v, lambda r: np.linalg.solve(A, r), b, tol=1e-12)
    assert hist[0] == pytest.approx(1.0)
    assert len(hist) == 2 and hist[1] <= 1e-13
    assert np.abs(x - np.linalg.solve(A, b)).max() <= 1e-12 * np.abs(np.linalg.solve(A, b)).max()


@pytest.mark.parametrize("eps", [1e-2, 1e-1])
def test_perturbed_inner_solver_contracts_by_the_closed_form_factor(eps):
    A, b, rng = _system(48, 2)
    E = eps * np.linalg.norm(A, 2) * (rng.normal(size=A.shape) + 1j * rng.normal(size=A.shape)) / np.sqrt(A.shape[0])
    q = np.linalg.norm(E @ np.linalg.inv(A + E), 2)
    assert q < 1
    x, hist = krylov.refine(lambda v: A @ v, lambda r: np.linalg.solve(A + E, r), b, tol=1e-10, max_outer=200)
    for k in range(len(hist) - 1):
        assert hist[k + 1] <= q * hist[k] * (1 + 1e-8) + 1e-15
    assert hist[-1] <= 1e-10
    true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert true == pytest.approx(hist[-1], rel=1e-6, abs=1e-15)


def test_pass_budget_is_respected():
    A, b, rng = _system(24, 3)
    E = 0.3 * np.linalg.norm(A, 2) * np.eye(A.shape[0])
    x, hist = krylov.refine(lambda v: A @ v, lambda r: np.linalg.solve(A + E, r), b, tol=1e-14, max_outer=3)
    assert len(hist) == 3
