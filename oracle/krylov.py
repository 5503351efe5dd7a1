"""Coarse-grid solve of Alg. 2: restarted FGMRES (oracle, complex128).

Alg. 2 solves D_c x_c = y_c only roughly (relative residual about 0.05) by
FGMRES; each iteration applies D_c once, followed by vector work that is
mostly the Gram-Schmidt orthogonalisation.  The reading fixed here: right-preconditioned
flexible GMRES with restart length m (Saad, Iterative Methods for Sparse
Linear Systems, Alg. 9.6), classical Gram-Schmidt in the Arnoldi step (the
same choice the paper makes for the aggregates), Givens rotations for the
small least-squares problem, convergence tested on the implicit residual
|g_{j+1}| <= tol * ||b||.  With no preconditioner it is plain GMRES(m).

Operator applications are counted: each Arnoldi step costs one, and every
restart after the first recomputes the true residual b - A x (one more).
"""
import numpy as np


def _vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def fgmres(apply, b, tol=0.05, restart=30, max_applies=200, precond=None):
    """Solve apply(x) = b from x = 0.  Returns (x, relres_history, n_applies).

    relres_history holds the implicit residual |g_{j+1}| / ||b|| after every
    Arnoldi step; the true residual is the caller's to check.
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    hist = []
    applies = 0
    if bnorm == 0:
        return x, hist, applies
    r = b.copy()
    while True:
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
        m = min(restart, max_applies - applies)
        if m <= 0:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        converged = False
        for j in range(m):
            z = V[j] if precond is None else precond(V[j])
            Z.append(z)
            w = apply(z)
            applies += 1
            # classical Gram-Schmidt: every coefficient from the same w
            for i in range(j + 1):
                H[i, j] = _vdot(V[i], w)
            for i in range(j + 1):
                w = w - H[i, j] * V[i]
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            # earlier Givens rotations applied to the new column
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            # the rotation that zeroes H[j+1, j]
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j] = np.conj(a) / den
            sn[j] = np.conj(c) / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or hnext == 0:
                converged = True
                break
            V.append(w / hnext)
        # back substitution on the k x k upper-triangular system
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
        if converged or applies >= max_applies:
            break
        r = b - apply(x)
        applies += 1
    return x, hist, applies


def refine(apply_outer, solve_inner, b, tol=1e-4, max_outer=50):
    """Iterative refinement: r = b - A x with the accurate operator, then
    x += solve_inner(r) with the cheap one, until ||r|| <= tol ||b||.
    Returns (x, true relative residual history)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    hist = []
    r = b.copy()
    for _ in range(max_outer):
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        if rel <= tol:
            break
        x = x + solve_inner(r)
        r = b - apply_outer(x)
    return x, hist
