"""GMRES for the left-preconditioned system M A u = M f (Section 2.4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Unrestarted GMRES (Saad & Schultz) with x0 = 0: Arnoldi by modified Gram-Schmidt,
Givens rotations on the Hessenberg matrix, stop when the preconditioned residual
|| M (f - A u_k) ||_2 <= tol || M f ||_2 ("relative residue", Section 3) or after
max_it steps.  N_iter is the number of Arnoldi steps taken.
"""
import numpy as np


def gmres(op, b, tol, max_it=200):
    """Solve op(x) = b.  Returns (x, iterations, residual history)."""
    b = np.asarray(b, dtype=complex)
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros_like(b), 0, [0.0]
    V = [b / beta]
    Hm = np.zeros((max_it + 1, max_it), complex)
    cs = np.zeros(max_it, complex)
    sn = np.zeros(max_it, complex)
    g = np.zeros(max_it + 1, complex)
    g[0] = beta
    hist = [1.0]
    k = 0
    for j in range(max_it):
        w = op(V[j])
        for i in range(j + 1):
            Hm[i, j] = np.vdot(V[i], w)
            w = w - Hm[i, j] * V[i]
        Hm[j + 1, j] = np.linalg.norm(w)
        for i in range(j):                      # previous rotations
            t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
            Hm[i + 1, j] = -np.conj(sn[i]) * Hm[i, j] + np.conj(cs[i]) * Hm[i + 1, j]
            Hm[i, j] = t
        a, bb = Hm[j, j], Hm[j + 1, j]
        r = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
        # unitary rotation [[cs, sn], [-conj(sn), conj(cs)]] mapping (a, bb) to (r, 0)
        cs[j] = np.conj(a) / r if r != 0 else 1.0
        sn[j] = np.conj(bb) / r if r != 0 else 0.0
        Hm[j, j] = r
        Hm[j + 1, j] = 0.0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        hist.append(abs(g[j + 1]) / beta)
        if hist[-1] <= tol or Hm[j, j] == 0:
            break
        nv = np.linalg.norm(w)
        V.append(w / nv if nv != 0 else w)
    y = np.linalg.solve(np.triu(Hm[:k, :k]), g[:k])
    x = sum(y[i] * V[i] for i in range(k))
    return x, k, hist


def preconditioned_solve(A, M_apply, f, tol, max_it=200):
    """GMRES on M A u = M f; A is a sparse matrix, M_apply a callable."""
    b = M_apply(f)
    return gmres(lambda x: M_apply(A @ x), b, tol, max_it)
