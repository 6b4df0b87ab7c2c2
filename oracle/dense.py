"""Own dense LU with partial pivoting, solve and inverse (brute-force pins).

Pivot rule: the row of largest |z| in the column, ties -> lowest row index.
"""
import numpy as np


def lu(A):
    """P A = L U.  Returns (LU packed, piv) with piv[r] = original row now at r."""
    A = np.array(A, dtype=np.complex128, copy=True)
    n = A.shape[0]
    piv = np.arange(n)
    for j in range(n):
        p = j + int(np.argmax(np.abs(A[j:, j])))
        if A[p, j] == 0:
            raise ZeroDivisionError("singular pivot at column %d" % j)
        if p != j:
            A[[j, p], :] = A[[p, j], :]
            piv[[j, p]] = piv[[p, j]]
        A[j + 1:, j] /= A[j, j]
        A[j + 1:, j + 1:] -= np.outer(A[j + 1:, j], A[j, j + 1:])
    return A, piv


def lu_solve(LU, piv, b):
    """Solve A x = b from lu(A) by forward then backward substitution."""
    b = np.asarray(b, dtype=np.complex128)
    y = b[piv].copy()
    n = LU.shape[0]
    for i in range(n):
        y[i] -= LU[i, :i] @ y[:i]
    for i in range(n - 1, -1, -1):
        y[i] = (y[i] - LU[i, i + 1:] @ y[i + 1:]) / LU[i, i]
    return y


def lu_solve_adjoint(LU, piv, c):
    """Solve A^H y = c from lu(A): A^H = U^H L^H P, so U^H z = c (forward),
    L^H w = z (backward, unit diagonal), y = P^T w."""
    z = np.asarray(c, dtype=np.complex128).copy()
    n = LU.shape[0]
    for i in range(n):
        z[i] = (z[i] - np.conj(LU[:i, i]) @ z[:i]) / np.conj(LU[i, i])
    for i in range(n - 1, -1, -1):
        z[i] -= np.conj(LU[i + 1:, i]) @ z[i + 1:]
    y = np.empty_like(z)
    y[piv] = z
    return y


def solve(A, b):
    LU, piv = lu(A)
    return lu_solve(LU, piv, b)


def inverse(A):
    LU, piv = lu(A)
    n = A.shape[0]
    return lu_solve(LU, piv, np.eye(n, dtype=np.complex128))
