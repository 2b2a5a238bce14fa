"""Dense Cholesky factorisation and triangular solves (test infrastructure only).

Paper passage: Sec. 2.3, Alg. 3 and Eqs. 3-4.  The printed listing updates
A_tj with L_ik L_jk, an index typo; Eq. 4 also carries a spurious square root.
The reading used here is the textbook right-looking factorisation that both
describe: for each column k, L_kk = sqrt(A_kk), L_ik = A_ik / L_kk below it,
then the trailing block loses the outer product of that column
(A_tj -= L_tk L_jk for t >= j > k).  Then A x = b is solved by forward
substitution L y = b and back substitution L^T x = y (the paragraph after
Eq. 4).  The inner loops are vectorised numpy; the k loop is explicit.
"""

import numpy as np


def cholesky(A):
    """Return lower-triangular L with A = L L^T for symmetric positive definite A."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    L = np.zeros_like(A)
    for k in range(n):
        if not A[k, k] > 0.0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        L[k, k] = np.sqrt(A[k, k])
        L[k + 1:, k] = A[k + 1:, k] / L[k, k]
        col = L[k + 1:, k]
        # Trailing update A_tj -= L_tk L_jk (only the lower triangle is read).
        A[k + 1:, k + 1:] -= np.outer(col, col)
    return L


def forward_substitution(L, b):
    """Solve L y = b for lower-triangular L."""
    b = np.asarray(b, dtype=np.float64)
    y = np.zeros_like(b)
    for i in range(L.shape[0]):
        y[i] = (b[i] - L[i, :i] @ y[:i]) / L[i, i]
    return y


def back_substitution(L, y):
    """Solve L^T x = y for lower-triangular L."""
    y = np.asarray(y, dtype=np.float64)
    n = L.shape[0]
    x = np.zeros_like(y)
    for i in range(n - 1, -1, -1):
        x[i] = (y[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x


def cholesky_solve(L, b):
    """x = A^-1 b given the factor L of A."""
    return back_substitution(L, forward_substitution(L, b))
