"""Dense reference matrices for the preconditioner tests: the oracle's
Poisson operator assembled column by column, the first- and second-order
approximate inverses M^-1 = K^T K of Sec. 3 built literally from their
definition (untruncated), and a plain PCG that counts iterations as the GPU
solver does."""
import numpy as np

import oracle


def dense_A(nx, ny, nz, deg):
    o = oracle.Oracle(nx, ny, nz, wind_dir_deg=deg)
    n = nx * ny * nz
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = o.apply_A(e.reshape(nz, ny, nx)).ravel()
    return A


def ai_inverse(A, w, order):
    """M^-1 = K^T K, K = sqrt(2-w) Dbar^-1/2 (I - L Dbar^-1 [+ (L Dbar^-1)^2]),
    Dbar = D / w, L the strictly lower triangle (x-fastest order)."""
    n = A.shape[0]
    Dbar = np.diag(A) / w
    LD = np.tril(A, -1) / Dbar[None, :]
    P = np.eye(n) - LD
    if order == 2:
        P = P + LD @ LD
    K = np.sqrt(2.0 - w) * (Dbar ** -0.5)[:, None] * P
    return K.T @ K, K


def condition(A, K=None, d=None):
    """Condition number of M^-1 A through the similar SPD matrix K A K^T (or
    D^-1/2 A D^-1/2 for Jacobi, A itself without a preconditioner)."""
    if K is not None:
        S = K @ A @ K.T
    elif d is not None:
        S = A / np.sqrt(np.outer(d, d))
    else:
        S = A
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    return ev[-1] / ev[0], ev[0]


def pcg_iterations(A, Minv, b, tol, rule, max_iter=100000):
    """Iterations of PCG from x = 0 until ||r|| <= tol ||b|| (rule
    "residual") or r.z <= tol ||b||^2 (rule "paper", App. A.3), counting
    like the GPU solver: tested after each update, the paper rule after the
    preconditioner."""
    x = np.zeros_like(b)
    r = b.copy()
    bb = b @ b
    if rule == "residual" and r @ r <= tol * tol * bb:
        return 0, x
    z = Minv @ r
    rz = r @ z
    if rule == "paper" and rz <= tol * bb:
        return 0, x
    d = np.zeros_like(b)
    beta = 0.0
    for it in range(1, max_iter + 1):
        d = z + beta * d
        q = A @ d
        alpha = rz / (d @ q)
        x += alpha * d
        r -= alpha * q
        if rule == "residual" and r @ r <= tol * tol * bb:
            return it, x
        z = Minv @ r
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        if rule == "paper" and rz <= tol * bb:
            return it, x
    raise RuntimeError("no convergence")
