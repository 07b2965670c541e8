"""Flexible conjugate gradients, Alg. 2 (oracle; test infrastructure only).

Reading: r_0 = b - J u_0; iterate while k < N_iter and ||r_k||_2 >=
tol ||b||_2 (the printed loop condition joins the two tests with "or", which
never stops when the iteration cap is reached); the preconditioner is
applied to r_k.

Pins (tests/test_oracle_multigrid.py): with the identity preconditioner every
iterate equals textbook CG's, and with a fixed SPD preconditioner M every
iterate equals textbook preconditioned CG's (in exact arithmetic FCG(1) with
a linear preconditioner is PCG); the multigrid-preconditioned solve reaches
1e-10 relative residual on the Poisson problem.
"""
import numpy as np


def fcg(A, b, x0=None, precond=None, tol=1e-10, max_iter=200, callback=None):
    """Returns (x, iterations, history of ||r_k|| / ||b||).  callback(k, x_k),
    if given, sees every iterate (k = 0 is the initial guess)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, [0.0]
    hist = [np.linalg.norm(r) / nb]
    if callback is not None:
        callback(0, x)
    k = 0
    d = q = None
    rho = None
    while k < max_iter and hist[-1] >= tol:
        v = precond(r) if precond is not None else r.copy()
        w = A @ v
        alpha = v @ r
        beta = v @ w
        if k == 0:
            d, q, rho_k = v, w, beta
        else:
            gamma = v @ q
            d = v - (gamma / rho) * d
            q = w - (gamma / rho) * q
            rho_k = beta - gamma * gamma / rho
        x = x + (alpha / rho_k) * d
        r = r - (alpha / rho_k) * q
        rho = rho_k
        k += 1
        hist.append(np.linalg.norm(r) / nb)
        if callback is not None:
            callback(k, x)
    return x, k, hist
