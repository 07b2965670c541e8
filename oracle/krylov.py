"""Flexible conjugate gradients, Alg. 2 (oracle; test infrastructure only).

Reading: r_0 = b - J u_0; iterate while k < N_iter and ||r_k||_2 >=
tol ||b||_2 (the printed loop condition joins the two tests with "or", which
never stops when the iteration cap is reached); the preconditioner is
applied to r_k.

Pins: with the identity preconditioner the iterates equal textbook CG; the
multigrid-preconditioned solve reaches 1e-10 relative residual on the
Poisson problem (tests/test_oracle_multigrid.py).
"""
import numpy as np


def fcg(A, b, x0=None, precond=None, tol=1e-10, max_iter=200):
    """Returns (x, iterations, history of ||r_k|| / ||b||)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, [0.0]
    hist = [np.linalg.norm(r) / nb]
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
    return x, k, hist
