"""DPG-MG V-cycle and preconditioned conjugate gradients (oracle), Sec. 3-4.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

V(nu, nu)-cycle on level l with residual r (Sec. 3 "V-cycle and smoother",
Sec. 4 list: one pre- and one post-smoothing step by default):

  h-level: condense the residual onto the macro grid,
           r_s <- r_s - sum_K A^K_SI (A^K_II)^{-1} r_I^K
  pre-smooth  nu times: x <- x + theta S (r_s - M x)   (from x = 0)
  restrict:   r_c = P^* (r_s - M x)    (P = injection or natural inclusion)
  recurse:    e_c = V(l - 1, r_c)      (level 0: dense Cholesky solve, or 0)
  prolong:    x <- x + P e_c
  post-smooth nu times
  h-level: back-substitute the interior, x_I = (A^K_II)^{-1} (r_I - A^K_IS x_S)

PCG (Sec. 3 first paragraph; Sec. 4 list): x_0 = 0, complex inner products
(a, b) = b^H a, stop when ||r_k||_2 <= tol ||b||_2 with r_k the recursively
updated residual.  The iteration count is the number of operator
applications (= V-cycle applications).
"""
import numpy as np
import scipy.linalg as sla

from .hierarchy import smoother


def vcycle(levels, l, r, nu_pre=1, nu_post=1):
    lev = levels[l]
    if l == 0:
        if lev.coarsest == "cholesky":
            return sla.cho_solve(lev.chol, r)
        if lev.coarsest == "smooth":
            return lev.theta * smoother(lev, r)
        return np.zeros_like(r)
    if lev.kind == "h":
        rs = np.where(lev.smask, r, 0.0)
        for Sg, Ig, T in zip(lev.S, lev.I, lev.T):
            rs[Sg] -= T @ r[Ig]
    else:
        rs = r
    M = lev.M
    x = np.zeros_like(r)
    for _ in range(nu_pre):
        x = x + lev.theta * smoother(lev, rs - M @ x)
    r1 = rs - M @ x
    if lev.kind == "p":
        rc = r1[lev.inj]
    else:
        rc = lev.P.conj().T @ r1
    ec = vcycle(levels, l - 1, rc, nu_pre, nu_post)
    if lev.kind == "p":
        x[lev.inj] += ec
    else:
        x = x + lev.P @ ec
    for _ in range(nu_post):
        x = x + lev.theta * smoother(lev, rs - M @ x)
    if lev.kind == "h":
        for Sg, Ig, T, Ai in zip(lev.S, lev.I, lev.T, lev.Aii_inv):
            x[Ig] = Ai @ r[Ig] - T.conj().T @ x[Sg]
    return x


def pcg(A, b, precond, tol=1e-8, max_iter=1000):
    """Preconditioned CG; returns (x, iterations, relative residual history)."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    hist = [1.0]
    if nb == 0.0:
        return x, 0, hist
    z = precond(r)
    pdir = z.copy()
    rho = np.vdot(z, r)             # (r, z) = z^H r
    it = 0
    while it < max_iter:
        q = A @ pdir
        alpha = rho / np.vdot(pdir, q)
        x = x + alpha * pdir
        r = r - alpha * q
        it += 1
        rel = np.linalg.norm(r) / nb
        hist.append(rel)
        if rel <= tol:
            break
        z = precond(r)
        rho_new = np.vdot(z, r)
        beta = rho_new / rho
        rho = rho_new
        pdir = z + beta * pdir
    return x, it, hist


def mg_pcg(levels, A, b, tol=1e-8, max_iter=1000, nu_pre=1, nu_post=1):
    L = len(levels) - 1
    return pcg(A, b, lambda r: vcycle(levels, L, r, nu_pre, nu_post), tol, max_iter)
