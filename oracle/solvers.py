"""FP64 ground-state solvers for the superblock (oracle; test infrastructure only).

The paper computes the superblock ground state by repeated H·v ("HMED",
discussion of Fig. 5) but does not name the eigensolver.  The oracle uses the
two standard choices, written out step by step:

* Lanczos with full reorthogonalisation (classical Gram-Schmidt applied
  twice), stopping when the Ritz residual estimate |beta_j s_j[last]| is at
  most tol*|theta|, or after a fixed number of steps;
* Davidson with the diagonal (Jacobi) preconditioner t = r / (theta - D).

Library routines serve as steps: numpy dot products and norms, and
scipy.linalg.eigh_tridiagonal / numpy.linalg.eigh for the small projected
eigenproblems.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh_tridiagonal


def lanczos_ground(apply, v0, max_iter=200, tol=1e-10, fixed_steps=False):
    """Lowest eigenpair of a symmetric operator by Lanczos with full reorthogonalisation.

    Returns (theta, x, info) with info = {"iters", "thetas", "resid_est"}.
    """
    q = np.asarray(v0, dtype=np.float64)
    q = q / np.linalg.norm(q)
    n = q.size
    kmax = min(max_iter, n)
    Q = np.zeros((kmax + 1, n))
    Q[0] = q
    alpha, beta, thetas, res = [], [], [], []
    theta, s = None, None
    for j in range(kmax):
        w = apply(Q[j])
        a = float(Q[j] @ w)
        w = w - a * Q[j]
        if j > 0:
            w = w - beta[j - 1] * Q[j - 1]
        for _ in range(2):                       # CGS2 against the whole basis
            w = w - Q[: j + 1].T @ (Q[: j + 1] @ w)
        b = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(b)
        if j == 0:
            ev, vec = np.array([a]), np.ones((1, 1))
        else:
            ev, vec = eigh_tridiagonal(np.array(alpha), np.array(beta[:-1]))
        theta, s = float(ev[0]), vec[:, 0]
        r = abs(b * s[-1])
        thetas.append(theta)
        res.append(r)
        if b <= 1e-300:
            break
        if not fixed_steps and r <= tol * abs(theta):
            break
        Q[j + 1] = w / b
    k = len(alpha)
    x = Q[:k].T @ s
    return theta, x / np.linalg.norm(x), {"iters": k, "thetas": thetas, "resid_est": res}


def davidson_ground(apply, diag, v0, max_iter=500, tol=1e-8, max_subspace=40, eps=1e-12):
    """Lowest eigenpair by Davidson with the Jacobi preconditioner.

    Stops when ||H x - theta x|| <= tol * |theta|.  Returns (theta, x, info).
    """
    x = np.asarray(v0, dtype=np.float64)
    x = x / np.linalg.norm(x)
    D = np.asarray(diag, dtype=np.float64)
    Vb = [x]
    AV = [apply(x)]
    theta, hist = None, []
    it = 0
    for it in range(1, max_iter + 1):
        Vm = np.array(Vb)
        Am = np.array(AV)
        G = Vm @ Am.T
        G = 0.5 * (G + G.T)
        ev, vec = np.linalg.eigh(G)
        theta, s = float(ev[0]), vec[:, 0]
        x = s @ Vm
        Ax = s @ Am
        r = Ax - theta * x
        rn = float(np.linalg.norm(r))
        hist.append((theta, rn))
        if rn <= tol * abs(theta):
            break
        den = theta - D
        den = np.where(np.abs(den) < eps, np.copysign(eps, den + 0.0), den)
        t = r / den
        if len(Vb) >= max_subspace:
            Vb, AV = [x / np.linalg.norm(x)], [Ax / np.linalg.norm(x)]
        for _ in range(2):
            for u in Vb:
                t = t - (u @ t) * u
        tn = np.linalg.norm(t)
        if tn <= 1e-14:
            break
        t = t / tn
        Vb.append(t)
        AV.append(apply(t))
    return theta, x / np.linalg.norm(x), {"iters": it, "hist": hist}


def dense_ground(H: np.ndarray):
    ev, vec = np.linalg.eigh(H)
    return float(ev[0]), vec[:, 0]
