"""Brute-force exact diagonalisation of full n-leg ladders (oracle; test infrastructure only).

Independent of the superblock code: the Hamiltonian of an n x L open ladder is
built state by state in the site occupation basis with bit arithmetic, never
from column or block operators.  Site (x, y) has index s = x*n + y (x along
the legs, y across the rungs).

* Heisenberg: bit s of the state = spin up at site s; bonds along the legs
  carry J_leg, bonds along the rungs J_rung; H = sum J (Sz Sz + (S+S- + S-S+)/2).
* Hubbard: fermion mode 2s + sigma (sigma = 0 up, 1 down); the sign of
  c^dag_i c_j is the parity of the occupied modes below each mode touched.
  The Hamiltonian is block diagonal in (N_up, N_dn) and built per sector.

These give the pins "untruncated DMRG equals ED": a superblock whose blocks
are exact columns has the same spectrum as the full ladder.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def ladder_bonds(n_legs: int, L: int, rung_pbc: bool = False):
    """(site_a, site_b, kind) with kind 'leg' or 'rung'."""
    bonds = []
    for x in range(L):
        for y in range(n_legs):
            s = x * n_legs + y
            if x + 1 < L:
                bonds.append((s, s + n_legs, "leg"))
            if y + 1 < n_legs:
                bonds.append((s, s + 1, "rung"))
            elif rung_pbc and n_legs > 2:
                bonds.append((s, x * n_legs, "rung"))
    return bonds


def heisenberg_matrix(n_legs: int, L: int, J_leg=1.0, J_rung=1.0, rung_pbc=False) -> np.ndarray:
    N = n_legs * L
    dim = 1 << N
    H = np.zeros((dim, dim))
    bonds = ladder_bonds(n_legs, L, rung_pbc)
    for st in range(dim):
        for a, b, kind in bonds:
            J = J_leg if kind == "leg" else J_rung
            ba, bb = (st >> a) & 1, (st >> b) & 1
            H[st, st] += J * (0.5 if ba == bb else -0.5) * 0.5
            if ba != bb:
                H[st ^ ((1 << a) | (1 << b)), st] += 0.5 * J
    return H


def heisenberg_spectrum(n_legs: int, L: int, **kw) -> np.ndarray:
    return np.linalg.eigvalsh(heisenberg_matrix(n_legs, L, **kw))


def spin_dot(N: int, a: int, b: int) -> np.ndarray:
    """S_a . S_b on N spin-1/2 sites (bit s of a state = spin up at site s)."""
    dim = 1 << N
    O = np.zeros((dim, dim))
    for st in range(dim):
        ba, bb = (st >> a) & 1, (st >> b) & 1
        if a == b:
            O[st, st] = 0.75
            continue
        O[st, st] += 0.25 if ba == bb else -0.25
        if ba != bb:
            O[st ^ ((1 << a) | (1 << b)), st] += 0.5
    return O


def heisenberg_ground_correlations(n_legs: int, L: int, J_leg=1.0, J_rung=1.0):
    """Ground energy, state and a function (a, b) -> <S_a . S_b> of the open ladder
    (site index x * n_legs + y), and <S_tot^2> = sum_ab <S_a . S_b>."""
    H = heisenberg_matrix(n_legs, L, J_leg=J_leg, J_rung=J_rung)
    w, v = np.linalg.eigh(H)
    psi = v[:, 0]
    N = n_legs * L
    corr = lambda a, b: float(psi @ spin_dot(N, a, b) @ psi)   # noqa: E731
    s2 = sum(corr(a, b) for a in range(N) for b in range(N))
    return float(w[0]), psi, corr, s2


def _sign_below(state: int, mode: int) -> int:
    return -1 if bin(state & ((1 << mode) - 1)).count("1") % 2 else 1


def _states(n_sites: int, n_up: int, n_dn: int):
    out = []
    for ups in combinations(range(n_sites), n_up):
        u = sum(1 << (2 * s) for s in ups)
        for dns in combinations(range(n_sites), n_dn):
            out.append(u | sum(1 << (2 * s + 1) for s in dns))
    return sorted(out)


def hubbard_sector_matrix(n_legs: int, L: int, n_up: int, n_dn: int, t=1.0, U=8.0,
                          rung_pbc=False) -> sp.csr_matrix:
    n_sites = n_legs * L
    states = _states(n_sites, n_up, n_dn)
    where = {s: i for i, s in enumerate(states)}
    bonds = ladder_bonds(n_legs, L, rung_pbc)
    rows, cols, vals = [], [], []
    for k, st in enumerate(states):
        dbl = sum(1 for s in range(n_sites) if (st >> (2 * s)) & 1 and (st >> (2 * s + 1)) & 1)
        if dbl:
            rows.append(k); cols.append(k); vals.append(U * dbl)
        for a, b, _ in bonds:
            for sig in range(2):
                for i, j in ((2 * a + sig, 2 * b + sig), (2 * b + sig, 2 * a + sig)):
                    # c^dag_i c_j |st>
                    if not (st >> j) & 1 or (st >> i) & 1:
                        continue
                    s1 = _sign_below(st, j)
                    mid = st ^ (1 << j)
                    s2 = _sign_below(mid, i)
                    new = mid | (1 << i)
                    rows.append(where[new]); cols.append(k); vals.append(-t * s1 * s2)
    n = len(states)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def hubbard_spectrum(n_legs: int, L: int, t=1.0, U=8.0, rung_pbc=False) -> np.ndarray:
    """All eigenvalues of the full Fock space, collected over (N_up, N_dn) sectors."""
    n_sites = n_legs * L
    ev = []
    for nu in range(n_sites + 1):
        for nd in range(n_sites + 1):
            H = hubbard_sector_matrix(n_legs, L, nu, nd, t, U, rung_pbc)
            ev.append(np.linalg.eigvalsh(H.toarray()))
    return np.sort(np.concatenate(ev))


def hubbard_ground(n_legs: int, L: int, t=1.0, U=8.0, rung_pbc=False, sector=None) -> float:
    """Lowest eigenvalue over all sectors, or in the given (N_up, N_dn) sector."""
    n_sites = n_legs * L
    sectors = [sector] if sector is not None else [(a, b) for a in range(n_sites + 1)
                                                   for b in range(n_sites + 1)]
    best = np.inf
    for nu, nd in sectors:
        H = hubbard_sector_matrix(n_legs, L, nu, nd, t, U, rung_pbc)
        if H.shape[0] <= 600:
            e = np.linalg.eigvalsh(H.toarray())[0]
        else:
            e = spla.eigsh(H, k=1, which="SA", tol=1e-13)[0][0]
        best = min(best, float(e))
    return best


def hopping_levels(n_legs: int, L: int, t=1.0, rung_pbc=False) -> np.ndarray:
    """Single-particle levels of -t * adjacency (the U = 0 Hubbard model)."""
    n_sites = n_legs * L
    A = np.zeros((n_sites, n_sites))
    for a, b, _ in ladder_bonds(n_legs, L, rung_pbc):
        A[a, b] = A[b, a] = 1.0
    return np.linalg.eigvalsh(-t * A)
