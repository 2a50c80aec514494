"""Exact operators of one lattice column of n sites (oracle; test infrastructure only).

A "column" is block 2 or block 3 of the superblock (paper Fig. 2): the n sites
x = const, y = 0..n-1 of the n-leg ladder, treated as one DMRG site of
dimension d (paper, discussion of Fig. 1(a): d = 2^n for spins, 4^n for the
Hubbard model).

Basis conventions (they are part of the library's vector layout):

* spin-1/2 column: state index i = sum_y b_y 2^y, b_y = 1 for spin up at leg y;
* Hubbard column: state index i = sum_y (n_{y,up} + 2 n_{y,dn}) 4^y, i.e. bit
  2y+s of i is the occupation of mode (y, s), s = 0 (up), 1 (down).  Fermion
  modes inside a column are ordered by that bit position; the annihilator of
  mode j carries the Jordan-Wigner string prod_{j'<j} (-1)^{n_j'}.

Operators are built here from Kronecker products of single-site (single-mode)
matrices; the brute-force ED in ``lattice_ed`` uses bit arithmetic instead, so
the two constructions are independent.

Model Hamiltonians (the paper names the models but does not write them out;
the readings below are the standard ones):

* Heisenberg: H = sum_<ij> J (S^z_i S^z_j + (S^+_i S^-_j + S^-_i S^+_j)/2),
  J_z = J_xy (paper, Fig. 3 discussion: J_z = J_xy = 1);
* Hubbard: H = -t sum_<ij>,s (c^dag_is c_js + h.c.) + U sum_i n_i,up n_i,dn.
"""
from __future__ import annotations

import numpy as np

SZ = np.diag([-0.5, 0.5])
SP = np.array([[0.0, 0.0], [1.0, 0.0]])  # |up><down|, basis (down, up)
A1 = np.array([[0.0, 1.0], [0.0, 0.0]])  # single-mode annihilator, basis (empty, occupied)
ZJ = np.diag([1.0, -1.0])                # single-mode parity (-1)^n


def _kron_all(mats):
    out = np.ones((1, 1))
    for a in mats:
        out = np.kron(out, a)
    return out


def spin_site_op(op: np.ndarray, y: int, n: int) -> np.ndarray:
    """op acting on leg y of an n-site spin column (leg 0 = least significant bit)."""
    mats = [np.eye(2)] * n
    mats = list(mats)
    mats[n - 1 - y] = op
    return _kron_all(mats)


def fermion_annihilator(j: int, n_modes: int) -> np.ndarray:
    """c_j with the Jordan-Wigner string over modes 0..j-1 (mode 0 = least significant bit)."""
    mats = []
    for k in range(n_modes - 1, -1, -1):
        if k > j:
            mats.append(np.eye(2))
        elif k == j:
            mats.append(A1)
        else:
            mats.append(ZJ)
    return _kron_all(mats)


def rung_bonds(n: int, pbc: bool):
    bonds = [(y, y + 1) for y in range(n - 1)]
    if pbc and n > 2:
        bonds.append((n - 1, 0))
    return bonds


class SpinColumn:
    """n spin-1/2 sites: Sz[y], Sp[y], Sm[y] and the rung Hamiltonian."""

    def __init__(self, n: int, J_rung: float, rung_pbc: bool = False):
        self.n = n
        self.d = 2 ** n
        self.Sz = [spin_site_op(SZ, y, n) for y in range(n)]
        self.Sp = [spin_site_op(SP, y, n) for y in range(n)]
        self.Sm = [s.T.copy() for s in self.Sp]
        H = np.zeros((self.d, self.d))
        for a, b in rung_bonds(n, rung_pbc):
            H += J_rung * (self.Sz[a] @ self.Sz[b]
                           + 0.5 * (self.Sp[a] @ self.Sm[b] + self.Sm[a] @ self.Sp[b]))
        self.H = H
        self.n_up = np.array([bin(i).count("1") for i in range(self.d)])


class HubbardColumn:
    """n Hubbard sites: c[y][s] (with in-column JW string), parity, rung Hamiltonian."""

    def __init__(self, n: int, t: float, U: float, rung_pbc: bool = False):
        self.n = n
        self.d = 4 ** n
        nm = 2 * n
        self.c = [[fermion_annihilator(2 * y + s, nm) for s in range(2)] for y in range(n)]
        self.cdag = [[self.c[y][s].T.copy() for s in range(2)] for y in range(n)]
        num = [[self.cdag[y][s] @ self.c[y][s] for s in range(2)] for y in range(n)]
        H = np.zeros((self.d, self.d))
        for a, b in rung_bonds(n, rung_pbc):
            for s in range(2):
                hop = self.cdag[a][s] @ self.c[b][s]
                H += -t * (hop + hop.T)
        for y in range(n):
            H += U * (num[y][0] @ num[y][1])
        self.H = H
        occ = np.array([[(i >> (2 * y + s)) & 1 for y in range(n) for s in range(2)]
                        for i in range(self.d)])
        self.n_up = occ[:, 0::2].sum(axis=1)
        self.n_dn = occ[:, 1::2].sum(axis=1)
        self.parity = np.where((self.n_up + self.n_dn) % 2 == 0, 1.0, -1.0)
        self.P = np.diag(self.parity)
