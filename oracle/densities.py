"""Site densities of the two central columns (oracle; test infrastructure only).

The paper's ground-state observables of its Hubbard study (the section on the 4 x 20
ladder): the hole density h(x,y) = 1 - <n_{x,y,up} + n_{x,y,dn}> (its Eq. (hole)), the
staggered spin density s(x,y) = <n_{x,y,up} - n_{x,y,dn}>, which the Lieb-Mattis
theorem makes vanish on every site of the finite ladder's ground state, and its
leg-direction profile S(x) = max_y |s(x,y)| (its Eq. (staggeed)).  One superblock holds
the sites of columns 2 and 3 exactly, so a DMRG step measures these two columns.

The occupation numbers are diagonal in the column basis (product states of the
column's modes or spins), so

    <n_{2,y,s}> = sum_{i2} occ_{y,s}(i2) w2(i2),  w2(i2) = sum_{i1,i3,i4} |x(i1,i2,i3,i4)|^2

over <x|x>, and likewise for column 3 with w3(i3).  For a spin column n_up / n_dn are
the probabilities of up / down (their sum is 1, h = 0, s = 2 <S^z>).
"""
from __future__ import annotations

import numpy as np

from .columns import HubbardColumn, SpinColumn
from .superblock import Superblock


def column_occupations(col) -> np.ndarray:
    """occ[i, y, s] of every column state i: electrons of spin s on leg y (the diagonal of
    c^dag_{y,s} c_{y,s}), or for a spin column 1 if leg y's spin is up (s = 0) / down
    (s = 1), read off the diagonal of S^z_y."""
    n, d = col.n, col.d
    occ = np.zeros((d, n, 2))
    for y in range(n):
        if isinstance(col, HubbardColumn):
            for s in range(2):
                occ[:, y, s] = np.diag(col.cdag[y][s] @ col.c[y][s])
        else:
            up = (np.diag(col.Sz[y]) > 0).astype(float)
            occ[:, y, 0] = up
            occ[:, y, 1] = 1.0 - up
    return occ


def site_densities(sb: Superblock, x: np.ndarray) -> dict:
    """n[c, y, s] for c = 0 (column 2) and 1 (column 3), the hole density h[c, y], the
    staggered spin density sd[c, y] and S[c] = max_y |sd[c, y]|."""
    P = sb.tensor(x) ** 2                    # indices (i1, i2, i4, i3)
    tot = P.sum()
    w2 = P.sum(axis=(0, 2, 3)) / tot
    w3 = P.sum(axis=(0, 1, 2)) / tot
    occ = column_occupations(sb.col)
    n = np.stack([np.einsum("i,iys->ys", w2, occ), np.einsum("i,iys->ys", w3, occ)])
    h = 1.0 - n[..., 0] - n[..., 1]
    sd = n[..., 0] - n[..., 1]
    return {"n": n, "h": h, "sd": sd, "S": np.abs(sd).max(axis=1)}


def exact_column_block(mdl: dict) -> dict:
    """A block of exactly one column (no truncation), in the block format of
    ``Superblock``: H, boundary operators, and for electrons the parity and the
    (N_up, N_dn) labels; for spins the N_up label."""
    n = mdl["n_legs"]
    if mdl["kind"] == "hubbard":
        col = HubbardColumn(n, mdl["t"], mdl["U"], mdl.get("rung_pbc", False))
        edge = [col.cdag[y][s].copy() for y in range(n) for s in range(2)]
        return {"m": col.d, "H": col.H.copy(), "edge": edge, "parity": col.parity.copy(),
                "qn": np.stack([col.n_up, col.n_dn], axis=1).astype(np.int32)}
    col = SpinColumn(n, mdl["J_rung"], mdl.get("rung_pbc", False))
    edge = []
    for y in range(n):
        edge += [col.Sz[y].copy(), col.Sp[y].copy()]
    return {"m": col.d, "H": col.H.copy(), "edge": edge,
            "qn": col.n_up.reshape(-1, 1).astype(np.int32)}
