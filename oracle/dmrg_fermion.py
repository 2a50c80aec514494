"""Finite-system direct 2-D DMRG for n-leg Hubbard ladders (oracle; test infrastructure only).

The same step as ``dmrg.py`` (the paper's description around its Fig. 2: superblock
ground state, density matrix of block 1 + column 2 or of column 3 + block 4, its leading
eigenvectors as the new block's basis, every operator the next step needs transformed
into it), for electrons:

* blocks carry the creation operators of their boundary column (mode 2y + s, spin s of
  leg y, in the block's own mode order), their fermion parity and their (N_up, N_dn)
  labels, in the format ``Superblock`` takes;
* the superblock ground state is searched in the target (N_up, N_dn) sector;
* the density matrices are diagonalised per (N_up, N_dn) sector and the m largest
  eigenvalues kept over all sectors, so every kept state has a definite label and parity;
* the warm-up grows block 1 and block 4 each from its own density matrix (a block grown on
  the right has the reversed mode order of its mirror image, so it is built, not copied);
* every step records the site densities of its two central columns (``densities.py``:
  the paper's hole density and staggered spin density).

Mode order inside an enlarged block follows ``Superblock``: block 1 then column 2 (so the
new boundary operators are the column's, carrying block 1's parity), column 3 then
block 4 (the column comes first and carries no string from the block).
"""
from __future__ import annotations

import numpy as np

from .densities import exact_column_block, site_densities
from .solvers import dense_ground, lanczos_ground
from .superblock import Superblock


def _labels(q_col: np.ndarray, q_blk: np.ndarray) -> np.ndarray:
    # labels of the enlarged index i_blk + m i_col
    return (q_col[:, None, :] + q_blk[None, :, :]).reshape(-1, q_col.shape[1])


def enlarge_left(mdl: dict, block: dict) -> dict:
    """Block 1 + column 2 before truncation (index i1 + m1 i2)."""
    sb = Superblock(mdl, block, block)
    col, n = sb.col, sb.n_legs
    P1 = np.diag(np.asarray(block["parity"], float))
    q_col = np.stack([col.n_up, col.n_dn], axis=1)
    return {"m": sb.m1 * col.d, "H": sb.H_left(),
            "edge": [np.kron(col.cdag[y][s], P1) for y in range(n) for s in range(2)],
            "parity": np.kron(col.parity, np.asarray(block["parity"], float)),
            "qn": _labels(q_col, np.asarray(block["qn"]))}


def enlarge_right(mdl: dict, block: dict) -> dict:
    """Column 3 + block 4 before truncation (index i4 + m4 i3)."""
    sb = Superblock(mdl, block, block)
    col, n = sb.col, sb.n_legs
    I4 = np.eye(sb.m4)
    q_col = np.stack([col.n_up, col.n_dn], axis=1)
    return {"m": sb.m4 * col.d, "H": sb.H_right(),
            "edge": [np.kron(col.cdag[y][s], I4) for y in range(n) for s in range(2)],
            "parity": np.kron(col.parity, np.asarray(block["parity"], float)),
            "qn": _labels(q_col, np.asarray(block["qn"]))}


def keep_states(rho: np.ndarray, qn: np.ndarray, m: int):
    """The m leading eigenvectors of a density matrix that conserves the labels qn,
    diagonalised per label (ties: larger eigenvalue first, then label order, then index).
    Returns (U, labels of the kept states, truncation error = 1 - kept weight)."""
    labels = sorted({tuple(r) for r in qn.tolist()})
    cand = []  # (-w, label index, k, vector)
    for li, lab in enumerate(labels):
        idx = np.flatnonzero((qn == np.asarray(lab)).all(axis=1))
        w, Q = np.linalg.eigh(rho[np.ix_(idx, idx)])
        for k in range(len(w)):
            v = np.zeros(rho.shape[0])
            v[idx] = Q[:, k]
            cand.append((-w[k], li, k, v))
    cand.sort(key=lambda c: (c[0], c[1], c[2]))
    kept = cand[:min(m, len(cand))]
    U = np.stack([c[3] for c in kept], axis=1)
    lab = np.array([labels[c[1]] for c in kept], dtype=np.int32)
    return U, lab, float(1.0 - sum(-c[0] for c in kept))


def renormalize(enl: dict, U: np.ndarray, lab: np.ndarray) -> dict:
    """The new block: U^T O U for H and the boundary operators; parity from the labels."""
    par = np.where(lab.sum(axis=1) % 2 == 0, 1.0, -1.0)
    return {"m": U.shape[1], "H": U.T @ enl["H"] @ U, "edge": [U.T @ E @ U for E in enl["edge"]],
            "parity": par, "qn": lab}


def sector_ground(sb: Superblock, target, seed: int = 0, tol: float = 1e-12):
    """Lowest state of the superblock in the (N_up, N_dn) sector; normalised vector."""
    mask = sb.sector_mask(target)
    idx = np.flatnonzero(mask)
    if len(idx) == 0:
        raise ValueError(f"empty sector {target}")
    if len(idx) <= 64:
        H = np.zeros((len(idx), len(idx)))
        for j, k in enumerate(idx):
            e = np.zeros(sb.n_vec)
            e[k] = 1.0
            H[:, j] = sb.apply(e)[idx]
        th, c = dense_ground(H)
        x = np.zeros(sb.n_vec)
        x[idx] = c
        return float(th), x / np.linalg.norm(x)
    fm = mask.astype(float)
    v0 = fm * np.random.default_rng(seed).standard_normal(sb.n_vec)
    th, x, _ = lanczos_ground(lambda v: fm * sb.apply(fm * v), v0, max_iter=min(400, len(idx)),
                              tol=tol)
    return float(th), x / np.linalg.norm(x)


def dmrg(mdl: dict, L: int, n_up: int, n_dn: int, m_warmup: int, m_sweeps: list) -> dict:
    """Warm-up growing both blocks (superblocks of 4, 6, ... columns at the proportional
    filling rounded half up), then one finite sweep per entry of m_sweeps on the L-column
    ladder at (n_up, n_dn).  L even, L >= 4.  Records per step the energy, truncation
    error, position l (columns in block 1), sweep (-1: warm-up) and the site densities of
    columns l and l + 1 (0-based)."""
    if L < 4 or L % 2:
        raise ValueError("L must be even and >= 4")
    half = (L - 2) // 2
    out = {"energy": [], "trunc": [], "l": [], "sweep": [], "n": [], "h": [], "sd": [], "S": []}

    def record(e, tr, dens, l, s):
        out["energy"].append(e)
        out["trunc"].append(tr)
        out["l"].append(l)
        out["sweep"].append(s)
        for k in ("n", "h", "sd", "S"):
            out[k].append(dens[k])

    def target_for(cols):
        # the ladder's filling on a superblock of fewer columns, rounded half up (the
        # paper does not say how the warm-up fills its smaller lattices)
        return (int(np.floor(n_up * cols / L + 0.5)), int(np.floor(n_dn * cols / L + 0.5)))

    one = exact_column_block(mdl)
    left = {1: one}
    right = {1: one}
    for l in range(1, half + 1):  # warm-up: superblock of 2l + 2 columns
        sb = Superblock(mdl, left[l], right[l])
        e, x = sector_ground(sb, target_for(2 * l + 2) if l < half else (n_up, n_dn))
        V = sb.V_of(x)
        tr = 0.0
        if l < half:
            enl = enlarge_left(mdl, left[l])
            U, lab, tr = keep_states(V @ V.T, enl["qn"], m_warmup)
            left[l + 1] = renormalize(enl, U, lab)
            enr = enlarge_right(mdl, right[l])
            U, lab, _ = keep_states(V.T @ V, enr["qn"], m_warmup)
            right[l + 1] = renormalize(enr, U, lab)
        record(e, tr, site_densities(sb, x), l, -1)

    def step(l, grow_left, m):
        r = L - 2 - l
        sb = Superblock(mdl, left[l], right[r])
        e, x = sector_ground(sb, (n_up, n_dn))
        V = sb.V_of(x)
        if grow_left:
            enl = enlarge_left(mdl, left[l])
            U, lab, tr = keep_states(V @ V.T, enl["qn"], m)
            left[l + 1] = renormalize(enl, U, lab)
        else:
            enr = enlarge_right(mdl, right[r])
            U, lab, tr = keep_states(V.T @ V, enr["qn"], m)
            right[r + 1] = renormalize(enr, U, lab)
        return e, tr, site_densities(sb, x)

    for s, m in enumerate(m_sweeps):
        for l in range(half, L - 3):        # to the right end
            e, tr, dens = step(l, True, m)
            record(e, tr, dens, l, s)
        for l in range(L - 3, 1, -1):       # to the left end
            e, tr, dens = step(l, False, m)
            record(e, tr, dens, l, s)
        for l in range(1, half):            # back to the middle
            e, tr, dens = step(l, True, m)
            record(e, tr, dens, l, s)
        sb = Superblock(mdl, left[half], right[half])  # the middle again: measure only
        e, x = sector_ground(sb, (n_up, n_dn))
        record(e, 0.0, site_densities(sb, x), half, s)
    return out
