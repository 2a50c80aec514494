"""Finite-system direct 2-D DMRG for n-leg spin ladders (oracle; test infrastructure only).

The paper's step (its description of the algorithm around Fig. 2): the superblock is
block 1 + two columns + block 4; the ground state of the superblock Hamiltonian is found
(HMED); the reduced density matrix of block 1 + column 2 is formed from it (DMF) and
diagonalised (DMD); its m leading eigenvectors become the basis of the new block, into
which every operator the next step needs is transformed.  Blocks grow by one whole
column (n sites) per step.  The infinite-system warm-up grows both blocks together (the
right block is the mirror image of the left one on a uniform open ladder); finite sweeps
then move the boundary column by column to one end, back to the other, and back to the
middle, rebuilding one block per step from the stored ones.

Plain FP64 numpy throughout: the superblock H·v, matrices and ground states come from
``oracle.superblock`` (dense eigh for small superblocks, Lanczos otherwise); ties in the
density-matrix spectrum are broken by a stable sort (larger eigenvalue first, then lower
index).  A block is the dict ``Superblock`` takes: {"m", "H", "edge"} with edge =
[S^z_0, S^+_0, S^z_1, S^+_1, ...] of the block's boundary column.
"""
from __future__ import annotations

import numpy as np

from .columns import SpinColumn
from .solvers import dense_ground, lanczos_ground
from .superblock import Superblock


def column_block(mdl: dict) -> dict:
    """A block of one column: its own Hamiltonian, boundary site operators (m = d) and the
    block's total S^z and S^+ (for <S^2> of the superblock state)."""
    col = SpinColumn(mdl["n_legs"], mdl["J_rung"], mdl.get("rung_pbc", False))
    edge = []
    for y in range(col.n):
        edge += [col.Sz[y].copy(), col.Sp[y].copy()]
    return {"m": col.d, "H": col.H.copy(), "edge": edge, "Sz": sum(col.Sz), "Sp": sum(col.Sp)}


def _edge_of_new_column(col: SpinColumn, m: int) -> list:
    # the added column is the boundary of the new block; index order (block fast,
    # column slow) makes a column operator X into kron(X, 1_m)
    edge = []
    for y in range(col.n):
        edge += [np.kron(col.Sz[y], np.eye(m)), np.kron(col.Sp[y], np.eye(m))]
    return edge


def _totals(col: SpinColumn, block: dict):
    # total S^z, S^+ of block + column in the index order block fast, column slow
    I_d, I_m = np.eye(col.d), np.eye(block["m"])
    return (np.kron(I_d, block["Sz"]) + np.kron(sum(col.Sz), I_m),
            np.kron(I_d, block["Sp"]) + np.kron(sum(col.Sp), I_m))


def enlarge_left(mdl: dict, block: dict):
    """Block 1 + column 2 before truncation: H_l of Eq. (dec) (index i1 + m1 i2), the
    new boundary operators and the total S^z, S^+."""
    sb = Superblock(mdl, block, block)
    return sb.H_left(), _edge_of_new_column(sb.col, block["m"]), _totals(sb.col, block)


def enlarge_right(mdl: dict, block: dict):
    """Column 3 + block 4 before truncation: H_r (index i4 + m4 i3), the new boundary
    operators (the added column borders the next column 3) and the total S^z, S^+."""
    sb = Superblock(mdl, block, block)
    return sb.H_right(), _edge_of_new_column(sb.col, block["m"]), _totals(sb.col, block)


def keep_states(rho: np.ndarray, m: int):
    """The m leading eigenvectors of a density matrix (DMD).  Returns (U, kept
    eigenvalues, truncation error = 1 - their sum, the gap at the cut)."""
    w, Q = np.linalg.eigh(rho)
    order = np.argsort(-w, kind="stable")
    k = min(m, len(w))
    keep = order[:k]
    cut_gap = float(w[order[k - 1]] - w[order[k]]) if k < len(w) else float("inf")
    return Q[:, keep], w[keep], float(1.0 - w[keep].sum()), cut_gap


def renormalize(H_enl: np.ndarray, edge_enl: list, totals, U: np.ndarray) -> dict:
    """The new block: every operator O of the enlarged block becomes U^T O U."""
    Sz, Sp = totals
    return {"m": U.shape[1], "H": U.T @ H_enl @ U, "edge": [U.T @ E @ U for E in edge_enl],
            "Sz": U.T @ Sz @ U, "Sp": U.T @ Sp @ U}


def _dot_spin(A1, B1, A2, B2):
    # S_1 . S_2 from S^z and S^+ of each: Sz1 Sz2 + (S+1 S-2 + S-1 S+2) / 2
    return [(1.0, A1, A2), (0.5, B1, B2.T), (0.5, B1.T, B2)]


def observables(sb: Superblock, x: np.ndarray, left: dict, right: dict) -> dict:
    """Of the superblock state x (paper's observables, restricted to what one superblock
    holds): <S_i . S_j> of the n leg bonds between columns 2 and 3, of the rung bonds of
    column 2 (y, y+1), and <S_tot^2> (the Lieb-Mattis check: 0 for the ladder's ground
    state).  Column 2 acts on the rows of V as X (x) 1_m1, column 3 on its columns as
    X (x) 1_m4."""
    V = sb.V_of(x)
    col, m1, m4 = sb.col, sb.m1, sb.m4
    row = lambda X: np.kron(X, np.eye(m1))      # noqa: E731
    cl = lambda X: np.kron(X, np.eye(m4))        # noqa: E731
    leg = []
    for y in range(col.n):
        e = 0.0
        for c, A, B in _dot_spin(col.Sz[y], col.Sp[y], col.Sz[y], col.Sp[y]):
            e += c * float(np.sum(V * (row(A) @ V @ cl(B).T)))
        leg.append(e)
    rung = []
    for y in range(col.n - 1):
        e = 0.0
        for c, A, B in _dot_spin(col.Sz[y], col.Sp[y], col.Sz[y + 1], col.Sp[y + 1]):
            e += c * float(np.sum(V * (row(A @ B) @ V)))
        rung.append(e)
    Sz_l = np.kron(np.eye(col.d), left["Sz"]) + row(sum(col.Sz))
    Sp_l = np.kron(np.eye(col.d), left["Sp"]) + row(sum(col.Sp))
    Sz_r = np.kron(np.eye(col.d), right["Sz"]) + cl(sum(col.Sz))
    Sp_r = np.kron(np.eye(col.d), right["Sp"]) + cl(sum(col.Sp))
    T1 = Sp_l @ V + V @ Sp_r.T                   # S^+_tot x
    T2 = Sz_l @ V + V @ Sz_r.T                   # S^z_tot x
    s2 = float(np.sum(T1 * T1) + np.sum(T2 * T2) + np.sum(V * T2))  # S^-S^+ + Sz^2 + Sz
    return {"leg": leg, "rung": rung, "s2": s2}


def superblock_ground(sb: Superblock, seed: int = 0, tol: float = 1e-12):
    """Ground energy and normalised vector (vector order of ``Superblock``)."""
    if sb.n_vec <= 1024:
        e, x = dense_ground(sb.dense())
        return float(e), x / np.linalg.norm(x)
    v0 = np.random.default_rng(seed).standard_normal(sb.n_vec)
    e, x, _ = lanczos_ground(sb.apply, v0, max_iter=min(400, sb.n_vec), tol=tol)
    return float(e), x / np.linalg.norm(x)


def step(mdl: dict, left: dict, right: dict, grow: str, m: int):
    """One DMRG step: superblock ground state, then the grown block ('left': block 1 +
    column 2 from rho_L = V V^T; 'right': column 3 + block 4 from rho_R = V^T V).
    Returns (energy, new block, truncation error, gap at the cut, observables)."""
    sb = Superblock(mdl, left, right)
    e, x = superblock_ground(sb)
    V = sb.V_of(x)
    if grow == "left":
        H_enl, edge, tot = enlarge_left(mdl, left)
        U, w, trunc, gap = keep_states(V @ V.T, m)
    else:
        H_enl, edge, tot = enlarge_right(mdl, right)
        U, w, trunc, gap = keep_states(V.T @ V, m)
    obs = observables(sb, x, left, right)
    return e, renormalize(H_enl, edge, tot, U), trunc, gap, obs


def dmrg(mdl: dict, L: int, m_warmup: int, m_sweeps: list) -> dict:
    """Infinite-system warm-up with m_warmup, then one finite sweep per entry of m_sweeps
    (to the right end, to the left end, back to the middle).  L even, L >= 4.

    Returns the energy, truncation error and cut gap of every step, in order, with the
    position (columns in block 1) and the sweep index (-1 for the warm-up)."""
    if L < 4 or L % 2:
        raise ValueError("L must be even and >= 4")
    half = (L - 2) // 2
    left = {1: column_block(mdl)}
    right = {1: column_block(mdl)}
    out = {"energy": [], "trunc": [], "gap": [], "l": [], "sweep": [], "leg": [], "rung": [],
           "s2": []}

    def record(e, trunc, gap, obs, l, s):
        out["energy"].append(e)
        out["trunc"].append(trunc)
        out["gap"].append(gap)
        out["l"].append(l)
        out["sweep"].append(s)
        out["leg"].append(obs["leg"])
        out["rung"].append(obs["rung"])
        out["s2"].append(obs["s2"])

    for l in range(1, half):  # warm-up: both blocks grow by one column
        e, blk, trunc, gap, obs = step(mdl, left[l], right[l], "left", m_warmup)
        left[l + 1] = blk
        right[l + 1] = blk  # mirror image on a uniform open ladder
        record(e, trunc, gap, obs, l, -1)
    if half == 1:
        e, _, trunc, gap, obs = step(mdl, left[1], right[1], "left", m_warmup)
        record(e, trunc, gap, obs, 1, -1)
    for s, m in enumerate(m_sweeps):
        for l in range(half, L - 3):            # to the right end
            e, left[l + 1], trunc, gap, obs = step(mdl, left[l], right[L - 2 - l], "left", m)
            record(e, trunc, gap, obs, l, s)
        for r in range(1, L - 3):               # to the left end
            l = L - 2 - r
            e, right[r + 1], trunc, gap, obs = step(mdl, left[l], right[r], "right", m)
            record(e, trunc, gap, obs, l, s)
        for l in range(1, half):                # back to the middle
            e, left[l + 1], trunc, gap, obs = step(mdl, left[l], right[L - 2 - l], "left", m)
            record(e, trunc, gap, obs, l, s)
        e, _, trunc, gap, obs = step(mdl, left[half], right[half], "left", m)
        record(e, trunc, gap, obs, half, s)
    return out
