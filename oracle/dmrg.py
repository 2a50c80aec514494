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
    """A block of one column: its own Hamiltonian and site operators (m = d)."""
    col = SpinColumn(mdl["n_legs"], mdl["J_rung"], mdl.get("rung_pbc", False))
    edge = []
    for y in range(col.n):
        edge += [col.Sz[y].copy(), col.Sp[y].copy()]
    return {"m": col.d, "H": col.H.copy(), "edge": edge}


def _edge_of_new_column(col: SpinColumn, m: int) -> list:
    # the added column is the boundary of the new block; index order (block fast,
    # column slow) makes a column operator X into kron(X, 1_m)
    edge = []
    for y in range(col.n):
        edge += [np.kron(col.Sz[y], np.eye(m)), np.kron(col.Sp[y], np.eye(m))]
    return edge


def enlarge_left(mdl: dict, block: dict):
    """Block 1 + column 2 before truncation: H_l of Eq. (dec) (index i1 + m1 i2) and the
    new boundary operators."""
    sb = Superblock(mdl, block, block)
    return sb.H_left(), _edge_of_new_column(sb.col, block["m"])


def enlarge_right(mdl: dict, block: dict):
    """Column 3 + block 4 before truncation: H_r (index i4 + m4 i3) and the new boundary
    operators (the added column borders the next column 3)."""
    sb = Superblock(mdl, block, block)
    return sb.H_right(), _edge_of_new_column(sb.col, block["m"])


def keep_states(rho: np.ndarray, m: int):
    """The m leading eigenvectors of a density matrix (DMD).  Returns (U, kept
    eigenvalues, truncation error = 1 - their sum, the gap at the cut)."""
    w, Q = np.linalg.eigh(rho)
    order = np.argsort(-w, kind="stable")
    k = min(m, len(w))
    keep = order[:k]
    cut_gap = float(w[order[k - 1]] - w[order[k]]) if k < len(w) else float("inf")
    return Q[:, keep], w[keep], float(1.0 - w[keep].sum()), cut_gap


def renormalize(H_enl: np.ndarray, edge_enl: list, U: np.ndarray) -> dict:
    """The new block: every operator O of the enlarged block becomes U^T O U."""
    return {"m": U.shape[1], "H": U.T @ H_enl @ U, "edge": [U.T @ E @ U for E in edge_enl]}


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
    column 2 from rho_L = V V^T; 'right': column 3 + block 4 from rho_R = V^T V)."""
    sb = Superblock(mdl, left, right)
    e, x = superblock_ground(sb)
    V = sb.V_of(x)
    if grow == "left":
        H_enl, edge = enlarge_left(mdl, left)
        U, w, trunc, gap = keep_states(V @ V.T, m)
    else:
        H_enl, edge = enlarge_right(mdl, right)
        U, w, trunc, gap = keep_states(V.T @ V, m)
    return e, renormalize(H_enl, edge, U), trunc, gap


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
    out = {"energy": [], "trunc": [], "gap": [], "l": [], "sweep": []}

    def record(e, trunc, gap, l, s):
        out["energy"].append(e)
        out["trunc"].append(trunc)
        out["gap"].append(gap)
        out["l"].append(l)
        out["sweep"].append(s)

    for l in range(1, half):  # warm-up: both blocks grow by one column
        e, blk, trunc, gap = step(mdl, left[l], right[l], "left", m_warmup)
        left[l + 1] = blk
        right[l + 1] = blk  # mirror image on a uniform open ladder
        record(e, trunc, gap, l, -1)
    if half == 1:
        e, _, trunc, gap = step(mdl, left[1], right[1], "left", m_warmup)
        record(e, trunc, gap, 1, -1)
    for s, m in enumerate(m_sweeps):
        for l in range(half, L - 3):            # to the right end
            e, left[l + 1], trunc, gap = step(mdl, left[l], right[L - 2 - l], "left", m)
            record(e, trunc, gap, l, s)
        for r in range(1, L - 3):               # to the left end
            l = L - 2 - r
            e, right[r + 1], trunc, gap = step(mdl, left[l], right[r], "right", m)
            record(e, trunc, gap, l, s)
        for l in range(1, half):                # back to the middle
            e, left[l + 1], trunc, gap = step(mdl, left[l], right[L - 2 - l], "left", m)
            record(e, trunc, gap, l, s)
        e, _, trunc, gap = step(mdl, left[half], right[half], "left", m)
        record(e, trunc, gap, half, s)
    return out
