"""H·v over P ranks that each hold a column slab of V (oracle; test infrastructure only).

The paper spreads V over processors and needs the product with H_r (and, in its
form, H_c V_c) on a re-distributed copy of V (its description of the parallel
H·v after Eq. (dec)).  Here rank g holds the columns (i3, i4) of V with i4 in a
contiguous range S_g, for every i3:

* H_l V acts on the row indices (i1, i2) only: local.
* sum_k A_k V B_k^T with A_k = a_k (x) 1 on i2 and B_k = b_k (x) 1 on i3 leaves i4
  alone: local.
* V H_r^T couples all columns (i3, i4): an all-to-all moves V from column slabs to
  row slabs (rank h receives the rows i1 in a contiguous range R_h of every slab),
  rank h applies the H_r terms, and a second all-to-all returns each slab's part.

Everything is the same FP64 einsum per Kronecker term as ``Superblock.apply``;
only the data placement differs.  ``exchange`` is any all-to-all of lists of
arrays (``simulate`` below runs the ranks in one process; the tests also run it
over torch.distributed with the gloo backend).
"""
from __future__ import annotations

import numpy as np


def ranges(n: int, parts: int):
    """Contiguous, balanced split of range(n) into `parts` pieces (some may be empty)."""
    edges = [(n * g) // parts for g in range(parts + 1)]
    return [np.arange(edges[g], edges[g + 1]) for g in range(parts)]


def local_terms(sb, Ws: np.ndarray) -> np.ndarray:
    """H_l and H_c terms on a slab W[i1, i2, i4 in S_g, i3] (identity on i4)."""
    out = np.zeros_like(Ws)
    for c, X, Y in sb.terms_l:
        out += c * np.einsum("ia,jb,abkl->ijkl", Y, X, Ws, optimize=True)
    for c, a, b in sb.terms_c:
        out += c * np.einsum("jb,lc,ibkc->ijkl", a, b, Ws, optimize=True)
    return out


def right_terms(sb, Wr: np.ndarray) -> np.ndarray:
    """H_r terms on a row slab W[i1 in R_h, i2, i4, i3] (identity on i1, i2)."""
    out = np.zeros_like(Wr)
    for c, X, Y in sb.terms_r:
        out += c * np.einsum("ka,lb,ijab->ijkl", Y, X, Wr, optimize=True)
    return out


def rank_step1(sb, Ws: np.ndarray, P: int):
    """Local terms of rank g's slab, and the pieces it sends: rows R_h of its slab to h."""
    R = ranges(sb.m1, P)
    return local_terms(sb, Ws), [Ws[R[h]] for h in range(P)]


def rank_step2(sb, recv: list, P: int):
    """Rank h: join the received pieces (slab g's columns S_g) into its row slab, apply
    the H_r terms, and cut the result back into per-slab pieces."""
    S = ranges(sb.m4, P)
    Wr = np.concatenate(recv, axis=2)          # i4 pieces in slab order
    Zr = right_terms(sb, Wr)
    return [Zr[:, :, S[g], :] for g in range(P)]


def rank_step3(local: np.ndarray, recv: list) -> np.ndarray:
    """Rank g: its slab of y = local terms + the H_r parts returned by every row owner."""
    return local + np.concatenate(recv, axis=0)  # i1 pieces in rank order


def slabs_of(sb, v: np.ndarray, P: int):
    W = sb.tensor(v)
    return [W[:, :, s, :] for s in ranges(sb.m4, P)]


def simulate(sb, v: np.ndarray, P: int) -> np.ndarray:
    """y = H v computed by P simulated ranks; returned in the usual vector order."""
    slabs = slabs_of(sb, v, P)
    s1 = [rank_step1(sb, slabs[g], P) for g in range(P)]
    s2 = [rank_step2(sb, [s1[g][1][h] for g in range(P)], P) for h in range(P)]
    ys = [rank_step3(s1[g][0], [s2[h][g] for h in range(P)]) for g in range(P)]
    return sb.flat(np.concatenate(ys, axis=2))
