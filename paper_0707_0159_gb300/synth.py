"""Seeded synthetic inputs for the superblock H·v hot path.

This module is the only code shared by the CUDA path's callers (tests, bench)
and the CPU oracle.  It draws random numbers and quantum-number labels and
nothing else: no operator of the method is combined, contracted or applied
here.  Every array is produced by ``numpy.random.default_rng(seed)`` so a
(seed, shape) pair always gives the same bytes on any machine.

The synthetic blocks stand in for the renormalised block 1 / block 4 of the
direct n-leg superblock (block 1 · column · column · block 4, paper Fig. 2).
The paper prints no block data, so the entries are drawn:

* block Hamiltonian ``H``: symmetric, entries N(0, 1/m) (upper triangle drawn,
  then mirrored);
* Heisenberg edge operators, one pair per leg y: ``Sz_y`` symmetric N(0, 1/m),
  ``Sp_y`` (S^+) N(0, 1/m); S^- is the transpose of S^+;
* Hubbard edge operators, one per leg y and spin s: ``cdag_{y,s}`` N(0, 1/m)
  restricted to parity-odd positions; the annihilator is the transpose;
  ``parity`` is a diagonal of +1/-1 (balanced, seeded split) and ``H`` is
  restricted to parity-even positions.

With quantum-number labels (``qn``), every operator is restricted to the
positions its symmetry allows: ``H`` and ``Sz`` keep the label, ``Sp`` raises
N_up by one, ``cdag_{y,up}`` raises N_up and ``cdag_{y,dn}`` raises N_dn.
Labels are absolute particle numbers: ``(N_up,)`` for spins, ``(N_up, N_dn)``
for electrons; states with equal labels are contiguous.
"""
from __future__ import annotations

import numpy as np

HEISENBERG = "heisenberg"
HUBBARD = "hubbard"


def _sym(rng: np.random.Generator, m: int, std: float) -> np.ndarray:
    a = rng.normal(0.0, std, (m, m))
    return np.triu(a) + np.triu(a, 1).T


def sector_sizes(offsets, widths, total: int, seed: int, lo: int = 5, hi: int = 400,
                 jitter: float = 0.10):
    """Uneven sector sizes with a Gaussian profile.

    ``offsets`` is a list of label offsets (tuples), ``widths`` the Gaussian
    width per component.  Size_q is proportional to exp(-sum_i q_i^2/(2 w_i^2))
    times (1 + jitter*U(-1,1)), clamped to [lo, hi] and adjusted so the sizes
    sum to ``total``.
    """
    rng = np.random.default_rng(seed)
    offs = [tuple(o) for o in offsets]
    w = np.array([np.exp(-sum(q * q / (2.0 * s * s) for q, s in zip(o, widths))) for o in offs])
    w *= 1.0 + jitter * rng.uniform(-1.0, 1.0, len(w))
    sizes = np.clip(np.rint(total * w / w.sum()).astype(np.int64), lo, hi)
    order = np.argsort(-w, kind="stable")
    guard = 0
    while sizes.sum() != total:
        diff = total - int(sizes.sum())
        step = 1 if diff > 0 else -1
        moved = False
        for i in order:
            if lo <= sizes[i] + step <= hi:
                sizes[i] += step
                moved = True
                if sizes.sum() == total:
                    break
        guard += 1
        if not moved or guard > 100000:
            raise ValueError("cannot distribute sector sizes within bounds")
    return offs, [int(s) for s in sizes]


def labels_from_sectors(base, offsets, sizes) -> np.ndarray:
    """Per-state labels (m x ncomp int32), sectors contiguous in the given order."""
    base = np.asarray(base, dtype=np.int64)
    rows = []
    for o, s in zip(offsets, sizes):
        rows.extend([base + np.asarray(o, dtype=np.int64)] * s)
    return np.asarray(rows, dtype=np.int32).reshape(len(rows), len(base))


def heisenberg_block(m: int, n_legs: int, seed: int, qn: np.ndarray | None = None) -> dict:
    """Seeded spin block: H, [Sz_0, Sp_0, Sz_1, Sp_1, ...]; labels (N_up,)."""
    rng = np.random.default_rng(seed)
    std = 1.0 / np.sqrt(m)
    H = _sym(rng, m, std)
    edge = []
    for _ in range(n_legs):
        sz = _sym(rng, m, std)
        sp = rng.normal(0.0, std, (m, m))
        edge += [sz, sp]
    if qn is not None:
        q = np.asarray(qn)[:, 0].astype(np.int64)
        same = q[:, None] == q[None, :]
        up = q[:, None] == q[None, :] + 1
        H = H * same
        edge = [e * (same if i % 2 == 0 else up) for i, e in enumerate(edge)]
        qn = np.ascontiguousarray(np.asarray(qn, dtype=np.int32).reshape(m, 1))
    return {"m": m, "H": H, "edge": edge, "parity": None, "qn": qn}


def hubbard_block(m: int, n_legs: int, seed: int, qn: np.ndarray | None = None) -> dict:
    """Seeded electron block: H, [cdag_{0,up}, cdag_{0,dn}, cdag_{1,up}, ...], parity."""
    rng = np.random.default_rng(seed)
    std = 1.0 / np.sqrt(m)
    H = _sym(rng, m, std)
    edge = [rng.normal(0.0, std, (m, m)) for _ in range(2 * n_legs)]
    if qn is None:
        par = np.ones(m)
        par[m // 2:] = -1.0
        par = rng.permutation(par)
        odd = par[:, None] != par[None, :]
        H = H * (~odd)
        edge = [e * odd for e in edge]
    else:
        qn = np.ascontiguousarray(np.asarray(qn, dtype=np.int32).reshape(m, 2))
        nu = qn[:, 0].astype(np.int64)
        nd = qn[:, 1].astype(np.int64)
        par = np.where((nu + nd) % 2 == 0, 1.0, -1.0)
        same = (nu[:, None] == nu[None, :]) & (nd[:, None] == nd[None, :])
        H = H * same
        raise_up = (nu[:, None] == nu[None, :] + 1) & (nd[:, None] == nd[None, :])
        raise_dn = (nd[:, None] == nd[None, :] + 1) & (nu[:, None] == nu[None, :])
        edge = [e * (raise_up if i % 2 == 0 else raise_dn) for i, e in enumerate(edge)]
    return {"m": m, "H": H, "edge": edge, "parity": par, "qn": qn}


def empty_block(kind: str, qn=None) -> dict:
    """The one-state block with no edge operators (a lattice end)."""
    par = np.ones(1) if kind == HUBBARD else None
    if qn is not None:
        qn = np.ascontiguousarray(np.asarray(qn, dtype=np.int32).reshape(1, -1))
    return {"m": 1, "H": np.zeros((1, 1)), "edge": [], "parity": par, "qn": qn}


def start_vector(n: int, seed: int) -> np.ndarray:
    """N(0,1) entries, length n (not normalised)."""
    return np.random.default_rng(seed).normal(0.0, 1.0, n)


# --- the named synthetic workloads -------------------------------------------------

def model(kind: str, n_legs: int, J_leg=1.0, J_rung=1.0, t=1.0, U=8.0, rung_pbc=False) -> dict:
    return {"kind": kind, "n_legs": n_legs, "J_leg": float(J_leg), "J_rung": float(J_rung),
            "t": float(t), "U": float(U), "rung_pbc": bool(rung_pbc)}


def workload_ladder2_heisenberg_m64():
    """2-leg Heisenberg ladder, J_leg=J_rung=1, m=64, d=4; V is 256x256."""
    mdl = model(HEISENBERG, 2)
    return mdl, heisenberg_block(64, 2, 0), heisenberg_block(64, 2, 1), None


def workload_ladder3_hubbard_m256(m: int = 256):
    """3-leg Hubbard ladder, t=1, U=8, d=64, dense; V is (64m)x(64m)."""
    mdl = model(HUBBARD, 3, t=1.0, U=8.0)
    return mdl, hubbard_block(m, 3, 10), hubbard_block(m, 3, 11), None


def workload_ladder4_heisenberg_sectors(m: int = 1024, block_sites: int = 20, seed: int = 20):
    """4-leg Heisenberg ladder, d=16, block N_up sectors q in -3..3 around half filling.

    Target: total N_up = half of (2*block_sites + 2*4) sites, i.e. S^z_tot = 0.
    """
    offs, sizes = sector_sizes([(q,) for q in range(-3, 4)], (1.0,), m, seed)
    lab = labels_from_sectors((block_sites // 2,), offs, sizes)
    offs4, sizes4 = sector_sizes([(q,) for q in range(-3, 4)], (1.0,), m, seed + 1)
    lab4 = labels_from_sectors((block_sites // 2,), offs4, sizes4)
    mdl = model(HEISENBERG, 4)
    target = ((2 * block_sites + 8) // 2,)
    return (mdl, heisenberg_block(m, 4, seed, lab), heisenberg_block(m, 4, seed + 1, lab4), target)


def workload_ladder3_hubbard_sectors(m: int = 1024, block_sites: int = 12, seed: int = 30,
                                     n_up: int = 15, n_dn: int = 15):
    """3-leg Hubbard ladder, t=1, U=8, d=64, (N_up, N_dn) sectors; 3x10 lattice at 15 up 15 dn."""
    grid = [(a, b) for a in range(-2, 3) for b in range(-2, 3)]
    lo = min(5, m // len(grid))
    offs, sizes = sector_sizes(grid, (1.2, 1.2), m, seed, lo=lo)
    base = (block_sites // 2, block_sites // 2)
    lab = labels_from_sectors(base, offs, sizes)
    offs4, sizes4 = sector_sizes(grid, (1.2, 1.2), m, seed + 1, lo=lo)
    lab4 = labels_from_sectors(base, offs4, sizes4)
    mdl = model(HUBBARD, 3, t=1.0, U=8.0)
    return (mdl, hubbard_block(m, 3, seed, lab), hubbard_block(m, 3, seed + 1, lab4), (n_up, n_dn))
