"""Pins of the CPU oracle against facts fixed outside it (CPU only).

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
transposed block operator, a wrong Jordan-Wigner sign, a wrong index map)
fails at least one of them:

* the paper's 1-based index maps for V and V_c against a reshape;
* four independent formulations of H·v (4-index Eq. (dec), the paper's
  H_l V + V H_r^T + H_c V_c, the A_k V B_k^T form, the explicit Kronecker
  matrix) against each other;
* closed-form spectra (spin dimer, 4-site ring, Hubbard dimer);
* "untruncated DMRG equals ED": superblocks built from exact columns against
  brute-force diagonalisation of the full ladder in the site basis;
* special cases: decoupled rungs (J_leg = 0) and free fermions (U = 0);
* Hermiticity, sector closure, the diagonal, and the solvers against eigh.
"""
import json
import os

import numpy as np
import pytest

from oracle import lattice_ed
from oracle.columns import HubbardColumn, SpinColumn
from oracle.solvers import davidson_ground, dense_ground, lanczos_ground
from oracle.superblock import Superblock
from paper_0707_0159_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def spin_column_block(n, J_rung=1.0):
    col = SpinColumn(n, J_rung)
    edge = []
    for y in range(n):
        edge += [col.Sz[y], col.Sp[y]]
    return {"m": col.d, "H": col.H, "edge": edge, "parity": None,
            "qn": col.n_up.reshape(-1, 1).astype(np.int32)}


def hubbard_column_block(n, t=1.0, U=8.0):
    col = HubbardColumn(n, t, U)
    edge = []
    for y in range(n):
        edge += [col.cdag[y][0], col.cdag[y][1]]
    return {"m": col.d, "H": col.H, "edge": edge, "parity": col.parity,
            "qn": np.stack([col.n_up, col.n_dn], 1).astype(np.int32)}


def sector_spectra(sb, labels_iter):
    H = sb.dense()
    out = []
    for target in labels_iter:
        mask = sb.sector_mask(target)
        if mask.any():
            out.append(np.linalg.eigvalsh(H[np.ix_(mask, mask)]))
    return np.sort(np.concatenate(out))


# ---- index maps (paper, text after Eq. (dec)) -------------------------------------------

def test_paper_index_maps():
    m, n_legs = 3, 1
    mdl = synth.model("heisenberg", n_legs)
    blk = synth.heisenberg_block(m, n_legs, 5)
    sb = Superblock(mdl, blk, synth.heisenberg_block(m, n_legs, 6))
    d = sb.d                                   # the paper's n in these formulas
    v = np.arange(sb.n_vec, dtype=float)
    V, Vc = sb.V_of(v), sb.Vc_of(v)
    for i1 in range(1, m + 1):
        for i2 in range(1, d + 1):
            for i3 in range(1, d + 1):
                for i4 in range(1, m + 1):
                    k = (i3 - 1) * m * m * d + (i4 - 1) * m * d + (i2 - 1) * m + i1
                    assert V[(i2 - 1) * m + i1 - 1, (i3 - 1) * m + i4 - 1] == v[k - 1]
                    assert Vc[(i3 - 1) * d + i2 - 1, (i4 - 1) * m + i1 - 1] == v[k - 1]
    assert np.array_equal(sb.v_of_Vc(Vc), v)


# ---- the formulations agree --------------------------------------------------------------

@pytest.mark.parametrize("kind", ["heisenberg", "hubbard"])
def test_formulations_agree(kind):
    n_legs = 2 if kind == "heisenberg" else 1
    mdl = synth.model(kind, n_legs, J_leg=0.7, J_rung=1.3, t=0.9, U=3.0)
    mk = synth.heisenberg_block if kind == "heisenberg" else synth.hubbard_block
    sb = Superblock(mdl, mk(3, n_legs, 1), mk(5, n_legs, 2))
    v = synth.start_vector(sb.n_vec, 3)
    y0 = sb.dense() @ v
    for y in (sb.apply(v), sb.apply_matrix_form(v), sb.apply_AVB(v)):
        assert np.linalg.norm(y - y0) <= 1e-13 * np.linalg.norm(y0)
    idx = np.random.default_rng(0).integers(0, sb.n_vec, 17)
    assert np.allclose(sb.apply_at(v, idx), y0[idx], rtol=1e-13, atol=1e-13)
    assert np.allclose(sb.diagonal(), np.diag(sb.dense()), rtol=0, atol=1e-14)


@pytest.mark.parametrize("kind", ["heisenberg", "hubbard"])
def test_hermitian_and_linear(kind):
    mdl = synth.model(kind, 2)
    mk = synth.heisenberg_block if kind == "heisenberg" else synth.hubbard_block
    sb = Superblock(mdl, mk(4, 2, 7), mk(6, 2, 8))
    rng = np.random.default_rng(1)
    v, w = rng.normal(size=sb.n_vec), rng.normal(size=sb.n_vec)
    Hv, Hw = sb.apply(v), sb.apply(w)
    assert abs(w @ Hv - Hw @ v) <= 1e-12 * np.linalg.norm(Hv) * np.linalg.norm(w)
    assert np.allclose(sb.apply(2.0 * v - 3.0 * w), 2.0 * Hv - 3.0 * Hw, atol=1e-12)


# ---- closed forms ---------------------------------------------------------------------------

def test_spin_dimer():
    mdl = synth.model("heisenberg", 1, J_leg=1.0)
    e = synth.empty_block("heisenberg")
    ev = np.linalg.eigvalsh(Superblock(mdl, e, e).dense())
    assert np.allclose(ev, GOLD["heisenberg_dimer"]["spectrum"], atol=1e-14)


def test_plaquette():
    mdl = synth.model("heisenberg", 2, J_leg=1.0, J_rung=1.0)
    e = synth.empty_block("heisenberg")
    ev = np.linalg.eigvalsh(Superblock(mdl, e, e).dense())
    assert abs(ev[0] - GOLD["heisenberg_plaquette"]["ground"]) <= 1e-13


def test_hubbard_dimer_spectrum():
    g = GOLD["hubbard_dimer"]
    mdl = synth.model("hubbard", 1, t=g["t"], U=g["U"])
    e = synth.empty_block("hubbard")
    ev = np.linalg.eigvalsh(Superblock(mdl, e, e).dense())
    assert np.allclose(ev, g["spectrum"], atol=1e-12)


# ---- untruncated superblock equals brute-force ED ---------------------------------------------

def test_ladder_2x4_heisenberg_equals_ed():
    mdl = synth.model("heisenberg", 2, J_leg=1.0, J_rung=1.0)
    blk = spin_column_block(2)
    ev = np.linalg.eigvalsh(Superblock(mdl, blk, blk).dense())
    ref = lattice_ed.heisenberg_spectrum(2, 4)
    assert np.allclose(ev, ref, atol=1e-12)


def test_ladder_3x2_anisotropic_couplings_equal_ed():
    # 3 legs, two columns, J_leg != J_rung; checks which bonds carry which J
    mdl = synth.model("heisenberg", 3, J_leg=0.6, J_rung=1.7)
    e = synth.empty_block("heisenberg")
    ev = np.linalg.eigvalsh(Superblock(mdl, e, e).dense())
    ref = lattice_ed.heisenberg_spectrum(3, 2, J_leg=0.6, J_rung=1.7)
    assert np.allclose(ev, ref, atol=1e-12)


@pytest.mark.parametrize("side", ["left", "right"])
def test_ladder_2x3_hubbard_equals_ed(side):
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    col = hubbard_column_block(2, 1.0, 8.0)
    e = synth.empty_block("hubbard", qn=(0, 0))
    sb = Superblock(mdl, col, e) if side == "left" else Superblock(mdl, e, col)
    targets = [(a, b) for a in range(7) for b in range(7)]
    ev = sector_spectra(sb, targets)
    ref = lattice_ed.hubbard_spectrum(2, 3, t=1.0, U=8.0)
    assert ev.shape == ref.shape
    assert np.allclose(ev, ref, atol=1e-10)


def test_ladder_2x4_hubbard_ground_equals_ed():
    # both blocks exact columns: every term of H_l, H_r and H_c carries fermion signs
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    col = hubbard_column_block(2, 1.0, 8.0)
    sb = Superblock(mdl, col, col)
    for target in [(4, 4), (3, 2)]:
        mask = sb.sector_mask(target)
        v0 = np.where(mask, synth.start_vector(sb.n_vec, 11), 0.0)
        th, x, info = lanczos_ground(sb.apply, v0, max_iter=300, tol=1e-12)
        ref = lattice_ed.hubbard_ground(2, 4, 1.0, 8.0, sector=target)
        assert abs(th - ref) <= 1e-9 * abs(ref), (target, th, ref)


# ---- special cases ---------------------------------------------------------------------------

def test_decoupled_rungs():
    mdl = synth.model("heisenberg", 2, J_leg=0.0, J_rung=1.0)
    blk = spin_column_block(2)
    ev = np.linalg.eigvalsh(Superblock(mdl, blk, blk).dense())
    assert abs(ev[0] - 4 * (-0.75)) <= 1e-12


def test_free_fermions():
    mdl = synth.model("hubbard", 2, t=1.0, U=0.0)
    col = hubbard_column_block(2, 1.0, 0.0)
    e = synth.empty_block("hubbard", qn=(0, 0))
    sb = Superblock(mdl, col, e)
    eps = lattice_ed.hopping_levels(2, 3)
    e0 = 2.0 * eps[eps < 0].sum()
    th, _, _ = lanczos_ground(sb.apply, synth.start_vector(sb.n_vec, 4), max_iter=400, tol=1e-13)
    assert abs(th - e0) <= 1e-9 * abs(e0)


# ---- sectors -------------------------------------------------------------------------------

def test_sector_closure_heisenberg():
    mdl, left, right, target = synth.workload_ladder4_heisenberg_sectors(m=48, block_sites=8)
    sb = Superblock(mdl, left, right)
    mask = sb.sector_mask(target)
    assert 0 < mask.sum() < mask.size
    v = np.where(mask, synth.start_vector(sb.n_vec, 5), 0.0)
    y = sb.apply(v)
    assert np.all(y[~mask] == 0.0)
    assert np.linalg.norm(y[mask]) > 0


def test_sector_closure_hubbard():
    mdl, left, right, target = synth.workload_ladder3_hubbard_sectors(m=25, block_sites=6, n_up=6, n_dn=6)
    sb = Superblock(mdl, left, right)
    mask = sb.sector_mask(target)
    assert 0 < mask.sum() < mask.size
    v = np.where(mask, synth.start_vector(sb.n_vec, 5), 0.0)
    y = sb.apply(v)
    assert np.all(y[~mask] == 0.0)


# ---- solvers ---------------------------------------------------------------------------------

def test_lanczos_against_eigh():
    mdl = synth.model("hubbard", 1)
    sb = Superblock(mdl, synth.hubbard_block(5, 1, 1), synth.hubbard_block(6, 1, 2))
    e0, _ = dense_ground(sb.dense())
    th, x, info = lanczos_ground(sb.apply, synth.start_vector(sb.n_vec, 2), max_iter=400, tol=1e-12)
    assert abs(th - e0) <= 1e-10 * abs(e0)
    r = sb.apply(x) - th * x
    assert np.linalg.norm(r) <= 1e-8
    # Ritz values of a growing Krylov space never increase (Cauchy interlacing)
    assert np.all(np.diff(info["thetas"]) <= 1e-12)


def test_davidson_against_eigh():
    mdl = synth.model("heisenberg", 2)
    sb = Superblock(mdl, synth.heisenberg_block(6, 2, 3), synth.heisenberg_block(7, 2, 4))
    e0, _ = dense_ground(sb.dense())
    th, x, info = davidson_ground(sb.apply, sb.diagonal(), synth.start_vector(sb.n_vec, 9),
                                  tol=1e-10, max_iter=300)
    assert abs(th - e0) <= 1e-10 * abs(e0)


def test_synth_is_deterministic_and_shaped():
    a = synth.hubbard_block(16, 3, 10)
    b = synth.hubbard_block(16, 3, 10)
    assert all(np.array_equal(x, y) for x, y in zip(a["edge"], b["edge"]))
    P = np.diag(a["parity"])
    for c in a["edge"]:
        assert np.allclose(P @ c @ P, -c)          # parity-odd edge operators
    assert np.allclose(P @ a["H"] @ P, a["H"])     # parity-even block Hamiltonian
    assert np.allclose(a["H"], a["H"].T)
    offs, sizes = synth.sector_sizes([(q,) for q in range(-3, 4)], (1.0,), 1024, 20)
    assert sum(sizes) == 1024 and min(sizes) >= 5 and max(sizes) <= 400
