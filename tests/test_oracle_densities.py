"""Pins of the oracle's site densities (the paper's hole density h(x,y), staggered spin
density s(x,y) and S(x)): brute-force lattice ED, the Lieb-Mattis zero, an independent
operator route, and the spin-column identities."""
import numpy as np
import pytest

from oracle.densities import column_occupations, exact_column_block, site_densities
from oracle.lattice_ed import _states, hubbard_sector_matrix
from oracle.solvers import lanczos_ground
from oracle.superblock import Superblock
from paper_0707_0159_gb300 import synth


def ed_site_densities(n_legs, L, n_up, n_dn, t=1.0, U=8.0):
    """<n_{site,s}> of the (n_up, n_dn) ground state of the n_legs x L Hubbard ladder by
    exact diagonalisation; site = x n_legs + y, mode 2 site + s."""
    H = hubbard_sector_matrix(n_legs, L, n_up, n_dn, t, U).toarray()
    w, V = np.linalg.eigh(H)
    assert w[1] - w[0] > 1e-3  # non-degenerate: the densities are unique
    psi2 = V[:, 0] ** 2
    st = np.array(_states(n_legs * L, n_up, n_dn))
    n = np.zeros((L, n_legs, 2))
    for x in range(L):
        for y in range(n_legs):
            for s in range(2):
                n[x, y, s] = psi2 @ ((st >> (2 * (x * n_legs + y) + s)) & 1)
    return float(w[0]), n


@pytest.fixture(scope="module")
def hubbard_2x4_doped():
    """2 x 4 Hubbard ladder (t = 1, U = 8) with 3 up and 3 down electrons: blocks 1 and 4
    are exact columns, so the superblock is the whole lattice."""
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    blk = exact_column_block(mdl)
    sb = Superblock(mdl, blk, blk)
    mask = sb.sector_mask((3, 3)).astype(float)
    v0 = mask * np.random.default_rng(0).standard_normal(sb.n_vec)
    e, x, _ = lanczos_ground(lambda v: mask * sb.apply(mask * v), v0, max_iter=300, tol=1e-12)
    return sb, e, x


def test_hubbard_densities_match_lattice_ed(hubbard_2x4_doped):
    sb, e, x = hubbard_2x4_doped
    e_ed, n_ed = ed_site_densities(2, 4, 3, 3)
    assert abs(e - e_ed) <= 1e-9 * abs(e_ed)
    got = site_densities(sb, x)
    assert np.allclose(got["n"], n_ed[1:3], atol=1e-8)   # columns 2, 3 = lattice x = 1, 2
    # the values themselves: two holes, more of them in the middle than at the ends
    assert np.allclose(got["h"], 1.0 - 2.0 * 0.355513, atol=1e-5)
    assert np.allclose(n_ed[[0, 3]], 0.394487, atol=1e-5)


def test_lieb_mattis_staggered_spin_density_vanishes(hubbard_2x4_doped):
    sb, _, x = hubbard_2x4_doped
    got = site_densities(sb, x)
    assert np.max(np.abs(got["sd"])) <= 1e-8 and np.max(got["S"]) <= 1e-8
    assert np.allclose(got["h"][0], got["h"][1], atol=1e-8)  # mirror symmetry of the ladder


def test_densities_equal_operator_expectation_values():
    """Independent route: <x| n_{y,s} acting on i2 (or i3) |x> with the column's number
    operator applied through Superblock's 4-index tensor, on a random vector with
    seeded blocks."""
    mdl = synth.model("hubbard", 2, t=1.0, U=4.0)
    sb = Superblock(mdl, synth.hubbard_block(5, 2, 1), synth.hubbard_block(7, 2, 2))
    x = np.random.default_rng(3).standard_normal(sb.n_vec)
    W = sb.tensor(x)
    got = site_densities(sb, x)
    norm = x @ x
    for y in range(2):
        for s in range(2):
            num = sb.col.cdag[y][s] @ sb.col.c[y][s]
            e2 = np.einsum("ajkl,bj,abkl->", W, num, W) / norm     # on i2
            e3 = np.einsum("ijkb,ab,ijka->", W, num, W) / norm     # on i3
            assert abs(got["n"][0, y, s] - e2) <= 1e-12
            assert abs(got["n"][1, y, s] - e3) <= 1e-12


def test_spin_columns_one_spin_per_site():
    mdl = synth.model("heisenberg", 3)
    sb = Superblock(mdl, synth.heisenberg_block(6, 3, 4), synth.heisenberg_block(5, 3, 5))
    x = np.random.default_rng(4).standard_normal(sb.n_vec)
    got = site_densities(sb, x)
    assert np.allclose(got["h"], 0.0, atol=1e-14)
    occ = column_occupations(sb.col)
    assert np.array_equal(occ.sum(axis=2), np.ones((sb.d, 3)))
    # s = 2 <S^z>: compare with S^z applied on i2
    W = sb.tensor(x)
    for y in range(3):
        e2 = np.einsum("ajkl,bj,abkl->", W, sb.col.Sz[y], W) / (x @ x)
        assert abs(got["sd"][0, y] - 2.0 * e2) <= 1e-12
