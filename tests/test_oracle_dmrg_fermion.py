"""Pins of the oracle's Hubbard DMRG sweep: untruncated sweeps reproduce brute-force ED
(energy and site densities of every measured column), truncated sweeps are variational
and converge towards ED, the staggered spin density vanishes (Lieb-Mattis), and the
kept states have definite labels and parities."""
import numpy as np
import pytest

from oracle import dmrg_fermion as D
from oracle.densities import exact_column_block
from paper_0707_0159_gb300 import synth

from test_oracle_densities import ed_site_densities


@pytest.fixture(scope="module")
def chain6():
    """1 x 6 Hubbard chain, U = 8, 2 up + 2 down electrons; m = 64 keeps every state
    (no cut has more than 3 sites on its small side)."""
    mdl = synth.model("hubbard", 1, t=1.0, U=8.0)
    return mdl, D.dmrg(mdl, 6, 2, 2, m_warmup=64, m_sweeps=[64, 64])


def test_untruncated_sweep_equals_ed(chain6):
    mdl, out = chain6
    e_ed, n_ed = ed_site_densities(1, 6, 2, 2)
    fin = [k for k, s in enumerate(out["sweep"]) if s >= 0]
    assert len(fin) == 2 * 5  # per sweep: 1 step right, 2 left, 1 back, the middle measured
    for k in fin:
        assert abs(out["energy"][k] - e_ed) <= 1e-10 * abs(e_ed)
        assert out["trunc"][k] <= 1e-12
        l = out["l"][k]
        assert np.allclose(out["n"][k], n_ed[l:l + 2], atol=1e-8), (k, l)
        assert np.max(np.abs(out["sd"][k])) <= 1e-8


def test_untruncated_2x6_ladder_equals_ed():
    """2 x 6 Hubbard ladder (two legs: every boundary operator of the enlarged blocks is
    exercised), U = 8, one up and one down electron: no cut carries more than
    1 + 6 + 6 + 1 = 14 Schmidt states, so m = 16 keeps all of them: the sweeps recover
    what the warm-up's smaller superblocks did not need, and the third sweep reproduces
    ED at every step."""
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    out = D.dmrg(mdl, 6, 1, 1, m_warmup=16, m_sweeps=[16, 16, 16])
    e_ed, n_ed = ed_site_densities(2, 6, 1, 1)
    fin = [k for k, s in enumerate(out["sweep"]) if s == 2]
    assert out["energy"][-1] <= out["energy"][1] + 1e-12  # the sweeps only lower it
    for k in fin:
        assert abs(out["energy"][k] - e_ed) <= 1e-10 * abs(e_ed)
        l = out["l"][k]
        assert np.allclose(out["n"][k], n_ed[l:l + 2], atol=1e-8), (k, l)


def test_truncated_sweeps_are_variational_and_depolarise_with_m():
    """1 x 10 Hubbard chain, U = 8, 4 up + 4 down electrons, m = 6 and 12: every energy
    lies above ED and m = 12 comes closer; the staggered spin density of the truncated
    state, clearly non-zero at m = 6, shrinks with m (the convergence to the unpolarised
    Lieb-Mattis pattern that the paper reports for its ladders)."""
    import scipy.sparse.linalg as spla
    from oracle.lattice_ed import hubbard_sector_matrix
    mdl = synth.model("hubbard", 1, t=1.0, U=8.0)
    e_ed = spla.eigsh(hubbard_sector_matrix(1, 10, 4, 4, 1.0, 8.0), k=1, which="SA",
                      tol=1e-13)[0][0]
    res = {}
    for m in (6, 12):
        out = D.dmrg(mdl, 10, 4, 4, m_warmup=m, m_sweeps=[m, m])
        fin = [k for k, s in enumerate(out["sweep"]) if s >= 0]
        assert min(out["energy"][k] for k in fin) >= e_ed - 1e-10
        res[m] = (out["energy"][fin[-1]], float(np.max(out["S"][fin[-1]])))
    assert res[12][0] < res[6][0] and abs(res[12][0] - e_ed) <= 5e-3 * abs(e_ed)
    assert res[6][1] > 1e-2 and res[12][1] < 0.1 * res[6][1]


def test_kept_states_have_definite_labels():
    mdl = synth.model("hubbard", 1, t=1.0, U=4.0)
    enl = D.enlarge_left(mdl, exact_column_block(mdl))
    rng = np.random.default_rng(1)
    A = rng.standard_normal((enl["m"], enl["m"]))
    # a label-conserving density matrix: zero the blocks between different labels
    same = (enl["qn"][:, None, :] == enl["qn"][None, :, :]).all(axis=2)
    rho = (A @ A.T) * same
    rho /= np.trace(rho)
    U, lab, tr = D.keep_states(rho, enl["qn"], 7)
    assert U.shape == (enl["m"], 7) and np.allclose(U.T @ U, np.eye(7), atol=1e-12)
    for j in range(7):
        support = np.flatnonzero(np.abs(U[:, j]) > 1e-14)
        assert (enl["qn"][support] == lab[j]).all()
    w = np.linalg.eigvalsh(rho)[::-1]
    assert abs(tr - (1.0 - w[:7].sum())) <= 1e-12
