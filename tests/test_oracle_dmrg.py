"""Pins of the oracle's finite-system direct 2-D DMRG (CPU).

* untruncated DMRG is exact: every step on a 2 x 4 and a 2 x 6 ladder whose blocks keep
  all their states reproduces the brute-force ED ground energy;
* truncated DMRG is variational: every energy lies above the ED ground energy, and the
  finite sweeps lower the warm-up energy;
* the density-matrix truncation error is 1 - (kept weight) and vanishes without truncation.
"""
import numpy as np
import pytest

from oracle import dmrg, lattice_ed
from paper_0707_0159_gb300 import synth


def ladder_model(J_leg=1.0, J_rung=0.8):
    return synth.model("heisenberg", 2, J_leg=J_leg, J_rung=J_rung)


def ed_ground(mdl, L):
    return float(lattice_ed.heisenberg_spectrum(2, L, J_leg=mdl["J_leg"], J_rung=mdl["J_rung"])[0])


def test_untruncated_2x4_equals_ed():
    mdl = ladder_model()
    out = dmrg.dmrg(mdl, 4, m_warmup=64, m_sweeps=[64])
    e_ed = ed_ground(mdl, 4)
    assert np.allclose(out["energy"], e_ed, rtol=0, atol=1e-10)
    assert max(out["trunc"]) <= 1e-12


def test_untruncated_2x6_equals_ed():
    mdl = ladder_model()
    out = dmrg.dmrg(mdl, 6, m_warmup=64, m_sweeps=[64])
    # the warm-up step is the 2 x 4 superblock; every finite-sweep step spans 2 x 6
    sweep = np.array(out["sweep"])
    e = np.array(out["energy"])
    assert np.isclose(e[sweep == -1][0], ed_ground(mdl, 4), rtol=0, atol=1e-10)
    assert np.allclose(e[sweep >= 0], ed_ground(mdl, 6), rtol=0, atol=1e-9)
    assert max(out["trunc"]) <= 1e-12


def test_truncated_2x6_is_variational_and_sweeps_improve():
    mdl = ladder_model()
    e_ed = ed_ground(mdl, 6)
    out = dmrg.dmrg(mdl, 6, m_warmup=6, m_sweeps=[6, 6])
    e = np.array(out["energy"])
    sweep = np.array(out["sweep"])
    assert np.all(e[sweep >= 0] >= e_ed - 1e-10)
    assert e[sweep == 1].min() <= e[sweep == 0].min() + 1e-12
    assert max(out["trunc"]) > 0.0
    # more states, closer to ED
    out12 = dmrg.dmrg(mdl, 6, m_warmup=12, m_sweeps=[12, 12])
    e12 = np.array(out12["energy"])[np.array(out12["sweep"]) >= 0]
    assert e12.min() <= e[sweep >= 0].min() + 1e-12
    assert e12.min() - e_ed < 0.05 * abs(e_ed)


def test_keep_states_weights():
    rng = np.random.default_rng(0)
    V = rng.standard_normal((12, 9))
    V /= np.linalg.norm(V)
    U, w, trunc, gap = dmrg.keep_states(V @ V.T, 4)
    full = np.linalg.eigvalsh(V @ V.T)[::-1]
    assert np.allclose(w, full[:4])
    assert trunc == pytest.approx(1.0 - full[:4].sum())
    assert np.allclose(U.T @ U, np.eye(4), atol=1e-12)
    assert gap == pytest.approx(full[3] - full[4])


def test_ed_bond_energies_and_lieb_mattis():
    # the bond expectations reproduce the energy; the ground state is a singlet
    n, L = 2, 4
    mdl = ladder_model()
    e, psi, corr, s2 = lattice_ed.heisenberg_ground_correlations(n, L, J_leg=1.0, J_rung=0.8)
    total = 0.0
    for a, b, kind in lattice_ed.ladder_bonds(n, L):
        total += (mdl["J_leg"] if kind == "leg" else mdl["J_rung"]) * corr(a, b)
    assert total == pytest.approx(e, abs=1e-12)
    assert abs(s2) <= 1e-10
    assert corr(0, 0) == pytest.approx(0.75)


def test_untruncated_observables_equal_ed():
    """Leg bonds between the central columns, rung bonds of column 2 and <S^2> of every
    finite-sweep step of an untruncated 2 x 6 sweep equal the ED values of those bonds."""
    n, L = 2, 6
    mdl = ladder_model()
    out = dmrg.dmrg(mdl, L, m_warmup=64, m_sweeps=[64])
    _, _, corr, s2 = lattice_ed.heisenberg_ground_correlations(n, L, J_leg=1.0, J_rung=0.8)
    assert abs(s2) <= 1e-10
    for k, sw in enumerate(out["sweep"]):
        if sw < 0:
            continue
        x2 = out["l"][k]                        # lattice column of column 2 (0-based)
        for y in range(n):
            assert out["leg"][k][y] == pytest.approx(corr(x2 * n + y, (x2 + 1) * n + y), abs=1e-9)
        for y in range(n - 1):
            assert out["rung"][k][y] == pytest.approx(corr(x2 * n + y, x2 * n + y + 1), abs=1e-9)
        assert abs(out["s2"][k]) <= 1e-8
