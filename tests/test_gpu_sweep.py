"""dmrg2d_sweep (finite-system direct 2-D DMRG on the GPU) against the oracle DMRG and ED.

* untruncated (every block keeps all its states): every finite-sweep step reproduces the
  ED ground energy of the 2 x 6 ladder;
* truncated, with the number of kept states chosen where the oracle's density-matrix
  spectrum has a gap at the cut (SU(2) multiplets are not split, so the kept subspace is
  unique): the per-step energies and truncation errors equal the oracle's;
* mixed precision (TF32 superblock H·v + FP64 refinement) on a 4-leg ladder gives the
  plain FP64 sweep's energies;
* the wavefunction transformation: untruncated, each carried-over ground state is the
  next superblock's ground state.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dmrg as odmrg  # noqa: E402
from oracle import lattice_ed  # noqa: E402
from paper_0707_0159_gb300 import dmrg2d, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def model(n, J_leg=1.0, J_rung=0.8):
    return synth.model("heisenberg", n, J_leg=J_leg, J_rung=J_rung)


def test_untruncated_sweep_equals_ed():
    mdl = model(2)
    out = dmrg2d.sweep(mdl, 6, m_warmup=64, m_sweeps=[64], precision="fp64", tol=1e-12,
                       max_iter=600)
    e_ed = float(lattice_ed.heisenberg_spectrum(2, 6, J_leg=1.0, J_rung=0.8)[0])
    e = np.array(out["energy"])
    sw = np.array(out["sweep"])
    assert np.allclose(e[sw >= 0], e_ed, rtol=0, atol=1e-9), (e, e_ed)
    assert max(out["trunc"]) <= 1e-12


@pytest.mark.parametrize("kind", ["dense", "sectors", "hubbard"])
def test_wavefunction_transformation_gives_the_next_ground_state(kind):
    """Without truncation the previous ground state, carried into the next superblock's
    basis, is that superblock's ground state: every finite step after the first (which
    starts from a random vector) converges at the first convergence check.  Dense
    superblocks, the S^z_tot = 0 sector (the label-by-label transformation of the packed
    state) and a Hubbard chain in its (N_up, N_dn) sector."""
    kw = dict(precision="fp64", tol=1e-10, max_iter=600)
    if kind == "hubbard":
        mdl = synth.model("hubbard", 1, t=1.0, U=4.0)
        kw.update(sectors=True, n_up=2, n_dn=2)
    else:
        mdl = model(2)
        kw.update(sectors=kind == "sectors")
    out = dmrg2d.sweep(mdl, 6, m_warmup=64, m_sweeps=[64, 64], **kw)
    sw = np.array(out["sweep"])
    it = np.array(out["iters"])[sw >= 0]
    assert it[0] > 10                      # seeded random start
    assert np.all(it[1:] <= 5), it         # one convergence check (every 5 steps)


@pytest.mark.parametrize("n,m", [(2, 8), (3, 16)])
def test_truncated_sweep_matches_oracle(n, m):
    mdl = model(n)
    ref = odmrg.dmrg(mdl, 6, m_warmup=m, m_sweeps=[m, m])
    assert min(ref["gap"]) > 1e-7          # the cut never splits a multiplet
    out = dmrg2d.sweep(mdl, 6, m_warmup=m, m_sweeps=[m, m], precision="fp64", tol=1e-12,
                       max_iter=800)
    assert out["n_steps"] == len(ref["energy"])
    assert out["l"] == ref["l"] and out["sweep"] == ref["sweep"]
    assert np.allclose(out["energy"], ref["energy"], rtol=1e-10, atol=0)
    assert np.allclose(out["trunc"], ref["trunc"], rtol=1e-5, atol=1e-12)


def test_mixed_precision_sweep_matches_fp64():
    mdl = model(4, J_rung=0.9)
    kw = dict(m_warmup=32, m_sweeps=[32], tol=1e-10, max_iter=600, krylov_dim=60)
    ref = dmrg2d.sweep(mdl, 6, precision="fp64", **kw)
    mix = dmrg2d.sweep(mdl, 6, precision="tf32", **kw)
    assert mix["l"] == ref["l"]
    # same kept subspaces as long as the density-matrix cuts are clean; energies agree
    assert np.allclose(mix["energy"], ref["energy"], rtol=1e-8, atol=0)


@pytest.mark.parametrize("n,m,L", [(2, 8, 6), (3, 16, 6), (2, 64, 6)])
def test_sector_sweep_matches_dense_sweep(n, m, L):
    """S^z_tot = 0 sector-restricted sweep (blocks labelled by N_up, density matrices per
    sector) against the dense sweep: same energies and truncation errors wherever the
    density-matrix cut has a gap (checked on the oracle), and exact when untruncated."""
    mdl = model(n)
    if m < 64:
        assert min(odmrg.dmrg(mdl, L, m_warmup=m, m_sweeps=[m, m])["gap"]) > 1e-7
    kw = dict(m_warmup=m, m_sweeps=[m, m], precision="fp64", tol=1e-12, max_iter=800)
    dense = dmrg2d.sweep(mdl, L, **kw)
    sec = dmrg2d.sweep(mdl, L, sectors=True, **kw)
    assert sec["l"] == dense["l"] and sec["sweep"] == dense["sweep"]
    assert np.allclose(sec["energy"], dense["energy"], rtol=1e-10, atol=0)
    assert np.allclose(sec["trunc"], dense["trunc"], rtol=1e-5, atol=1e-12)


@pytest.mark.parametrize("n,m,sectors", [(2, 8, False), (3, 16, True), (2, 64, True)])
def test_sweep_observables_match_oracle(n, m, sectors):
    """Per-step bond energies (leg bonds between the central columns, rung bonds of column
    2) and <S_tot^2> at the end of each sweep, against the oracle's
    measurements on its own DMRG run (same kept subspaces where the cuts have gaps)."""
    mdl = model(n)
    ref = odmrg.dmrg(mdl, 6, m_warmup=m, m_sweeps=[m, m])
    out = dmrg2d.sweep(mdl, 6, m_warmup=m, m_sweeps=[m, m], precision="fp64", tol=1e-12,
                       max_iter=800, sectors=sectors)
    assert out["l"] == ref["l"]
    assert np.allclose(np.array(out["leg_bond"]), np.array(ref["leg"]), rtol=0, atol=1e-8)
    if n > 1:
        assert np.allclose(np.array(out["rung_bond"]), np.array(ref["rung"]), rtol=0, atol=1e-8)
    s2 = np.array(out["s2"])
    measured = ~np.isnan(s2)
    assert measured.sum() == 2                   # the last step of each sweep
    assert np.allclose(s2[measured], np.array(ref["s2"])[measured], rtol=0, atol=1e-7)
    assert np.all(np.abs(s2[measured]) <= 1e-3)  # Lieb-Mattis: singlet ground state


# ---- Hubbard ladders (electrons, target (N_up, N_dn) sector) ---------------------------------

def _hubbard_exact(n_legs, L, n_up, n_dn, m, sweeps, last):
    from test_oracle_densities import ed_site_densities
    mdl = synth.model("hubbard", n_legs, t=1.0, U=8.0)
    out = dmrg2d.sweep(mdl, L, m, [m] * sweeps, sectors=True, n_up=n_up, n_dn=n_dn, tol=1e-11,
                       max_iter=400, krylov_dim=200)
    e_ed, n_ed = ed_site_densities(n_legs, L, n_up, n_dn)
    fin = [k for k, s in enumerate(out["sweep"]) if s >= last]
    assert len(fin) >= 5
    for k in fin:
        assert abs(out["energy"][k] - e_ed) <= 1e-9 * abs(e_ed), (k, out["energy"][k], e_ed)
        l = out["l"][k]
        assert np.allclose(out["n"][k], n_ed[l:l + 2], atol=1e-7), (k, l)
        assert np.allclose(out["h"][k], 1.0 - n_ed[l:l + 2].sum(axis=2), atol=1e-7)
        assert np.max(np.abs(out["sd"][k])) <= 1e-7 and np.max(out["S"][k]) <= 1e-7
    return out


def test_hubbard_ladder_sweep_equals_ed():
    """2 x 6 Hubbard ladder, U = 8, 1 up + 1 down electron, m = 16 (above the largest
    Schmidt rank, 14): the sweeps recover the states the warm-up did not keep (its density
    matrices cover only the sectors its smaller superblocks' targets reach), and the last
    sweep reproduces ED at every step: energy, the central columns' hole density and the
    vanishing staggered spin density."""
    _hubbard_exact(2, 6, 1, 1, 16, 4, 3)


def test_hubbard_chain_sweep_equals_ed_at_every_step():
    """1 x 6 Hubbard chain, U = 8, 2 up + 2 down electrons, m = 64 (every state kept).
    The warm-up's 4-site superblock targets the rounded filling (1, 1), so labels such as
    (2, 0) carry no weight there; the blocks keep their states with weight 0, as the oracle
    does, and every finite step then reproduces ED (energy, densities), the warm-up step
    the oracle's energy."""
    from oracle import dmrg_fermion as odf
    from test_oracle_densities import ed_site_densities
    mdl = synth.model("hubbard", 1, t=1.0, U=8.0)
    out = dmrg2d.sweep(mdl, 6, 64, [64, 64], sectors=True, n_up=2, n_dn=2, tol=1e-12,
                       max_iter=400, krylov_dim=200)
    ref = odf.dmrg(mdl, 6, 2, 2, m_warmup=64, m_sweeps=[64, 64])
    e_ed, n_ed = ed_site_densities(1, 6, 2, 2)
    warm = [k for k, s in enumerate(out["sweep"]) if s < 0]
    fin = [k for k, s in enumerate(out["sweep"]) if s >= 0]
    assert len(warm) == 1 and len(fin) == 2 * 5
    assert abs(out["energy"][warm[0]] - ref["energy"][0]) <= 1e-10 * abs(ref["energy"][0])
    for k in fin:
        assert abs(out["energy"][k] - e_ed) <= 1e-9 * abs(e_ed), (k, out["energy"][k], e_ed)
        assert out["trunc"][k] <= 1e-12
        l = out["l"][k]
        assert np.allclose(out["n"][k], n_ed[l:l + 2], atol=1e-7), (k, l)
        assert np.max(np.abs(out["sd"][k])) <= 1e-7


@pytest.mark.parametrize("n_up,n_dn,m", [(3, 2, 8), (2, 1, 6)])
def test_truncated_hubbard_ladder_sweep_matches_oracle(n_up, n_dn, m):
    """2 x 6 Hubbard ladder, U = 8, truncated to m states, where every cut of the oracle's
    run falls in a gap of the density-matrix spectrum (kept weight >= 1e-4, relative gap
    >= 0.17 at (3, 2), m = 8; >= 8e-4 and 0.33 at (2, 1), m = 6): the kept subspaces are
    unique, so the GPU sweep equals the oracle step by step (energies, truncation errors,
    densities).  The oracle also records the full-lattice superblock at the end of its
    warm-up, which the library measures as the first step of sweep 0."""
    from oracle import dmrg_fermion as odf
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    out = dmrg2d.sweep(mdl, 6, m, [m, m], sectors=True, n_up=n_up, n_dn=n_dn, tol=1e-12,
                       max_iter=600, krylov_dim=200)
    ref = odf.dmrg(mdl, 6, n_up, n_dn, m_warmup=m, m_sweeps=[m, m])
    keep = [k for k in range(len(ref["l"])) if not (ref["sweep"][k] < 0 and ref["l"][k] == 2)]
    assert out["l"] == [ref["l"][k] for k in keep]
    assert out["sweep"] == [ref["sweep"][k] for k in keep]
    for i, k in enumerate(keep):
        assert abs(out["energy"][i] - ref["energy"][k]) <= 1e-9 * abs(ref["energy"][k]), \
            (i, out["energy"][i], ref["energy"][k])
        last_of_sweep = k + 1 == len(ref["l"]) or ref["sweep"][k + 1] != ref["sweep"][k]
        if not last_of_sweep:   # the oracle records 0 at its measure-only middle step
            assert abs(out["trunc"][i] - ref["trunc"][k]) <= 1e-9, \
                (i, out["trunc"][i], ref["trunc"][k])
        assert np.allclose(out["n"][i], np.asarray(ref["n"][k]), atol=1e-7), i


@pytest.mark.parametrize("kind", ["heisenberg", "hubbard"])
def test_sweep_state_continues_across_calls(kind):
    """dmrg2d_state: one sweep per call on one state, twice, does what one call of two
    sweeps does (same steps, energies, truncation errors); the second call starts from the
    ground state the first one left and continues the sweep index; lattice fields that
    differ from the state's are refused."""
    if kind == "heisenberg":
        mdl, kw = model(2), dict(sectors=True)
    else:
        mdl, kw = synth.model("hubbard", 2, t=1.0, U=8.0), dict(sectors=True, n_up=3, n_dn=2)
    solve = dict(tol=1e-12, max_iter=600, krylov_dim=120)
    once = dmrg2d.sweep(mdl, 6, 8, [8, 12], **kw, **solve)
    st = dmrg2d.SweepState(mdl, 6, 8, **kw)
    a = st.sweep([8], **solve)
    assert st.info()["sweeps_done"] == 1 and st.info()["warmed_up"] == 1
    b = st.sweep([12], **solve)
    info = st.info()
    assert info["sweeps_done"] == 2 and abs(info["last_energy"] - once["energy"][-1]) <= 1e-12
    both = {k: a[k] + b[k] for k in ("energy", "trunc", "l", "sweep")}
    assert both["l"] == once["l"] and both["sweep"] == once["sweep"]
    assert max(s for s in b["sweep"]) == 1 and min(s for s in b["sweep"]) == 1
    assert np.allclose(both["energy"], once["energy"], rtol=0, atol=1e-11)
    assert np.allclose(both["trunc"], once["trunc"], rtol=0, atol=1e-11)
    # b's first step starts from a's last ground state: few solver steps
    assert b["iters"][0] <= once["iters"][len(a["energy"])] + 2
    bad = dmrg2d.SweepState(mdl, 6, 8, **kw)
    bad._fixed["n_columns"] = 8                 # a call whose lattice differs from the state
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        bad.sweep([8], **solve)
    assert e.value.code == -1
    st.free()
    bad.free()


@pytest.mark.parametrize("n,m", [(2, 8), (3, 16)])
def test_davidson_sweep_matches_oracle(n, m):
    """The sweep with the Davidson solver (Jacobi preconditioner) in place of Lanczos gives
    the oracle's energies and truncation errors step by step."""
    mdl = model(n)
    ref = odmrg.dmrg(mdl, 6, m_warmup=m, m_sweeps=[m, m])
    assert min(ref["gap"]) > 1e-7
    out = dmrg2d.sweep(mdl, 6, m_warmup=m, m_sweeps=[m, m], precision="fp64", tol=1e-12,
                       max_iter=800, krylov_dim=32, solver="davidson", precond="jacobi")
    assert out["l"] == ref["l"] and out["sweep"] == ref["sweep"]
    assert np.allclose(out["energy"], ref["energy"], rtol=1e-10, atol=0)
    assert np.allclose(out["trunc"], ref["trunc"], rtol=1e-5, atol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "tf32"])
def test_learned_preconditioner_trains_inside_the_sweep(precision):
    """Davidson with the learned preconditioner in a sector sweep: the network trains on
    the Jacobi solves of the warm-up and the first sweep (its parameters change, the time
    is reported apart), the later sweeps precondition with it, and every step's energy is
    the oracle's (2 x 8 ladder, m = 8 then 16: the density-matrix cuts have gaps, so the
    kept subspaces are unique), as are those of the Jacobi and Lanczos sweeps."""
    mdl = model(2)
    ms = dict(m_warmup=8, m_sweeps=[8, 16, 16])
    ref = odmrg.dmrg(mdl, 8, **ms)
    assert min(ref["gap"]) > 1e-7
    kw = dict(**ms, precision=precision, tol=1e-11, max_iter=800, krylov_dim=32,
              sectors=True, solver="davidson")
    jac = dmrg2d.sweep(mdl, 8, precond="jacobi", **kw)
    net = dmrg2d.MLP(hidden=64, seed=3)
    p0 = net.get_params()
    lrn = dmrg2d.sweep(mdl, 8, precond="mlp", mlp=net, mlp_train_sweeps=1, mlp_epochs=2, **kw)
    assert lrn["train_seconds"] > 0 and jac["train_seconds"] == 0
    p1 = net.get_params()
    assert np.all(np.isfinite(p1)) and not np.array_equal(p1, p0)
    lan = dmrg2d.sweep(mdl, 8, **{k: v for k, v in kw.items() if k != "solver"})
    # a network used as given (no training) leaves its parameters alone
    lrn2 = dmrg2d.sweep(mdl, 8, precond="mlp", mlp=net, mlp_epochs=0, **kw)
    assert np.array_equal(net.get_params(), p1) and lrn2["train_seconds"] == 0
    for out in (jac, lrn, lan, lrn2):
        assert out["l"] == ref["l"] and out["sweep"] == ref["sweep"]
        assert np.allclose(out["energy"], ref["energy"], rtol=1e-9, atol=0)
