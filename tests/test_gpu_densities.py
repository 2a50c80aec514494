"""Site densities of the two central columns on the GPU (dmrg2d_site_densities) against
the oracle: dense and sector-packed vectors, the bench-size superblock, and the doped
2 x 4 Hubbard ladder solved on the GPU against brute-force ED (the paper's hole density
and the Lieb-Mattis zero of the staggered spin density)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.densities import exact_column_block, site_densities as oracle_densities  # noqa: E402
from oracle.superblock import Superblock  # noqa: E402
from paper_0707_0159_gb300 import dmrg2d, synth  # noqa: E402

from test_oracle_densities import ed_site_densities  # noqa: E402

pytestmark = pytest.mark.gpu


def gpu(ops, x):
    return dmrg2d.site_densities(ops, torch.from_numpy(np.ascontiguousarray(x)).cuda())


def close(got, ref, atol):
    for k in ("n", "h", "sd", "S"):
        assert np.allclose(got[k], ref[k], atol=atol, rtol=0), (k, got[k], ref[k])


@pytest.mark.parametrize("case", [("hubbard", 2, 33, 20), ("hubbard", 3, 8, 5),
                                  ("heisenberg", 3, 40, 24), ("heisenberg", 4, 17, 9),
                                  ("hubbard", 2, 1, 1), ("heisenberg", 2, 1, 6)])
def test_dense_random_vector(case):
    """Including the lattice ends: one-state blocks without boundary operators."""
    kind, nl, m1, m4 = case
    mdl = synth.model(kind, nl, J_leg=0.8, J_rung=1.1, t=1.0, U=6.0)
    mk = synth.heisenberg_block if kind == "heisenberg" else synth.hubbard_block
    left = mk(m1, nl, 1) if m1 > 1 else synth.empty_block(kind)
    right = mk(m4, nl, 2) if m4 > 1 else synth.empty_block(kind)
    ops = dmrg2d.build_ops(mdl, left, right)
    sb = Superblock(mdl, left, right)
    x = synth.start_vector(sb.n_vec, 9)
    close(gpu(ops, x), oracle_densities(sb, x), 1e-12)


@pytest.mark.parametrize("name", ["heisenberg_4leg", "hubbard_3leg"])
def test_sector_packed_vector(name):
    if name == "heisenberg_4leg":
        mdl, left, right, target = synth.workload_ladder4_heisenberg_sectors(m=48, block_sites=8)
    else:
        mdl, left, right, target = synth.workload_ladder3_hubbard_sectors(m=40, block_sites=6,
                                                                          n_up=6, n_dn=6)
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    sb = Superblock(mdl, left, right)
    idx = dmrg2d.sector_dense_index(ops)
    valid = idx >= 0
    xp = np.where(valid, synth.start_vector(len(idx), 13), 0.0)
    xd = np.zeros(sb.n_vec)
    xd[idx[valid]] = xp[valid]
    close(gpu(ops, xp), oracle_densities(sb, xd), 1e-12)


def test_bench_size_superblock():
    """The 3-leg Hubbard superblock of the benchmark (V 16384 x 16384, 2.7e8 entries)."""
    mdl, left, right, _ = synth.workload_ladder3_hubbard_m256()
    ops = dmrg2d.build_ops(mdl, left, right)
    sb = Superblock(mdl, left, right)
    x = synth.start_vector(sb.n_vec, 12)
    close(gpu(ops, x), oracle_densities(sb, x), 1e-12)


def grouped_by_label(blk):
    """The same block in a basis whose states are grouped by quantum-number label (the
    layout sector-restricted superblocks take): a permutation of the basis."""
    qn = np.asarray(blk["qn"])
    p = np.lexsort(qn.T[::-1])
    out = dict(blk)
    out["H"] = blk["H"][np.ix_(p, p)]
    out["edge"] = [e[np.ix_(p, p)] for e in blk["edge"]]
    out["qn"] = np.ascontiguousarray(qn[p])
    if "parity" in blk:
        out["parity"] = np.asarray(blk["parity"])[p]
    return out


def test_doped_hubbard_ladder_ground_state_against_ed():
    """2 x 4 Hubbard ladder (t = 1, U = 8), 3 up + 3 down electrons, blocks 1 and 4 exact
    columns: the GPU ground state's densities on columns 2, 3 equal the lattice ED's at
    x = 1, 2; the staggered spin density vanishes (Lieb-Mattis)."""
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    blk = grouped_by_label(exact_column_block(mdl))
    ops = dmrg2d.build_ops(mdl, blk, blk, target=(3, 3))
    idx = dmrg2d.sector_dense_index(ops)
    x0 = np.where(idx >= 0, synth.start_vector(len(idx), 2), 0.0)
    x = torch.from_numpy(x0).cuda()
    e, st, code = dmrg2d.lanczos_ground(ops, x, tol=1e-12, max_iter=400, krylov_dim=200)
    e_ed, n_ed = ed_site_densities(2, 4, 3, 3)
    assert code == 0 and abs(e - e_ed) <= 1e-9 * abs(e_ed)
    got = dmrg2d.site_densities(ops, x)
    assert np.allclose(got["n"], n_ed[1:3], atol=1e-7)
    assert np.allclose(got["h"], 1.0 - n_ed[1:3].sum(axis=2), atol=1e-7)
    assert np.max(np.abs(got["sd"])) <= 1e-7 and np.max(got["S"]) <= 1e-7
