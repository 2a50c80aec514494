"""Sector-restricted (quantum-number) superblocks on the GPU against the oracle.

The packed layout is rebuilt here from its documented rule (include/dmrg2d.h), not
taken from the library: for every combined left label qL in increasing order, a
column-major matrix whose rows are, for i2 = 0..d-1, the block-1 sector with label
qL - q(i2) padded to a multiple of 8 rows, and whose columns are, for i3 = 0..d-1,
the block-4 sector with label Q - qL - q(i3).  The oracle applies the full H to the
dense vector; the sector part must match to 1e-12 (FP64) and padding must stay zero.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.solvers import lanczos_ground as oracle_lanczos  # noqa: E402
from oracle.superblock import Superblock  # noqa: E402
from paper_0707_0159_gb300 import dmrg2d, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def runs(qn):
    out = []
    i = 0
    qn = [tuple(int(x) for x in r) for r in np.asarray(qn)]
    while i < len(qn):
        j = i + 1
        while j < len(qn) and qn[j] == qn[i]:
            j += 1
        out.append((qn[i], i, j - i))
        i = j
    return {lab: (first, dim) for lab, first, dim in out}


def packed_map(sb, target):
    """dense index of every packed position (-1 for padding), from the documented rule."""
    m1, d, m4 = sb.m1, sb.d, sb.m4
    s1, s4 = runs(sb.left["qn"]), runs(sb.right["qn"])
    qc = [tuple(int(x) for x in r) for r in sb.column_labels()]
    Q = tuple(int(x) for x in target)
    sub = lambda a, b: tuple(x - y for x, y in zip(a, b))
    addl = lambda a, b: tuple(x + y for x, y in zip(a, b))
    qls = set()
    for i2 in range(d):
        for lab in s1:
            qL = addl(lab, qc[i2])
            if any(sub(sub(Q, qL), qc[i3]) in s4 for i3 in range(d)):
                qls.add(qL)
    out = []
    for qL in sorted(qls):
        rows = [(i2, *s1[sub(qL, qc[i2])]) for i2 in range(d) if sub(qL, qc[i2]) in s1]
        cols = [(i3, *s4[sub(sub(Q, qL), qc[i3])]) for i3 in range(d)
                if sub(sub(Q, qL), qc[i3]) in s4]
        row_idx = []
        for i2, first, dim in rows:
            pad = (dim + 7) // 8 * 8
            row_idx += [(i2, first + i) for i in range(dim)] + [None] * (pad - dim)
        for i3, first, dim in cols:
            for j in range(dim):
                i4 = first + j
                for r in row_idx:
                    if r is None:
                        out.append(-1)
                    else:
                        i2, i1 = r
                        out.append(i1 + m1 * i2 + m1 * d * i4 + m1 * d * m4 * i3)
    return np.array(out, dtype=np.int64)


CASES = {
    "heisenberg_4leg": lambda: synth.workload_ladder4_heisenberg_sectors(m=48, block_sites=8),
    "hubbard_3leg": lambda: synth.workload_ladder3_hubbard_sectors(m=25, block_sites=6,
                                                                    n_up=6, n_dn=6),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def sector_case(request):
    mdl, left, right, target = CASES[request.param]()
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    pmap = packed_map(sb, target)
    return request.param, mdl, left, right, target, sb, ops, pmap


def test_layout_matches_documented_rule(sector_case):
    name, mdl, left, right, target, sb, ops, pmap = sector_case
    assert ops.info["n_vec"] == len(pmap)
    mask = sb.sector_mask(target)
    valid = pmap[pmap >= 0]
    assert len(np.unique(valid)) == len(valid) == mask.sum()   # a bijection onto the sector
    assert np.all(mask[valid])
    lib_map = dmrg2d.sector_dense_index(ops)
    assert np.array_equal(lib_map, pmap)


@pytest.mark.parametrize("prec,tol", [(dmrg2d.FP64, 1e-12), (dmrg2d.FP64X, 1e-12),
                                      (dmrg2d.FP32, 1e-5)])
def test_sector_hv_matches_oracle(sector_case, prec, tol):
    name, mdl, left, right, target, sb, ops, pmap = sector_case
    valid = pmap >= 0
    vp = np.where(valid, synth.start_vector(len(pmap), 31), 0.0)
    vd = np.zeros(sb.n_vec)
    vd[pmap[valid]] = vp[valid]
    yd = sb.apply(vd)
    ref = np.zeros(len(pmap))
    ref[valid] = yd[pmap[valid]]
    dt = torch.float64 if prec in (dmrg2d.FP64, dmrg2d.FP64X) else torch.float32
    x = torch.from_numpy(vp).to("cuda", dt)
    y = torch.full((len(pmap),), 7.0, dtype=dt, device="cuda")   # padding must be overwritten
    dmrg2d.apply_H(ops, x, y, prec)
    torch.cuda.synchronize()
    got = y.double().cpu().numpy()
    assert np.all(got[~valid] == 0.0)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= tol, err
    # the oracle's H keeps the sector closed, so nothing was dropped by the restriction
    assert np.linalg.norm(yd[~sb.sector_mask(target)]) == 0.0


def test_sector_flops_count_only_sector_work(sector_case):
    name, mdl, left, right, target, sb, ops, pmap = sector_case
    dense = dmrg2d.build_ops(mdl, left, right)
    assert 0 < ops.info["flops_per_apply"] < dense.info["flops_per_apply"]


def test_sector_lanczos_matches_dense_solver(sector_case):
    """Sector Lanczos against dense Lanczos started from the same (sector) vector.

    A Krylov space built from a vector inside the sector never leaves it, so the
    dense solver (itself pinned to the oracle) reaches the sector ground state.
    """
    name, mdl, left, right, target, sb, ops, pmap = sector_case
    valid = pmap >= 0
    vp = np.where(valid, synth.start_vector(len(pmap), 8), 0.0)
    x = torch.from_numpy(vp).cuda()
    e, st, code = dmrg2d.lanczos_ground(ops, x, max_iter=800, krylov_dim=300, tol=1e-10)
    assert code == 0, st
    vd = np.zeros(sb.n_vec)
    vd[pmap[valid]] = vp[valid]
    dense = dmrg2d.build_ops(mdl, left, right)
    xd = torch.from_numpy(vd).cuda()
    e_d, st_d, code_d = dmrg2d.lanczos_ground(dense, xd, max_iter=800, krylov_dim=300, tol=1e-10)
    assert code_d == 0, st_d
    assert abs(e - e_d) <= 1e-9 * abs(e_d), (e, e_d)
    # the returned vector is an eigenvector of the oracle's H (residual check, dense space)
    xs = x.cpu().numpy()
    xv = np.zeros(sb.n_vec)
    xv[pmap[valid]] = xs[valid]
    r = sb.apply(xv) - e * xv
    assert np.linalg.norm(r) <= 1e-6 * abs(e)


def test_tiny_sector_lanczos_matches_oracle():
    # 2-leg Hubbard, blocks of 12 states in 9 (N_up, N_dn) sectors, 12 sites at 5 up 6 down
    grid = [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)]
    offs, sizes = synth.sector_sizes(grid, (1.0, 1.0), 12, 4, lo=1)
    lab = synth.labels_from_sectors((2, 2), offs, sizes)
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    left, right = synth.hubbard_block(12, 2, 4, lab), synth.hubbard_block(12, 2, 5, lab)
    target = (5, 6)
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    pmap = packed_map(sb, target)
    valid = pmap >= 0
    vp = np.where(valid, synth.start_vector(len(pmap), 2), 0.0)
    x = torch.from_numpy(vp).cuda()
    e, st, code = dmrg2d.lanczos_ground(ops, x, max_iter=300, krylov_dim=300, tol=1e-11)
    assert code == 0, st
    vd = np.zeros(sb.n_vec)
    vd[pmap[valid]] = vp[valid]
    e_ref, _, info = oracle_lanczos(sb.apply, vd, max_iter=300, tol=1e-11)
    assert abs(e - e_ref) <= 1e-9 * abs(e_ref), (e, e_ref)


def test_sector_mixed_solver_with_float_pair_refinement(sector_case):
    """The mixed solver on a sector superblock with its outer-loop H·v in float pairs
    (FP64X) reaches the plain FP64 Lanczos energy from the same start vector."""
    name, mdl, left, right, target, sb, ops, pmap = sector_case
    valid = pmap >= 0
    vp = np.where(valid, synth.start_vector(len(pmap), 8), 0.0)
    x64 = torch.from_numpy(vp).cuda()
    e64, st64, c64 = dmrg2d.lanczos_ground(ops, x64, max_iter=800, krylov_dim=300, tol=1e-11)
    assert c64 == 0, st64
    low = dmrg2d.TF32 if ops.info["tc_ok"] else dmrg2d.FP32
    x = torch.from_numpy(vp).cuda()
    e, st, code = dmrg2d.lanczos_ground(ops, x, precision=low, refine=1, tol=1e-9,
                                        inner_iter=60, outer_max=40,
                                        refine_precision=dmrg2d.FP64X)
    assert code == 0, st
    assert st["n_hv_fp64"] > 0
    assert abs(e - e64) <= 1e-9 * abs(e64), (e, e64)
    assert np.all(x.cpu().numpy()[~valid] == 0.0)
