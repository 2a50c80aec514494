"""Grouped tensor-core H·v (work list over row x column segments) against the oracle.

Covers every tile configuration on dense superblocks whose block sizes the dense
kernel cannot take (m not a multiple of 128), the dense kernel against the grouped
one on the same superblock, sector-restricted superblocks in TF32 and BF16, the
autotuner, and the sign-deduplicated operator pool (H_l/H_r blocks stored once).
Tolerances as for the dense tensor-core tests: TF32 <= 1e-3, BF16 <= 6e-3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.superblock import Superblock  # noqa: E402
from paper_0707_0159_gb300 import dmrg2d, synth  # noqa: E402

from test_gpu_sectors import packed_map  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = {dmrg2d.TF32: 1e-3, dmrg2d.BF16: 6e-3, dmrg2d.BF16X3: 1e-4}


def make(kind, n_legs, m1, m4, seed=0):
    mdl = synth.model(kind, n_legs, J_leg=0.8, J_rung=1.1, t=1.0, U=6.0)
    mk = synth.heisenberg_block if kind == "heisenberg" else synth.hubbard_block
    return mdl, mk(m1, n_legs, seed + 1), mk(m4, n_legs, seed + 2)


def run(ops, v, prec):
    x = torch.from_numpy(v).cuda()
    if prec == dmrg2d.BF16X3:
        x = dmrg2d.convert_input(x, prec)
    else:
        x = x.float() if prec == dmrg2d.TF32 else x.bfloat16()
    y = torch.full((v.size,), 3.0, dtype=torch.float32, device="cuda")
    dmrg2d.apply_H(ops, x, y, prec)
    torch.cuda.synchronize()
    dmrg2d.check_device(ops)
    return y.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", [("hubbard", 2, 72, 40), ("heisenberg", 3, 136, 264)])
@pytest.mark.parametrize("prec", [dmrg2d.TF32, dmrg2d.BF16])
def test_grouped_dense_every_config(case, prec):
    mdl, left, right = make(*case)
    ops = dmrg2d.build_ops(mdl, left, right)
    assert ops.info["tc_ok"] == 1
    sb = Superblock(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 3)
    ref = sb.apply(v)
    with pytest.raises(dmrg2d.Dmrg2dError):
        dmrg2d.set_tile_config(ops, prec, 0)   # the dense kernel does not take these shapes
    for cfg in range(1, 7):
        dmrg2d.set_tile_config(ops, prec, cfg)
        err = rel(run(ops, v, prec), ref)
        assert err <= TOL[prec], (cfg, dmrg2d.tile_config_name(cfg), err)


@pytest.mark.parametrize("prec", [dmrg2d.TF32, dmrg2d.BF16])
def test_dense_and_grouped_kernels_agree(prec):
    mdl, left, right = make("hubbard", 2, 128, 256)
    ops = dmrg2d.build_ops(mdl, left, right)
    sb = Superblock(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 4)
    ref = sb.apply(v)
    out = {}
    for cfg in (0, 1, 4, 7, 8, 9, 20, 24):
        dmrg2d.set_tile_config(ops, prec, cfg)
        out[cfg] = run(ops, v, prec)
        assert rel(out[cfg], ref) <= TOL[prec]
    # same operands, same K order within a piece: the kernels agree far below the tolerance
    # (config 20, two passes, rounds the first pass's partial sum to FP32 once more)
    for cfg in (1, 4, 7, 8, 9, 20, 24):
        assert rel(out[cfg], out[0]) <= (2e-5 if cfg == 20 else 1e-6), cfg


@pytest.mark.parametrize("case", [("heisenberg", 3, 256, 256), ("hubbard", 1, 512, 512),
                                  ("heisenberg", 2, 256, 512)])
@pytest.mark.parametrize("prec", [dmrg2d.TF32, dmrg2d.BF16])
def test_cta_pair_kernel_matches_oracle_and_dense(case, prec):
    """The CTA-pair kernel (configs 10 to 13, and 21 in two passes; 20 is the two-pass
    dense kernel) on shapes with one and two 256-row piece pairs per block row and one and
    two 256-column pieces per block column."""
    mdl, left, right = make(*case)
    ops = dmrg2d.build_ops(mdl, left, right)
    sb = Superblock(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 6)
    ref = sb.apply(v)
    dmrg2d.set_tile_config(ops, prec, 0)
    y0 = run(ops, v, prec)
    for cfg in (10, 11, 12, 13, 20, 21, 23, 25, 26):  # blocks / pool / two passes / 3-D
        dmrg2d.set_tile_config(ops, prec, cfg)
        y = run(ops, v, prec)
        assert rel(y, ref) <= TOL[prec], (cfg, rel(y, ref))
        assert rel(y, y0) <= (2e-5 if cfg >= 20 else 1e-6), cfg


CASES = {
    "heisenberg_4leg": lambda: synth.workload_ladder4_heisenberg_sectors(m=48, block_sites=8),
    "hubbard_3leg": lambda: synth.workload_ladder3_hubbard_sectors(m=25, block_sites=6,
                                                                    n_up=6, n_dn=6),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", [dmrg2d.TF32, dmrg2d.BF16])
def test_sector_tensor_core_matches_oracle(name, prec):
    mdl, left, right, target = CASES[name]()
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    assert ops.info["tc_ok"] == 1
    pmap = packed_map(sb, target)
    valid = pmap >= 0
    vp = np.where(valid, synth.start_vector(len(pmap), 31), 0.0)
    vd = np.zeros(sb.n_vec)
    vd[pmap[valid]] = vp[valid]
    yd = sb.apply(vd)
    ref = np.zeros(len(pmap))
    ref[valid] = yd[pmap[valid]]
    # moves fused / in their own kernel / the segment kernels (22)
    for cfg in list(range(1, 7)) + list(range(14, 20)) + [22]:
        dmrg2d.set_tile_config(ops, prec, cfg)
        got = run(ops, vp, prec)
        assert np.all(got[~valid] == 0.0)
        assert rel(got, ref) <= TOL[prec], (cfg, rel(got, ref))


@pytest.mark.parametrize("prec", [dmrg2d.TF32, dmrg2d.BF16])
def test_autotune_picks_a_working_config(prec):
    mdl, left, right, target = CASES["heisenberg_4leg"]()
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    best, ms = dmrg2d.autotune(ops, prec)
    assert 1 <= best < 7 or 14 <= best < 20 or best == 22
    assert ms[22] > 0
    assert all(ms[i] == -1.0 for i in (0, 7, 8, 9, 10, 11, 12, 13, 20, 21))
    assert all(t > 0 for t in ms[1:7] + ms[14:20])
    assert ms[best] == min(t for t in ms if t > 0)
    sb = Superblock(mdl, left, right)
    pmap = packed_map(sb, target)
    valid = pmap >= 0
    vp = np.where(valid, synth.start_vector(len(pmap), 5), 0.0)
    vd = np.zeros(sb.n_vec)
    vd[pmap[valid]] = vp[valid]
    ref = np.zeros(len(pmap))
    ref[valid] = sb.apply(vd)[pmap[valid]]
    assert rel(run(ops, vp, prec), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [dmrg2d.TF32, dmrg2d.BF16])
def test_sector_apply_captured_in_cuda_graph(prec):
    """apply_H on a sector-restricted superblock (grouped persistent launch + scalar
    moves) recorded once in a CUDA graph and replayed: the replays equal the direct call,
    and a replay after the input changed sees the new input."""
    mdl, left, right, target = CASES["hubbard_3leg"]()
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    pmap = packed_map(sb, target)
    valid = pmap >= 0
    dt = torch.float32 if prec == dmrg2d.TF32 else torch.bfloat16
    vs = [torch.from_numpy(np.where(valid, synth.start_vector(len(pmap), s), 0.0)).cuda().to(dt)
          for s in (41, 42)]
    direct = []
    for v in vs:
        y = torch.empty(len(pmap), dtype=torch.float32, device="cuda")
        dmrg2d.apply_H(ops, v, y, prec)
        direct.append(y.clone())
    x = vs[0].clone()
    y = torch.zeros(len(pmap), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):                 # warm-up on the capture stream
        dmrg2d.apply_H(ops, x, y, prec)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        dmrg2d.apply_H(ops, x, y, prec)
    for k in (0, 1, 0):
        x.copy_(vs[k])
        y.fill_(-7.0)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(y, direct[k]), k
    dmrg2d.check_device(ops)


@pytest.mark.parametrize("name", sorted(CASES))
def test_sector_bf16x3_matches_oracle(name):
    """Split BF16 on sector-restricted superblocks: the three products through the grouped
    kernel (moves in its epilogue or in their own kernel), within 1e-4 of the oracle, and
    at least 20 times closer than plain BF16."""
    mdl, left, right, target = CASES[name]()
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    pmap = packed_map(sb, target)
    valid = pmap >= 0
    vp = np.where(valid, synth.start_vector(len(pmap), 31), 0.0)
    vd = np.zeros(sb.n_vec)
    vd[pmap[valid]] = vp[valid]
    ref = np.zeros(len(pmap))
    ref[valid] = sb.apply(vd)[pmap[valid]]
    for cfg in (1, 4, 14, 17, 22):
        dmrg2d.set_tile_config(ops, dmrg2d.BF16, cfg)
        got = run(ops, vp, dmrg2d.BF16X3)
        assert np.all(got[~valid] == 0.0)
        e3 = rel(got, ref)
        e1 = rel(run(ops, vp, dmrg2d.BF16), ref)
        assert e3 <= TOL[dmrg2d.BF16X3] and e3 * 20 <= e1, (cfg, e3, e1)


@pytest.mark.parametrize("cfg", [0, 1, 4, 7, 8, 10, 11, 13, 20, 21])
def test_dense_bf16x3_every_kernel(cfg):
    """Split BF16 through every dense tile configuration chosen for BF16 (the operator
    pool and the two-pass form are replaced by per-position blocks in one pass)."""
    mdl, left, right = make("heisenberg", 2, 256, 512)
    ops = dmrg2d.build_ops(mdl, left, right)
    sb = Superblock(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 8)
    ref = sb.apply(v)
    dmrg2d.set_tile_config(ops, dmrg2d.BF16, cfg)
    assert rel(run(ops, v, dmrg2d.BF16X3), ref) <= TOL[dmrg2d.BF16X3]


@pytest.mark.parametrize("prec", [dmrg2d.TF32, dmrg2d.BF16])
@pytest.mark.parametrize("sizes", ["small", "mixed"])
def test_segment_kernels_on_uneven_sectors(prec, sizes):
    """The segment kernels (configuration 22) against the oracle where sectors are a few
    states (N and K far below one instruction's 16 / one stage's 32) and where they exceed
    one piece (row segments over 128 states: two N ranges in pass 1; column segments over
    256: two in pass 2), ragged everywhere; and the same result as the grouped kernel."""
    if sizes == "small":
        mdl, left, right, target = synth.workload_ladder3_hubbard_sectors(m=40, block_sites=6,
                                                                          n_up=6, n_dn=6)
    else:   # 2-leg Heisenberg, block sectors [12, 128, 311, 137, 12] (m = 600)
        offs, sz = synth.sector_sizes([(q,) for q in range(-2, 3)], (0.8,), 600, 3)
        assert max(sz) > 256 and min(sz) < 16
        lab = synth.labels_from_sectors((5,), offs, sz)
        mdl = synth.model("heisenberg", 2, J_leg=0.8, J_rung=1.1)
        left, right = synth.heisenberg_block(600, 2, 7, lab), synth.heisenberg_block(600, 2, 8, lab)
        target = (12,)
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    pmap = packed_map(sb, target)
    valid = pmap >= 0
    vp = np.where(valid, synth.start_vector(len(pmap), 17), 0.0)
    vd = np.zeros(sb.n_vec)
    vd[pmap[valid]] = vp[valid]
    ref = np.zeros(len(pmap))
    ref[valid] = sb.apply(vd)[pmap[valid]]
    dmrg2d.set_tile_config(ops, prec, 22)
    got = run(ops, vp, prec)
    assert np.all(got[~valid] == 0.0)
    assert rel(got, ref) <= TOL[prec], rel(got, ref)
    dmrg2d.set_tile_config(ops, prec, 4)
    assert rel(got, run(ops, vp, prec)) <= 1e-5
