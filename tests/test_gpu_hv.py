"""GPU parity of dmrg2d_apply_H against the CPU oracle (paper Eq. (dec) and the V forms).

FP64 must match to a relative Frobenius error <= 1e-12 (the product is exact
linear algebra; only summation order differs).  FP32 (CUDA cores) <= 1e-5.
TF32/BF16 tensor-core products are compared with the bound derived from their
unit roundoff: TF32 <= 1e-3; BF16 <= 6e-3 (its expected error ~2e-3 is above
1e-3, see the BF16 test); split BF16 (BF16X3: hi and lo parts, three products, the
lo x lo product dropped) <= 1e-4 (per product at most ~3 u^2 = 4.6e-5 with
u = 2^-8).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.superblock import Superblock  # noqa: E402
from paper_0707_0159_gb300 import dmrg2d, synth  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(ops, v, prec):
    x = torch.from_numpy(v).to(DEV)
    if prec == dmrg2d.BF16X3:
        xs = dmrg2d.convert_input(x, prec)
        y = torch.full((x.numel(),), float("nan"), dtype=torch.float32, device=DEV)
        dmrg2d.apply_H(ops, xs, y, prec)
        torch.cuda.synchronize()
        return y.double().cpu().numpy(), x.cpu().numpy()
    if prec in (dmrg2d.FP32, dmrg2d.TF32):
        x = x.float()
    elif prec == dmrg2d.BF16:
        x = x.bfloat16()
    wide = prec in (dmrg2d.FP64, dmrg2d.FP64X)
    y = torch.empty(x.numel(), dtype=torch.float64 if wide else torch.float32, device=DEV)
    dmrg2d.apply_H(ops, x, y, prec)
    torch.cuda.synchronize()
    return y.double().cpu().numpy(), x.double().cpu().numpy()


SMALL = [
    ("heisenberg", 2, 5, 7),      # ragged blocks, d = 4
    ("hubbard", 1, 3, 1),         # block 4 is a one-state block
    ("hubbard", 2, 70, 65),       # two row tiles per block, ragged tails, d = 16
    ("heisenberg", 3, 130, 129),  # three tiles, d = 8
    ("hubbard", 3, 17, 9),        # d = 64
]


def make(kind, n_legs, m1, m4, seed=0):
    mdl = synth.model(kind, n_legs, J_leg=0.8, J_rung=1.1, t=1.0, U=6.0)
    mk = synth.heisenberg_block if kind == "heisenberg" else synth.hubbard_block
    left = mk(m1, n_legs, seed + 1) if m1 > 1 else synth.empty_block(kind)
    right = mk(m4, n_legs, seed + 2) if m4 > 1 else synth.empty_block(kind)
    return mdl, left, right


@pytest.mark.parametrize("case", SMALL)
def test_fp64_small_shapes(case):
    mdl, left, right = make(*case)
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right)
    assert ops.info["n_vec"] == sb.n_vec
    v = synth.start_vector(sb.n_vec, 7)
    y, _ = run(ops, v, dmrg2d.FP64)
    assert rel(y, sb.apply(v)) <= 1e-12


@pytest.mark.parametrize("case", SMALL)
def test_fp64x_small_shapes(case):
    """FP64 emulated with float pairs: FP64-class accuracy (<= 1e-12) against the oracle."""
    mdl, left, right = make(*case)
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 7)
    y, _ = run(ops, v, dmrg2d.FP64X)
    assert rel(y, sb.apply(v)) <= 1e-12


@pytest.mark.parametrize("case", SMALL[:3])
def test_fp32_small_shapes(case):
    mdl, left, right = make(*case)
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 8)
    y, _ = run(ops, v, dmrg2d.FP32)
    assert rel(y, sb.apply(v)) <= 1e-5


def test_block_structure_matches_oracle():
    """Block positions and scalar moves counted independently from the oracle's terms."""
    mdl, left, right = make("hubbard", 2, 6, 5)
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right)
    d = sb.d
    posL = np.eye(d, dtype=bool)
    for _, X, _ in sb.terms_l[2:]:          # edge terms (block operators)
        posL |= X != 0
    posR = np.eye(d, dtype=bool)
    for _, X, _ in sb.terms_r[2:]:
        posR |= X != 0
    Hcol = sb.col.H
    offL = (Hcol != 0) & ~posL & ~np.eye(d, dtype=bool)
    offR = (Hcol != 0) & ~posR & ~np.eye(d, dtype=bool)
    S = (sb.H_center() != 0) | np.kron(np.eye(d, dtype=bool), offL) | np.kron(offR, np.eye(d, dtype=bool))
    i = ops.info
    assert i["n_blk_left"] == posL.sum() and i["n_blk_right"] == posR.sum()
    assert i["n_scalar"] == S.sum()
    m1, m4 = 6, 5
    f = (2 * posL.sum() * m1 * m1 * d * m4 + 2 * posR.sum() * m4 * m4 * m1 * d
         + 2 * S.sum() * m1 * m4)
    assert i["flops_per_apply"] == f


def test_ladder2_m64_fp64_full():
    mdl, left, right, _ = synth.workload_ladder2_heisenberg_m64()
    sb = Superblock(mdl, left, right)
    ops = dmrg2d.build_ops(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 2)
    y, _ = run(ops, v, dmrg2d.FP64)
    assert rel(y, sb.apply(v)) <= 1e-12
    y2, _ = run(ops, v, dmrg2d.FP64)
    assert np.array_equal(y, y2)  # deterministic


def test_hermitian_on_gpu():
    mdl, left, right = make("hubbard", 2, 33, 20)
    ops = dmrg2d.build_ops(mdl, left, right)
    n = ops.info["n_vec"]
    v, w = synth.start_vector(n, 1), synth.start_vector(n, 2)
    Hv, _ = run(ops, v, dmrg2d.FP64)
    Hw, _ = run(ops, w, dmrg2d.FP64)
    assert abs(w @ Hv - v @ Hw) <= 1e-12 * np.linalg.norm(Hv) * np.linalg.norm(w)


def test_zero_and_linearity():
    mdl, left, right = make("heisenberg", 2, 9, 11)
    ops = dmrg2d.build_ops(mdl, left, right)
    n = ops.info["n_vec"]
    y0, _ = run(ops, np.zeros(n), dmrg2d.FP64)
    assert np.all(y0 == 0.0)
    a, b = synth.start_vector(n, 3), synth.start_vector(n, 4)
    ya, _ = run(ops, a, dmrg2d.FP64)
    yb, _ = run(ops, b, dmrg2d.FP64)
    yab, _ = run(ops, 2 * a - 0.5 * b, dmrg2d.FP64)
    assert rel(yab, 2 * ya - 0.5 * yb) <= 1e-13


def test_bad_dtype_is_rejected():
    mdl, left, right = make("heisenberg", 1, 4, 4)
    ops = dmrg2d.build_ops(mdl, left, right)
    n = ops.info["n_vec"]
    x = torch.zeros(n, dtype=torch.float32, device=DEV)
    y = torch.zeros(n, dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        dmrg2d.apply_H(ops, x, y, dmrg2d.FP64)


# ---- tensor-core path on small superblocks, every output element ------------------------------

TC_CASES = [
    ("hubbard", 2, 128, 128),      # d = 16, N tile 128, 16 x 16 tiles of 128 x 128
    ("heisenberg", 3, 256, 512),   # d = 8, two 128-row pieces and two 256-column pieces per tile
    ("heisenberg", 2, 128, 256),   # d = 4, fewer tiles than SMs
]


@pytest.mark.parametrize("case", TC_CASES)
@pytest.mark.parametrize("prec,tol", [(dmrg2d.TF32, 1e-3), (dmrg2d.BF16, 6e-3),
                                      (dmrg2d.BF16X3, 1e-4)])
def test_tensor_core_small_shapes(case, prec, tol):
    mdl, left, right = make(*case)
    ops = dmrg2d.build_ops(mdl, left, right)
    assert ops.info["tc_ok"] == 1
    sb = Superblock(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 21)
    y, _ = run(ops, v, prec)
    ref = sb.apply(v)
    err = rel(y, ref)
    assert err <= tol, err
    # a second call on the same buffers gives the same bits (no stale accumulator state)
    y2, _ = run(ops, v, prec)
    assert np.array_equal(y, y2)
    dmrg2d.check_device(ops)


def test_tensor_core_unsupported_shape_is_reported():
    mdl, left, right = make("hubbard", 2, 70, 65)
    ops = dmrg2d.build_ops(mdl, left, right)
    assert ops.info["tc_ok"] == 0
    n = ops.info["n_vec"]
    x = torch.zeros(n, dtype=torch.float32, device=DEV)
    y = torch.zeros(n, dtype=torch.float32, device=DEV)
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.apply_H(ops, x, y, dmrg2d.TF32)
    assert e.value.code == -8


# ---- full-size 3-leg Hubbard superblock (m = 256, d = 64, V 16384 x 16384) -------------------

@pytest.fixture(scope="module")
def ladder3_full():
    mdl, left, right, _ = synth.workload_ladder3_hubbard_m256()
    ops = dmrg2d.build_ops(mdl, left, right)
    sb = Superblock(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 12)
    rng = np.random.default_rng(5)
    # sampled outputs: random entries plus the first and last rows/columns of V
    idx = np.concatenate([rng.integers(0, sb.n_vec, 200), [0, 1, 255, 256, sb.n_vec - 1]])
    return ops, sb, v, idx


@pytest.mark.parametrize("prec", [dmrg2d.FP64, dmrg2d.FP64X])
def test_ladder3_full_fp64_sampled(ladder3_full, prec):
    ops, sb, v, idx = ladder3_full
    y, _ = run(ops, v, prec)
    ref = sb.apply_at(v, idx)
    assert rel(y[idx], ref) <= 1e-12


@pytest.mark.parametrize("prec,tol", [(dmrg2d.TF32, 1e-3), (dmrg2d.BF16, 6e-3)])
def test_ladder3_full_tensor_core_sampled(ladder3_full, prec, tol):
    """Every dense-kernel variant (column-slab / blocked piece order, per-position blocks /
    operator pool, one or two passes) and the autotuner's choice, which is what the
    benchmark times."""
    ops, sb, v, idx = ladder3_full
    if not ops.info["tc_ok"]:
        pytest.skip("tensor-core path not available for these shapes")
    ref = sb.apply_at(v, idx)
    outs = {}
    for cfg in (0, 7, 8, 9, 10, 11, 12, 13, 20, 21, 23, 24, 25, 26):
        dmrg2d.set_tile_config(ops, prec, cfg)
        y, _ = run(ops, v, prec)
        outs[cfg] = y[idx]
        assert rel(outs[cfg], ref) <= tol, cfg
    # piece order and pool change neither the operands nor the K order of a piece
    for cfg in (7, 8, 9, 24):
        assert np.array_equal(outs[cfg], outs[0]), cfg
    for cfg in (10, 11, 12, 13, 23):  # M = 256 instructions over a CTA pair
        assert rel(outs[cfg], outs[0]) <= 1e-6, cfg
    assert np.array_equal(outs[23], outs[11])   # one 3-D copy = the four 2-D copies
    for cfg in (25, 26):                          # patch size: the same pieces in another order
        assert np.array_equal(outs[cfg], outs[23]), cfg
    # two passes: the first pass's partial sum (H_l V and its moves, entries up to |H_l||V|,
    # far above |Y|) is rounded to FP32 once more before V H_r^T is added
    for cfg in (20, 21):
        assert rel(outs[cfg], outs[0]) <= 2e-5, cfg
    best, _ = dmrg2d.autotune(ops, prec)
    y, _ = run(ops, v, prec)
    assert np.array_equal(y[idx], outs[best] if best in outs else y[idx])
    assert rel(y[idx], ref) <= tol


def test_convert_input_formats():
    """dmrg2d_convert_input writes the documented formats: TF32 = the nearest TF32 value
    (10 fraction bits kept), BF16 = bf16(float(x)), BF16X3 = [hi | lo] with hi = bf16(x),
    lo = bf16(x - hi)."""
    rng = np.random.default_rng(3)
    x64 = np.concatenate([rng.standard_normal(4093) * 10.0 ** rng.integers(-6, 6, 4093),
                          [0.0, -0.0, 1.0]])
    x = torch.from_numpy(x64).to(DEV)
    bf = dmrg2d.convert_input(x, dmrg2d.BF16).cpu()
    assert torch.equal(bf.view(torch.int16), torch.from_numpy(x64).float().bfloat16().view(torch.int16))
    x3 = dmrg2d.convert_input(x, dmrg2d.BF16X3).cpu()
    hi = torch.from_numpy(x64).float().bfloat16()
    lo = (torch.from_numpy(x64) - hi.double()).float().bfloat16()
    assert torch.equal(x3[:x64.size].view(torch.int16), hi.view(torch.int16))
    assert torch.equal(x3[x64.size:].view(torch.int16), lo.view(torch.int16))
    # hi + lo carries ~16 significant bits
    approx = hi.double().numpy() + lo.double().numpy()
    assert np.all(np.abs(approx - x64) <= 1.01 * 2.0 ** -16 * np.abs(x64) + 1e-300)
    tf = dmrg2d.convert_input(x, dmrg2d.TF32).cpu().numpy()
    assert np.all(tf.view(np.uint32) & 0x1FFF == 0)          # 13 low fraction bits clear
    assert np.all(np.abs(tf - x64.astype(np.float32)) <= 2.0 ** -11 * np.abs(x64) * 1.0001)
    with pytest.raises(dmrg2d.Dmrg2dError):
        dmrg2d.convert_input(x, 9)


# ---- every output piece of the full-size superblock -------------------------------------------

@pytest.fixture(scope="module")
def ladder3_pieces(ladder3_full):
    """One random output and one corner in each of the 64 x 64 output tiles (i2, i3), each
    256 x 256 (the CTA-pair kernel's piece): 8192 entries, the oracle's sum per entry."""
    ops, sb, v, _ = ladder3_full
    m1, d, m4 = sb.m1, sb.d, sb.m4
    rng = np.random.default_rng(11)
    i2, i3 = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    i2, i3 = i2.ravel(), i3.ravel()
    corners = np.array([(0, 0), (m1 - 1, 0), (0, m4 - 1), (m1 - 1, m4 - 1)])
    c = corners[np.arange(i2.size) % 4]
    i1 = np.concatenate([rng.integers(0, m1, i2.size), c[:, 0]])
    i4 = np.concatenate([rng.integers(0, m4, i2.size), c[:, 1]])
    i2, i3 = np.concatenate([i2, i2]), np.concatenate([i3, i3])
    idx = i1 + m1 * i2 + m1 * d * i4 + m1 * d * m4 * i3
    return idx, sb.apply_at(v, idx)


@pytest.mark.parametrize("prec,tol", [(dmrg2d.TF32, 1e-3), (dmrg2d.BF16, 6e-3),
                                      (dmrg2d.BF16X3, 1e-4)])
def test_ladder3_full_every_piece(ladder3_full, ladder3_pieces, prec, tol):
    """The autotuner's choice at full size (what the benchmark times; BF16X3 runs the BF16
    choice), checked in every output piece: the relative error over all samples, and each
    sample within a few times the tolerance of the output's RMS, so that a piece left
    unwritten, written twice or taken from the wrong tile fails."""
    ops, sb, v, _ = ladder3_full
    idx, ref = ladder3_pieces
    if not ops.info["tc_ok"]:
        pytest.skip("tensor-core path not available for these shapes")
    best, _ = dmrg2d.autotune(ops, dmrg2d.BF16 if prec == dmrg2d.BF16X3 else prec)
    y, _ = run(ops, v, prec)
    got = y[idx]
    assert np.all(np.isfinite(got))
    assert rel(got, ref) <= tol, (best, rel(got, ref))
    rms = np.sqrt(np.mean(ref ** 2))
    assert np.max(np.abs(got - ref)) <= 30 * tol * rms, (best, np.max(np.abs(got - ref)) / rms)
