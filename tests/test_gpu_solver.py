"""GPU ground-state solvers against the oracle and brute-force ED."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lattice_ed  # noqa: E402
from oracle.columns import HubbardColumn, SpinColumn  # noqa: E402
from oracle.solvers import lanczos_ground as oracle_lanczos  # noqa: E402
from oracle.superblock import Superblock  # noqa: E402
from paper_0707_0159_gb300 import dmrg2d, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def spin_column_block(n):
    col = SpinColumn(n, 1.0)
    edge = []
    for y in range(n):
        edge += [col.Sz[y], col.Sp[y]]
    return {"m": col.d, "H": col.H, "edge": edge, "parity": None, "qn": None}


def hubbard_column_block(n, t=1.0, U=8.0):
    col = HubbardColumn(n, t, U)
    edge = []
    for y in range(n):
        edge += [col.cdag[y][0], col.cdag[y][1]]
    return {"m": col.d, "H": col.H, "edge": edge, "parity": col.parity, "qn": None}


def gpu_ground(ops, v0, **kw):
    x = torch.from_numpy(np.asarray(v0, dtype=np.float64)).to(DEV)
    e, st, code = dmrg2d.lanczos_ground(ops, x, **kw)
    return e, x.cpu().numpy(), st, code


def test_ladder2_m64_200_steps_against_oracle():
    mdl, left, right, _ = synth.workload_ladder2_heisenberg_m64()
    ops = dmrg2d.build_ops(mdl, left, right)
    sb = Superblock(mdl, left, right)
    v0 = synth.start_vector(sb.n_vec, 2)
    e, x, st, code = gpu_ground(ops, v0, max_iter=200, krylov_dim=200, fixed_steps=1)
    assert code == 0 and st["iters"] == 200 and st["n_hv_fp64"] == 200
    e_ref, x_ref, _ = oracle_lanczos(sb.apply, v0, max_iter=200, fixed_steps=True)
    assert abs(e - e_ref) <= 1e-10 * abs(e_ref)
    r = sb.apply(x) - e * x                       # residual with the oracle's H
    assert np.linalg.norm(r) <= 1e-6 * abs(e)
    assert abs(abs(x @ x_ref) - 1.0) <= 1e-8


def test_untruncated_ladder_2x4_equals_ed():
    mdl = synth.model("heisenberg", 2)
    blk = spin_column_block(2)
    ops = dmrg2d.build_ops(mdl, blk, blk)
    e, _, st, code = gpu_ground(ops, synth.start_vector(ops.info["n_vec"], 1), max_iter=200,
                                krylov_dim=200, tol=1e-13)
    e_ed = lattice_ed.heisenberg_spectrum(2, 4)[0]
    assert abs(e - e_ed) <= 1e-10 * abs(e_ed)


def test_untruncated_hubbard_2x3_equals_ed():
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    col = hubbard_column_block(2)
    ops = dmrg2d.build_ops(mdl, col, synth.empty_block("hubbard"))
    e, _, st, code = gpu_ground(ops, synth.start_vector(ops.info["n_vec"], 1), max_iter=400,
                                krylov_dim=400, tol=1e-13)
    e_ed = lattice_ed.hubbard_ground(2, 3, 1.0, 8.0)
    assert abs(e - e_ed) <= 1e-10 * abs(e_ed)


def test_lanczos_deterministic_and_restart():
    mdl, left, right, _ = synth.workload_ladder2_heisenberg_m64()
    ops = dmrg2d.build_ops(mdl, left, right)
    v0 = synth.start_vector(ops.info["n_vec"], 4)
    e1, x1, _, c1 = gpu_ground(ops, v0, max_iter=300, krylov_dim=300, tol=1e-11)
    e2, x2, _, c2 = gpu_ground(ops, v0, max_iter=300, krylov_dim=300, tol=1e-11)
    assert c1 == 0 and e1 == e2 and np.array_equal(x1, x2)
    # a small basis with explicit restarts reaches the same eigenvalue
    e3, _, st3, c3 = gpu_ground(ops, v0, max_iter=2000, krylov_dim=40, tol=1e-11)
    assert c3 == 0 and abs(e3 - e1) <= 1e-9 * abs(e1)


def test_enoconv_is_reported():
    mdl, left, right, _ = synth.workload_ladder2_heisenberg_m64()
    ops = dmrg2d.build_ops(mdl, left, right)
    e, _, st, code = gpu_ground(ops, synth.start_vector(ops.info["n_vec"], 4), max_iter=5,
                                krylov_dim=5, tol=1e-14)
    assert code == -5 and np.isfinite(e) and st["iters"] == 5


@pytest.fixture(scope="module")
def ladder2_m128():
    """2-leg Hubbard superblock, m = 128, d = 16, converged plain FP64 reference."""
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    left, right = synth.hubbard_block(128, 2, 40), synth.hubbard_block(128, 2, 41)
    ops = dmrg2d.build_ops(mdl, left, right)
    v0 = synth.start_vector(ops.info["n_vec"], 3)
    e64, _, st64, c64 = gpu_ground(ops, v0, max_iter=3000, krylov_dim=300, tol=1e-10)
    return ops, v0, e64, st64, c64


def test_fp64_lanczos_converges(ladder2_m128):
    ops, v0, e64, st64, c64 = ladder2_m128
    assert c64 == 0, st64
    assert st64["resid"] <= 1e-10 * abs(e64)


@pytest.mark.parametrize("prec,rprec", [(dmrg2d.FP32, dmrg2d.FP64), (dmrg2d.TF32, dmrg2d.FP64),
                                        (dmrg2d.BF16, dmrg2d.FP64), (dmrg2d.TF32, dmrg2d.FP64X),
                                        (dmrg2d.BF16X3, dmrg2d.FP64)])
def test_mixed_precision_reaches_fp64_energy(ladder2_m128, prec, rprec):
    ops, v0, e64, st64, c64 = ladder2_m128
    assert ops.info["tc_ok"]
    e, x, st, code = gpu_ground(ops, v0, precision=prec, refine=1, tol=1e-8, inner_iter=60,
                                outer_max=40, refine_precision=rprec)
    assert code == 0, st
    assert abs(e - e64) <= 1e-8 * abs(e64), (e, e64, st)
    assert st["resid"] <= 1e-8 * abs(e)
    assert st["n_hv_fp64"] < st64["n_hv_fp64"], (st, st64)


# ---- the small eigensolve (a tridiagonal's lowest eigenpair) ------------------------------

def _tridiag_gpu(a, b):
    at = torch.tensor(np.asarray(a, float), device=DEV)
    bt = torch.tensor(np.asarray(b, float), device=DEV)
    th, s, res, status = dmrg2d.tridiag_lowest(at, bt)
    return th, s.cpu().numpy(), res, status


@pytest.mark.parametrize("k", [1, 2, 3, 50, 257, 512])
def test_tridiag_lowest_laplacian_closed_form(k):
    # T = tridiag(-1, 2, -1): lowest eigenvalue 2 - 2 cos(pi / (k + 1)), eigenvector
    # sin(j pi / (k + 1)), j = 1..k
    a, b = np.full(k, 2.0), np.full(k, -1.0)
    b[k - 1] = 0.5                      # the residual coupling, not part of T
    th, s, res, status = _tridiag_gpu(a, b)
    assert status == 0
    lam = 2.0 - 2.0 * np.cos(np.pi / (k + 1))
    assert abs(th - lam) <= 1e-14 * 4
    v = np.sin(np.arange(1, k + 1) * np.pi / (k + 1))
    v /= np.linalg.norm(v)
    assert np.abs(s - v).max() <= 1e-10
    assert abs(res - 0.5 * abs(v[-1])) <= 1e-12


@pytest.mark.parametrize("k,seed,scale", [(7, 0, 1.0), (64, 1, 1e3), (200, 2, 1e-2), (512, 3, 1.0)])
def test_tridiag_lowest_against_eigh(k, seed, scale):
    rng = np.random.default_rng(seed)
    a, b = scale * rng.standard_normal(k), scale * rng.standard_normal(k)
    if k > 20:
        b[k // 2] = 0.0                 # a reducible T: the lowest pair may sit in either part
    th, s, res, status = _tridiag_gpu(a, b)
    T = np.diag(a) + np.diag(b[:k - 1], 1) + np.diag(b[:k - 1], -1)
    w, V = np.linalg.eigh(T)
    assert status == 0
    assert abs(th - w[0]) <= 1e-13 * np.abs(w).max()
    assert np.linalg.norm(T @ s - th * s) <= 1e-12 * np.abs(w).max()
    assert abs(np.linalg.norm(s) - 1.0) <= 1e-13
    first = s[np.flatnonzero(s)[0]]
    assert first > 0
    if w[1] - w[0] > 1e-6 * np.abs(w).max():     # a simple eigenvalue: the vector is unique
        assert abs(abs(s @ V[:, 0]) - 1.0) <= 1e-10


def test_tridiag_lowest_rejects_bad_sizes_and_reports_nan():
    a = torch.zeros(513, dtype=torch.float64, device=DEV)
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.tridiag_lowest(a, a.clone())
    assert e.value.code == -2
    a = torch.tensor([1.0, float("nan"), 2.0], dtype=torch.float64, device=DEV)
    th, s, res, status = dmrg2d.tridiag_lowest(a, torch.ones_like(a))
    assert status == 1 and np.isnan(th)


# ---- thick restart --------------------------------------------------------------------------

def test_thick_restart_reaches_the_oracle_energy_in_fewer_steps():
    mdl, left, right, _ = synth.workload_ladder2_heisenberg_m64()
    ops = dmrg2d.build_ops(mdl, left, right)
    sb = Superblock(mdl, left, right)
    v0 = synth.start_vector(ops.info["n_vec"], 4)
    e_ref, _, _ = oracle_lanczos(sb.apply, v0, max_iter=400, tol=1e-12)
    e_x, _, st_x, c_x = gpu_ground(ops, v0, max_iter=3000, krylov_dim=30, tol=1e-11)
    e_t, x_t, st_t, c_t = gpu_ground(ops, v0, max_iter=3000, krylov_dim=30, tol=1e-11,
                                     thick_keep=8)
    assert c_x == 0 and c_t == 0
    assert abs(e_t - e_ref) <= 1e-10 * abs(e_ref), (e_t, e_ref)
    assert abs(e_x - e_ref) <= 1e-10 * abs(e_ref), (e_x, e_ref)
    assert st_t["iters"] < st_x["iters"], (st_t, st_x)
    r = sb.apply(x_t) - e_t * x_t        # an eigenvector of the oracle's H
    assert np.linalg.norm(r) <= 1e-9 * abs(e_t)
    # deterministic, and every kept-space size gives the same eigenpair
    e_t2, x_t2, _, _ = gpu_ground(ops, v0, max_iter=3000, krylov_dim=30, tol=1e-11, thick_keep=8)
    assert e_t2 == e_t and np.array_equal(x_t2, x_t)
    for keep in (1, 20, 29):
        e_k, _, st_k, c_k = gpu_ground(ops, v0, max_iter=3000, krylov_dim=30, tol=1e-11,
                                       thick_keep=keep)
        assert c_k == 0 and abs(e_k - e_ref) <= 1e-10 * abs(e_ref), (keep, e_k, st_k)


def test_thick_restart_on_a_sector_superblock():
    # sector layout: the kept Ritz vectors and the continuation vector stay zero on padding
    grid = [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)]
    offs, sizes = synth.sector_sizes(grid, (1.0, 1.0), 12, 4, lo=1)
    lab = synth.labels_from_sectors((2, 2), offs, sizes)
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    left, right = synth.hubbard_block(12, 2, 4, lab), synth.hubbard_block(12, 2, 5, lab)
    ops = dmrg2d.build_ops(mdl, left, right, target=(5, 6))
    pad = dmrg2d.sector_dense_index(ops) < 0
    v0 = np.where(pad, 0.0, synth.start_vector(ops.info["n_vec"], 2))
    e_full, _, _, c0 = gpu_ground(ops, v0, max_iter=400, krylov_dim=400, tol=1e-11)
    e, x, st, code = gpu_ground(ops, v0, max_iter=3000, krylov_dim=24, tol=1e-11, thick_keep=6)
    assert c0 == 0 and code == 0
    assert abs(e - e_full) <= 1e-10 * abs(e_full)
    assert np.all(x[pad] == 0.0)


def test_thick_keep_is_validated():
    mdl, left, right, _ = synth.workload_ladder2_heisenberg_m64()
    ops = dmrg2d.build_ops(mdl, left, right)
    x = torch.from_numpy(synth.start_vector(ops.info["n_vec"], 4)).to(DEV)
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.lanczos_ground(ops, x, thick_keep=33)
    assert e.value.code == -1
