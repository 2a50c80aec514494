"""Davidson with the Jacobi and the learned preconditioner, and the network's kernels (GPU).

* diag(H) on the device against the oracle's diagonal (dense and sector layouts);
* Davidson (FP64, Jacobi) reaches the Lanczos ground energy;
* the MLP's forward pass, loss and gradient (FP32 kernels) against the FP64 oracle;
* training by the library's Adam step lowers the loss;
* the trained preconditioner against plain Jacobi on unseen seeds: both converge to
  the same energy; iterations and time of each are reported (the gain).
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as omlp  # noqa: E402
from oracle.superblock import Superblock  # noqa: E402
from paper_0707_0159_gb300 import dmrg2d, synth  # noqa: E402

from test_gpu_sectors import packed_map  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def test_diagonal_dense_matches_oracle():
    mdl = synth.model("hubbard", 2, t=1.0, U=6.0)
    left, right = synth.hubbard_block(9, 2, 1), synth.hubbard_block(7, 2, 2)
    ops = dmrg2d.build_ops(mdl, left, right)
    sb = Superblock(mdl, left, right)
    D = torch.empty(sb.n_vec, dtype=torch.float64, device=DEV)
    dmrg2d.diagonal(ops, D)
    assert np.allclose(D.cpu().numpy(), sb.diagonal(), rtol=0, atol=1e-13)


def test_diagonal_sectors_matches_oracle():
    mdl, left, right, target = synth.workload_ladder4_heisenberg_sectors(m=48, block_sites=8)
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    sb = Superblock(mdl, left, right)
    pmap = packed_map(sb, target)
    D = torch.empty(len(pmap), dtype=torch.float64, device=DEV)
    dmrg2d.diagonal(ops, D)
    got = D.cpu().numpy()
    valid = pmap >= 0
    assert np.allclose(got[valid], sb.diagonal()[pmap[valid]], rtol=0, atol=1e-13)
    assert np.all(got[~valid] == 0.0)


def test_davidson_jacobi_matches_lanczos():
    mdl, left, right, _ = synth.workload_ladder2_heisenberg_m64()
    ops = dmrg2d.build_ops(mdl, left, right)
    v0 = synth.start_vector(ops.info["n_vec"], 2)
    x = torch.from_numpy(v0).to(DEV)
    e_l, st_l, c_l = dmrg2d.lanczos_ground(ops, x, max_iter=400, krylov_dim=400, tol=1e-11)
    assert c_l == 0
    for pre in ("jacobi",):
        x = torch.from_numpy(v0).to(DEV)
        e, st, code = dmrg2d.davidson_ground(ops, x, precond=pre, tol=1e-10, max_iter=600)
        assert code == 0, (pre, st)
        assert abs(e - e_l) <= 1e-10 * abs(e_l), (pre, e, e_l)


def test_mlp_kernels_match_oracle():
    H, B = 32, 1000
    net = dmrg2d.MLP(hidden=H, seed=3)
    rng = np.random.default_rng(0)
    # random parameters everywhere (a new network's output layer starts at zero)
    net.set_params((0.3 * rng.standard_normal(net.n_params)).astype(np.float32))
    p = net.get_params().astype(np.float64)
    X = rng.normal(size=(B, 4)).astype(np.float32)
    w = rng.normal(size=B).astype(np.float32)
    T = rng.normal(size=B).astype(np.float32)
    Xt, wt, Tt = (torch.from_numpy(a).to(DEV) for a in (X, w, T))
    Y = torch.empty(B, dtype=torch.float32, device=DEV)
    net.forward(Xt, Y)
    y_ref, _ = omlp.forward(p, H, X.astype(np.float64))
    assert np.allclose(Y.cpu().numpy(), y_ref, rtol=1e-4, atol=1e-5)
    g = torch.empty(net.n_params, dtype=torch.float32, device=DEV)
    loss = net.loss_grad(Xt, wt, Tt, g)
    g_ref = omlp.grad(p, H, X.astype(np.float64), w.astype(np.float64), T.astype(np.float64))
    assert abs(loss - omlp.loss(p, H, X, w, T)) <= 1e-5 * abs(loss)
    err = np.linalg.norm(g.cpu().numpy() - g_ref) / np.linalg.norm(g_ref)
    assert err <= 1e-4, err


def test_mlp_training_lowers_loss():
    H, B = 64, 4096
    net = dmrg2d.MLP(hidden=H, seed=1)
    rng = np.random.default_rng(2)
    d = rng.uniform(0.2, 4.0, B)
    X = omlp.features(d, 0.0, 1.0, 0.5, 0.3).astype(np.float32)
    w = rng.normal(size=B).astype(np.float32)
    T = (w * (-1.0 / d)).astype(np.float32)       # the Jacobi factor as the target
    Xt, wt, Tt = (torch.from_numpy(a).to(DEV) for a in (X, w, T))
    first = net.train_step(Xt, wt, Tt, 1e-3)
    for _ in range(400):
        last = net.train_step(Xt, wt, Tt, 1e-3)
    assert last <= 0.1 * first, (first, last)


# ---- the learned preconditioner on the sector-restricted 3-leg Hubbard superblock ---------

def hubbard_case(seed):
    return synth.workload_ladder3_hubbard_sectors(m=40, block_sites=6, seed=seed, n_up=6, n_dn=6)


def davidson_run(ops, v0, **kw):
    x = torch.from_numpy(v0).to(DEV)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = dmrg2d.davidson_ground(ops, x, **kw)
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def train_mlp(seeds, hidden=256, cap=60, batch=8192, epochs=6):
    net = dmrg2d.MLP(hidden=hidden, seed=7)
    rng = np.random.default_rng(11)
    for seed in seeds:
        mdl, left, right, target = hubbard_case(seed)
        ops = dmrg2d.build_ops(mdl, left, right, target=target)
        n = ops.info["n_vec"]
        v0 = synth.start_vector(n, seed + 100)
        xl = torch.zeros(cap * n, dtype=torch.float64, device=DEV)
        rl = torch.zeros(cap * n, dtype=torch.float64, device=DEV)
        x = torch.from_numpy(v0).to(DEV)
        e, st, code, thetas = dmrg2d.davidson_ground(ops, x, precond="jacobi", tol=1e-10,
                                                     max_iter=400, log=(cap, xl, rl))
        assert code == 0
        D = torch.empty(n, dtype=torch.float64, device=DEV)
        dmrg2d.diagonal(ops, D)
        steps = min(cap, st["iters"]) - 1
        X = torch.empty(batch * 4, dtype=torch.float32, device=DEV)
        w = torch.empty(batch, dtype=torch.float32, device=DEV)
        T = torch.empty(batch, dtype=torch.float32, device=DEV)
        for _ in range(epochs):
            for k in range(steps):
                idx = torch.from_numpy(rng.integers(0, n, batch)).to(DEV)
                dmrg2d.mlp_make_batch(ops, xl[k * n:(k + 1) * n], rl[k * n:(k + 1) * n],
                                      thetas[k], x, D, idx, X, w, T)
                net.train_step(X, w, T, 3e-4)
    return net


def test_learned_preconditioner_against_jacobi():
    net = train_mlp(seeds=[0, 1, 2, 3])
    rows = []
    for seed in (32, 33):
        mdl, left, right, target = hubbard_case(seed)
        ops = dmrg2d.build_ops(mdl, left, right, target=target)
        v0 = synth.start_vector(ops.info["n_vec"], seed + 100)
        (e_j, st_j, c_j), t_j = davidson_run(ops, v0, precond="jacobi", tol=1e-9, max_iter=800)
        (e_m, st_m, c_m), t_m = davidson_run(ops, v0, precond="mlp", mlp=net, tol=1e-9,
                                             max_iter=800)
        assert c_j == 0 and c_m == 0, (st_j, st_m)
        assert abs(e_m - e_j) <= 1e-8 * abs(e_j)
        rows.append((seed, st_j["iters"], st_m["iters"], t_j, t_m))
    print("\nseed  jacobi_iters  mlp_iters  jacobi_s  mlp_s")
    for r in rows:
        print("%4d  %12d  %9d  %8.3f  %5.3f" % r)
    # the learned factor must not be catastrophically worse than the formula it replaces
    assert sum(r[2] for r in rows) <= 2 * sum(r[1] for r in rows)


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_mixed_davidson_reaches_fp64_energy(prec):
    """Davidson with the low-precision H·v (TF32, or split BF16) to a residual above its
    rounding floor, then the FP64 outer loop: the FP64 Lanczos energy to 1e-9, on a sector
    superblock, with the Jacobi and with a (fresh: y = 0, i.e. Jacobi) network."""
    mdl, left, right, target = synth.workload_ladder3_hubbard_sectors(m=64, block_sites=6,
                                                                      n_up=6, n_dn=6)
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    pad = dmrg2d.sector_dense_index(ops) < 0
    v0 = np.where(pad, 0.0, synth.start_vector(ops.info["n_vec"], 9))
    x = torch.from_numpy(v0).to(DEV)
    e_l, st_l, c_l = dmrg2d.lanczos_ground(ops, x, max_iter=2000, krylov_dim=200, tol=1e-11,
                                           thick_keep=32)
    assert c_l == 0
    net = dmrg2d.MLP(hidden=64, seed=3)
    for pre in ("jacobi", "mlp"):
        x = torch.from_numpy(v0).to(DEV)
        e, st, code = dmrg2d.davidson_ground(ops, x, precond=pre, mlp=net if pre == "mlp" else None,
                                             precision=prec, refine=1, tol=1e-3, refine_tol=1e-9,
                                             max_iter=300, inner_iter=40, outer_max=40)
        assert code == 0, (pre, st)
        assert abs(e - e_l) <= 1e-9 * abs(e_l), (pre, e, e_l)
        assert st["resid"] <= 1e-9 * abs(e) and st["n_hv_low"] > 0
