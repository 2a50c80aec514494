"""The allocation-free Lanczos entry point against the allocating one (GPU).

dmrg2d_lanczos_ground_noalloc serves callers that cannot call cudaMalloc (device
memory owned by another allocator, or loops that cannot take cudaMalloc's implicit
synchronisation).  It keeps all scratch in the library's static device array.  This
file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_0707_0159_gb300 import dmrg2d, synth  # noqa: E402

pytestmark = pytest.mark.gpu

OPTS = dict(max_iter=400, krylov_dim=24, tol=1e-10, check_every=5)


def test_noalloc_matches_allocating_solver_on_two_calls():
    # 2-leg Heisenberg ladder superblock, m = 64, d = 4: V is 256 x 256
    mdl, left, right, _ = synth.workload_ladder2_heisenberg_m64()
    ops = dmrg2d.build_ops(mdl, left, right)
    x0 = torch.from_numpy(synth.start_vector(ops.info["n_vec"], 6)).cuda()
    x_ref = x0.clone()
    e_ref, st_ref, c_ref = dmrg2d.lanczos_ground(ops, x_ref, **OPTS)
    assert c_ref == 0
    for _ in range(2):   # the second call reuses the array the first one left behind
        x = x0.clone()
        e, st, code = dmrg2d.lanczos_ground_noalloc(ops, x, **OPTS)
        assert code == 0, dmrg2d.last_error()
        assert abs(e - e_ref) <= 1e-10 * abs(e_ref), (e, e_ref)
        assert st["iters"] == st_ref["iters"]
        diff = torch.linalg.vector_norm(x - x_ref).item()
        assert diff <= 1e-8, diff


def test_noalloc_sector_superblock_with_nonzero_padding():
    """A sector-restricted superblock whose start vector is nonzero on the padding rows:
    both solvers zero the padding first, so they agree (and the result's padding is 0)."""
    grid = [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)]
    offs, sizes = synth.sector_sizes(grid, (1.0, 1.0), 12, 4, lo=1)
    lab = synth.labels_from_sectors((2, 2), offs, sizes)
    mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
    left, right = synth.hubbard_block(12, 2, 4, lab), synth.hubbard_block(12, 2, 5, lab)
    ops = dmrg2d.build_ops(mdl, left, right, target=(5, 6))
    pad = dmrg2d.sector_dense_index(ops) < 0
    assert pad.any()
    x0 = torch.from_numpy(synth.start_vector(ops.info["n_vec"], 3)).cuda()  # nonzero everywhere
    x_ref = x0.clone()
    e_ref, st_ref, c_ref = dmrg2d.lanczos_ground(ops, x_ref, **OPTS)
    assert c_ref == 0
    for _ in range(2):
        x = x0.clone()
        e, st, code = dmrg2d.lanczos_ground_noalloc(ops, x, **OPTS)
        assert code == 0, dmrg2d.last_error()
        assert abs(e - e_ref) <= 1e-10 * abs(e_ref), (e, e_ref)
        assert st["iters"] == st_ref["iters"]
        assert torch.linalg.vector_norm(x - x_ref).item() <= 1e-8
        assert np.all(x.cpu().numpy()[pad] == 0.0)


def test_noalloc_rejects_problems_beyond_its_scratch():
    mdl, left, right, _ = synth.workload_ladder2_heisenberg_m64()
    ops = dmrg2d.build_ops(mdl, left, right)
    x = torch.from_numpy(synth.start_vector(ops.info["n_vec"], 6)).cuda()
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.lanczos_ground_noalloc(ops, x, max_iter=400, krylov_dim=200)
    assert e.value.code == -2 and "static scratch" in str(e.value)
    with pytest.raises(dmrg2d.Dmrg2dError) as e:   # the basis cap, reported as such
        dmrg2d.lanczos_ground_noalloc(ops, x, max_iter=2000, krylov_dim=600)
    assert e.value.code == -2 and "exceeds 512" in str(e.value)
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.lanczos_ground_noalloc(ops, x, precision="tf32", refine=1)
    assert e.value.code == -8
