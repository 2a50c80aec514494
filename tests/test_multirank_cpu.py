"""Multi-rank paths on the CPU (gloo, world size 2; no GPU).

* the column-slab partition of H·v (oracle/partition.py) against the single-process
  H·v, with the ranks simulated in one process and as two gloo processes exchanging
  their pieces with all-to-all;
* the benchmark's replica bookkeeping: every rank gets the slowest rank's time and
  the job throughput counts every replica.
"""
import os
import socket
import sys
import tempfile

import numpy as np
import pytest

from oracle import partition
from oracle.superblock import Superblock
from paper_0707_0159_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def small_case(kind, m1, m4, seed=3):
    if kind == "heisenberg":
        mdl = synth.model("heisenberg", 2, J_leg=1.0, J_rung=1.0)
        left, right = synth.heisenberg_block(m1, 2, seed), synth.heisenberg_block(m4, 2, seed + 1)
    else:
        mdl = synth.model("hubbard", 2, t=1.0, U=8.0)
        left, right = synth.hubbard_block(m1, 2, seed), synth.hubbard_block(m4, 2, seed + 1)
    return Superblock(mdl, left, right)


@pytest.mark.parametrize("kind", ["heisenberg", "hubbard"])
@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_partition_simulated_ranks(kind, P):
    # m4 = 4 < P = 5 leaves an empty slab; m1 = 7 splits unevenly
    sb = small_case(kind, 7, 4)
    v = synth.start_vector(sb.n_vec, 9)
    y = partition.simulate(sb, v, P)
    assert np.allclose(y, sb.apply(v), rtol=0, atol=1e-13 * np.abs(sb.apply(v)).max())


def test_partition_ranges_cover():
    for n, P in ((7, 3), (4, 5), (256, 8), (1, 2)):
        r = partition.ranges(n, P)
        assert len(r) == P
        assert np.array_equal(np.concatenate(r), np.arange(n))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sb = small_case("hubbard", 6, 5)
        v = synth.start_vector(sb.n_vec, 4)
        mine = partition.slabs_of(sb, v, world)[rank]

        def exchange(pieces):
            # all-to-all of FP64 arrays of known shapes: flatten, send, reshape
            shapes_out = [p.shape for p in pieces]
            send = torch.from_numpy(np.concatenate([p.reshape(-1) for p in pieces]))
            shape_t = torch.tensor([list(s) for s in shapes_out], dtype=torch.int64)
            got = torch.empty_like(shape_t)          # row h: shape of the piece from rank h
            dist.all_to_all_single(got, shape_t)
            sizes_in = [int(np.prod(got[h].tolist())) for h in range(world)]
            recv = torch.empty(sum(sizes_in), dtype=torch.float64)
            dist.all_to_all_single(recv, send, output_split_sizes=sizes_in,
                                   input_split_sizes=[int(np.prod(s)) for s in shapes_out])
            parts, o = [], 0
            for h in range(world):
                parts.append(recv[o:o + sizes_in[h]].numpy().reshape(got[h].tolist()))
                o += sizes_in[h]
            return parts

        local, send1 = partition.rank_step1(sb, mine, world)
        send2 = partition.rank_step2(sb, exchange(send1), world)
        y_mine = partition.rank_step3(local, exchange(send2))
        ref = partition.slabs_of(sb, sb.apply(v), world)[rank]
        err = float(np.abs(y_mine - ref).max() / np.abs(ref).max())

        # replica bookkeeping of the benchmark
        sys.path.insert(0, ROOT)
        import bench
        slowest = bench.max_over_ranks(1.0 + rank, "cpu")
        job = bench.job_tflops(2e12, slowest, world)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{err!r} {slowest!r} {job!r}\n")
    finally:
        dist.destroy_process_group()


def test_partition_and_bench_bookkeeping_gloo_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    with tempfile.TemporaryDirectory() as out_dir:
        mp.start_processes(_gloo_worker, args=(world, _free_port(), out_dir), nprocs=world,
                           start_method="spawn", join=True)
        rows = []
        for r in range(world):
            with open(os.path.join(out_dir, f"rank{r}.txt")) as f:
                rows.append([float(x) for x in f.read().split()])
    for err, slowest, job in rows:
        assert err <= 1e-13
        assert slowest == 2.0                      # max over ranks of (1.0, 2.0) ms
        assert job == pytest.approx(2 * 2e12 / 2e-3 / 1e12)


def test_bench_cpulist_parser():
    """The sysfs CPU-list format the benchmark reads to place pinned buffers near the GPU."""
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()
