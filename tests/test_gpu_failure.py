"""Failure detection on the GPU without a fault: a bounded device wait runs out.

The tensor-core kernels bound every mbarrier wait; on expiry they record the site in a
device flag, stop, release tensor memory and return.  dmrg2d_wait_selftest drives that
routine on an mbarrier nothing arrives on (a 50 ms limit); the status comes back as
ETIMEOUT and the context keeps working.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.superblock import Superblock  # noqa: E402
from paper_0707_0159_gb300 import dmrg2d, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    code = dmrg2d.wait_selftest(0.05)
    assert code == -6, dmrg2d.last_error()
    assert "gave up" in dmrg2d.last_error()
    # the same context still computes: a small FP64 H·v against the oracle
    mdl, left, right, _ = synth.workload_ladder2_heisenberg_m64()
    ops = dmrg2d.build_ops(mdl, left, right)
    sb = Superblock(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 8)
    x = torch.from_numpy(v).cuda()
    y = torch.empty_like(x)
    dmrg2d.apply_H(ops, x, y, dmrg2d.FP64)
    torch.cuda.synchronize()
    dmrg2d.check_device(ops)
    ref = sb.apply(v)
    assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    # and a second give-up is reported again
    assert dmrg2d.wait_selftest(0.02) == -6
