"""A state split over 2^g shards (Section 2.2, step 2) with every shard held by the CUDA
library on one GPU: the shard planner's schedule (pairwise half-shard exchanges for gates on
global qubits, Section 3.1) with the library's kernels for the local gates reproduces the
FP64 oracle's run of the whole state."""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07140_gb300 import build
    build.build()
    import paper_2008_07140_gb300 as q
    return q


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-6)])
@pytest.mark.parametrize("n,g", [(14, 1), (15, 2)])
def test_qsim_shards_on_one_gpu_reproduce_the_oracle(qs, dtype, tol, n, g):
    from paper_2008_07140_gb300 import sharded
    from test_sharded import mixed_ops
    ops = mixed_ops(n, seed=100 + n)
    gates = sharded.expand_for_shards(n, ops)
    shards = [sharded.QsimShard(n - g, dtype, first=(r == 0)) for r in range(1 << g)]
    ex = sharded.LocalShards(n, g, shards)
    ex.run_gates(gates)
    got = ex.to_numpy()
    ref = oracle.run(n, ops)
    assert ex.planner.exchanges > 0
    assert np.max(np.abs(got - ref)) <= tol
    for s in shards:
        s.close()
