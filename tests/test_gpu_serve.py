"""Serving on the GPU: every request's result is the same alone and in the
mix (bit-exact: integer protocol), and equals the oracle element by element."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_04909_gb300 import Context, Params
from paper_2309_04909_gb300 import workloads as W
from paper_2309_04909_gb300.serve import Engine, ServingSetup
from tests._util import to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SEED = 0x5E21E


def test_serving_results_identical_alone_and_in_mix():
    ctx = Context(SEED)
    prm = Params(64, 24, 0)
    setup = ServingSetup(ctx, prm, budget_bytes=2 << 30, seed=4, pool_images=4)
    trace = W.serving_trace(rate_per_s=4000.0, duration_s=0.02, seed=4, max_images=4)
    reqs = setup.requests_from_trace(trace)
    assert len(reqs) > 20
    # the first half arrive together, so iterations are shared whatever the
    # GPU's speed; the rest keep their Poisson arrivals
    for r in reqs[:len(reqs) // 2]:
        r.arrival_s = 0.0
    for sched in (1, 0):
        for r in reqs:
            r.offset = r.admitted_s = r.finished_s = None
            r.done = r.retired = 0
        got = {}

        def keep(r):   # snapshot before the engine frees (and later reuses) the block
            m0, m1 = setup.outputs(r)
            got[r.rid] = (m0.clone(), m1.clone())

        stats = Engine(setup.executor(schedule=sched), setup.budget, max_iter_elems=1 << 20,
                       min_chunk=1 << 14).run(reqs, on_complete=keep)
        torch.cuda.synchronize()
        assert stats.completed == len(reqs) == len(got)
        assert stats.iterations < len(reqs)          # requests shared iterations
        for r in reqs:
            i0, i1 = setup.inputs(r)
            a0, a1 = ctx.relu(prm, i0.contiguous(), i1.contiguous(), tensor_id=setup.tensor_id(r))
            m0, m1 = got[r.rid]
            assert torch.equal(a0, m0) and torch.equal(a1, m1), r.rid
    # every element of every request against the oracle
    P = O.params(64, 24, 0)
    for r in reqs:
        i0, i1 = setup.inputs(r)
        e0, e1 = O.relu(P, to_np(i0), to_np(i1), SEED, setup.tensor_id(r),
                        threads=O.max_threads())
        m0, m1 = got[r.rid]
        assert np.array_equal(to_np(m0), e0) and np.array_equal(to_np(m1), e1), r.rid
    ctx.close()
