"""Served streams: each stream's results are the same alone and in the continuous-batching mix."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_served_equals_alone_and_oracle():
    import torch

    import paper_1503_06203_gb300 as xe
    from paper_1503_06203_gb300 import serve
    xe.build()
    specs = [serve.StreamSpec(64, 4), serve.StreamSpec(128, 2), serve.StreamSpec(256, 1), serve.StreamSpec(64, 8)]
    t_max = 1024
    pool_bytes = 8 << 20
    pool_np = synth.gauss_flat(pool_bytes, 2.5, 4242)
    pool = torch.from_numpy(pool_np).pin_memory()
    arrivals = serve.poisson_arrivals(2000.0, 96, len(specs), 256, t_max, pool_bytes, specs, 9)
    # served (bursty arrivals, so launches carry several frames), readout every 4 frames
    srv = serve.Server(specs, t_max, pool, budget_bytes=2 << 20, readout_every=4)
    srv.keep_readouts = True
    st = srv.run_served(arrivals)
    served = [list(r) for r in srv.readouts]
    assert st.frames == len(arrivals) and np.isfinite(st.latencies_ms).all()
    # each stream alone: its own frames, one per launch
    for sid in range(len(specs)):
        alone = serve.Server([specs[sid]], t_max, pool, budget_bytes=2 << 20, readout_every=4)
        alone.keep_readouts = True
        mine = [serve.Arrival(a.t, 0, a.T, a.offset) for a in arrivals if a.stream == sid]
        alone.run_plain(mine)
        assert len(alone.readouts[0]) == len(served[sid])
        for a, b in zip(alone.readouts[0], served[sid]):
            assert torch.equal(a, b)
        # and the first integration against the oracle
        if served[sid]:
            s = specs[sid]
            frames = [pool_np[a.offset:a.offset + a.T * s.F * s.N].reshape(a.T, s.F, s.N) for a in mine[:4]]
            ref = sum(oracle.visibilities(np.ascontiguousarray(x)) for x in frames)
            assert np.array_equal(served[sid][0].numpy().astype(np.int64), ref)
