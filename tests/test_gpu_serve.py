"""Serving on the GPU: each request's result is the same when served in a
mix of concurrent batches (continuous batching, tensor-core path for large
batches) as when computed alone."""
import numpy as np
import pytest
import torch

from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S
from paper_1904_02033_b300.serve import GpuExecutor, Request, Scheduler, run_open_loop

pytestmark = pytest.mark.gpu


def test_results_identical_alone_and_in_the_mix():
    dbs, keys = {}, {}
    for name, (d, n) in {"A": (8, 900), "B": (16, 2000)}.items():
        ctx = S.sanns_ctx_create(256, 2, 40, 0, d)
        db = S.sanns_encode_db(ctx, torch.from_numpy(inputs.uniform_coords(n, d, n)).cuda())
        S.sanns_db_prepare_batched(ctx, db)
        db.batched = True
        dbs[name] = (ctx, db)
        keys[name] = S.sanns_keygen(ctx, 3)
    rnd = np.random.default_rng(0)
    reqs = []
    t = 0.0
    for rid in range(60):
        name = "A" if rnd.random() < 0.5 else "B"
        ctx, _ = dbs[name]
        q = torch.from_numpy(inputs.uniform_coords(1, ctx.d, 100 + rid)).cuda()
        qid = torch.tensor([rid], dtype=torch.int64).to(torch.uint64).cuda()
        ct = S.sanns_encrypt_query(ctx, keys[name], q, 7, qid)
        t += float(rnd.exponential(2e-4))
        reqs.append(Request(rid=rid, db=name, arrival=t, payload=(ct, qid)))
    torch.cuda.synchronize()
    ex = GpuExecutor(dbs, slots=3, max_batch=16, batched_min=4, mask_seed=5)
    sched = Scheduler(ex, max_batch=16, slots=3)
    stats = run_open_loop(sched, reqs)
    torch.cuda.synchronize()
    for name, (ctx, _) in dbs.items():
        S.sanns_device_status(ctx)
    assert len(stats.latencies) == 60
    assert max(n for _, n, _ in stats.batches) > 1        # batching happened
    for r in reqs:
        ctx, db = dbs[r.db]
        solo_out, solo_srv = S.sanns_distances(ctx, db, r.payload[0], 5, r.payload[1])
        torch.cuda.synchronize()
        assert torch.equal(r.result[0].cpu(), solo_out.cpu()), r.rid
        assert torch.equal(r.result[1].cpu(), solo_srv.cpu()), r.rid
