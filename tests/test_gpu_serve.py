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


def test_memory_budget_binds_defers_then_admits_with_identical_results():
    """A device-memory budget that holds one small batch at a time (library
    scratch of the tensor-core path included): admissions are deferred while a
    batch is in flight, every request is served once memory frees up, and
    each result equals the query computed alone."""
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 8)
    db = S.sanns_encode_db(ctx, torch.from_numpy(inputs.uniform_coords(3000, 8, 1)).cuda())
    S.sanns_db_prepare_batched(ctx, db)
    db.batched = True
    sk = S.sanns_keygen(ctx, 2)
    dbs = {"A": (ctx, db)}
    ex = GpuExecutor(dbs, slots=3, max_batch=16, batched_min=4, mask_seed=5)
    # the library reports the tensor path's scratch, and the executor counts it
    assert S.sanns_distances_scratch_bytes(ctx, 4, True) > 0
    assert S.sanns_distances_scratch_bytes(ctx, 4, False) == 0
    assert ex.bytes_for("A", 4) == 4 * ex.bytes_for("A", 1) + S.sanns_distances_scratch_bytes(ctx, 4, True)
    budget = ex.bytes_for("A", 4) + ex.bytes_for("A", 1) // 2   # one batch of 4 fits, two do not
    sched = Scheduler(ex, max_batch=16, slots=3, mem_budget=budget)
    reqs = []
    for rid in range(40):
        q = torch.from_numpy(inputs.uniform_coords(1, 8, 200 + rid)).cuda()
        qid = torch.tensor([rid], dtype=torch.int64).to(torch.uint64).cuda()
        reqs.append(Request(rid=rid, db="A", arrival=0.0,
                            payload=(S.sanns_encrypt_query(ctx, sk, q, 9, qid), qid)))
    torch.cuda.synchronize()
    stats = run_open_loop(sched, reqs)
    torch.cuda.synchronize()
    S.sanns_device_status(ctx)
    assert len(stats.latencies) == 40 and stats.rejected == 0
    assert stats.deferred > 0                          # memory, not slots, was the limit
    assert max(n for _, n, _ in stats.batches) <= 4
    assert ex.tensor_batches > 0                       # batches of 4 took the tensor-core path
    for r in reqs:
        solo_out, solo_srv = S.sanns_distances(ctx, db, r.payload[0], 5, r.payload[1])
        torch.cuda.synchronize()
        assert torch.equal(r.result[0].cpu(), solo_out.cpu()), r.rid
        assert torch.equal(r.result[1].cpu(), solo_srv.cpu()), r.rid


def test_calibration_tables_and_routing():
    """Calibration times both paths on each database; the executor then routes
    each batch size to the path its tables say is faster, and the results
    stay identical to the query computed alone."""
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 8)
    db = S.sanns_encode_db(ctx, torch.from_numpy(inputs.uniform_coords(3000, 8, 4)).cuda())
    S.sanns_db_prepare_batched(ctx, db)
    db.batched = True
    sk = S.sanns_keygen(ctx, 2)
    q = torch.from_numpy(inputs.uniform_coords(5, 8, 5)).cuda()
    qids = torch.arange(5, dtype=torch.int64).to(torch.uint64).cuda()
    ct = S.sanns_encrypt_query(ctx, sk, q, 9, qids)
    ex = GpuExecutor({"A": (ctx, db)}, slots=2, max_batch=16, batched_min=4, mask_seed=5)
    costs = ex.calibrate({"A": (ct, qids)}, per_query_sizes=(1, 2), tensor_sizes=(4, 16), reps=2)
    t = costs["A"]
    assert [b for b, _ in t["per_query"]] == [1, 2] and [b for b, _ in t["tensor"]] == [4, 16]
    assert all(ms > 0 for _, ms in t["per_query"] + t["tensor"])
    from paper_1904_02033_b300.serve import tensor_path_is_faster
    for n in (1, 3, 4, 9, 16):
        assert ex.uses_tensor_path("A", n) == (n >= 4 and tensor_path_is_faster(t["per_query"], t["tensor"], n))
    # forced routes: the tensor path wherever allowed, then never
    for tensor_ms in (0.0, float("inf")):
        ex.costs["A"]["tensor"] = [(1, tensor_ms), (2, tensor_ms)]
        before = ex.tensor_batches
        reqs = [Request(rid=i, db="A", arrival=0.0, payload=(ct[i:i + 1], qids[i:i + 1])) for i in range(5)]
        stats = run_open_loop(Scheduler(ex, max_batch=16, slots=1), reqs)
        torch.cuda.synchronize()
        S.sanns_device_status(ctx)
        assert len(stats.latencies) == 5
        assert (ex.tensor_batches > before) == (tensor_ms == 0.0)
        for r in reqs:
            solo_out, solo_srv = S.sanns_distances(ctx, db, r.payload[0], 5, r.payload[1])
            assert torch.equal(r.result[0], solo_out) and torch.equal(r.result[1], solo_srv), r.rid
