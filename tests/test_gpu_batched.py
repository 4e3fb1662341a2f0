"""GPU parity of the batched tensor-core MAC: its ciphertexts must be
bit-identical to the plain per-query path and to the oracle."""
import numpy as np
import pytest
import torch

from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("tile", [0, 1], ids=["tile128", "tile256pair"])
@pytest.mark.parametrize("cfg,n,B", [
    ((256, 2, 40, 0, 16), 700, 3),          # one ragged N tile, partial M tile
    ((256, 3, 60, 0, 96), 256 * 300, 9),    # two N tiles (K = 300), three M tiles
    ((64, 2, 50, 0, 13), 64 * 5 - 1, 1),    # d not a multiple of 8, B = 1
    ((8192, 3, 60, 0, 128), 8192 * 2 + 5, 2),  # d = 128: partial sums up to 2^24
    ((256, 2, 60, 0, 24), 256 * 600 - 3, 20),  # 40 query rows: two query tiles, K = 600
])
def test_batched_equals_plain_and_oracle(cfg, n, B, tile):
    N, L, bits, rule, d = cfg
    ctx = S.sanns_ctx_create(*cfg)
    S.sanns_batched_tune(ctx, tile=tile)
    rnd = np.random.default_rng(n + B)
    coords = rnd.integers(0, 256, size=(n, d), dtype=np.uint8)
    coords[: min(n, 50)] = 255      # extreme digits on the database side
    perm = inputs.permutation(n, 3)
    q = rnd.integers(0, 256, size=(B, d), dtype=np.uint8)
    qids = cu(np.arange(10, 10 + B, dtype=np.uint64))
    sk = S.sanns_keygen(ctx, 4)
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    S.sanns_db_prepare_batched(ctx, db)
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 5, qids)
    plain_out, plain_srv = S.sanns_distances(ctx, db, ct_in, 6, qids)
    acc_plain = S.sanns_distances_mac(ctx, db, ct_in)
    acc_batch = S.sanns_distances_batched_mac(ctx, db, ct_in)
    S.sanns_device_status(ctx)
    assert torch.equal(acc_batch.cpu(), acc_plain.cpu())
    bout, bsrv = S.sanns_distances_batched(ctx, db, ct_in, 6, qids)
    S.sanns_device_status(ctx)
    assert torch.equal(bout.cpu(), plain_out.cpu())
    assert torch.equal(bsrv.cpu(), plain_srv.cpu())
    if N <= 256:
        O = Oracle(*cfg)
        out0, srv0 = O.distances(ct_in.cpu().numpy()[0], coords, perm, 6, 10)
        assert np.array_equal(bout.cpu().numpy()[0], out0)
        s, _ = O.keygen(4)
        cli = O.decrypt_shares(out0, s, q[0], n)
        brute = np.sum((coords[perm].astype(np.int64) - q[0].astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((cli.astype(np.int64) + srv0) % O.t, brute)


def test_batched_needs_prepare_and_small_d():
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 200)
    db = S.sanns_encode_db(ctx, cu(inputs.uniform_coords(300, 200, 1)))
    with pytest.raises(S.SannsError):
        S.sanns_db_prepare_batched(ctx, db)
    ct = torch.zeros((1, 200, 2, 2, 256), dtype=torch.uint64, device="cuda")
    with pytest.raises(S.SannsError):
        S.sanns_distances_batched_mac(ctx, db, ct)


def test_batched_autotune_keeps_results_identical():
    cfg = (256, 2, 40, 0, 16)
    n, B = 256 * 40 + 7, 5
    ctx = S.sanns_ctx_create(*cfg)
    coords = inputs.uniform_coords(n, cfg[4], 21)
    q = inputs.uniform_coords(B, cfg[4], 22)
    qids = cu(np.arange(B, dtype=np.uint64))
    sk = S.sanns_keygen(ctx, 23)
    db = S.sanns_encode_db(ctx, cu(coords), cu(inputs.permutation(n, 24)))
    S.sanns_db_prepare_batched(ctx, db)
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 25, qids)
    out = torch.empty((B, db.K, 2, 2, 256), dtype=torch.uint64, device="cuda")
    idx, ms = S.sanns_autotune_batched(ctx, db, ct_in, out, reps=1)
    assert 0 <= idx < len(S.BATCHED_CONFIGS) and len(ms) == len(S.BATCHED_CONFIGS)
    assert all(m > 0 for m in ms)
    acc_plain = S.sanns_distances_mac(ctx, db, ct_in)
    assert torch.equal(out.cpu(), acc_plain.cpu())
    acc_b = S.sanns_distances_batched_mac(ctx, db, ct_in)
    S.sanns_device_status(ctx)
    assert torch.equal(acc_b.cpu(), acc_plain.cpu())


def test_measured_tensor_rates_rank_the_instruction_families():
    """The library's rate probe: the tcgen05 fp16 MMA the batched kernel uses
    is faster than the legacy fp16 mma.sync, which is faster per operation
    than the legacy s8 mma.sync (the only INT8 tensor instruction on sm_103a)."""
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 8)
    r = S.sanns_measure_mma_rates(ctx)
    assert r["tcgen05_f16_tflops"] > r["mma_sync_f16_tflops"] > r["mma_sync_s8_tops"] > 0
    # sanity bound: no more than the nominal dense fp16 peak plus margin
    assert r["tcgen05_f16_tflops"] < 3000
