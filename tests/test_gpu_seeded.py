"""Seeded query ciphertexts: the server rebuilds c1 from the encryption seed
and the query ids, so the client sends c0 alone.  The rebuilt ciphertexts are
bit-identical to the full encryption on the GPU and to the oracle's."""
import numpy as np
import pytest
import torch

from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg,B", [((256, 2, 40, 0, 5), 3), ((8192, 3, 60, 0, 7), 2),
                                   ((64, 1, 60, 0, 224), 1)])
def test_expanded_query_equals_encryption_and_oracle(cfg, B):
    ctx = S.sanns_ctx_create(*cfg)
    d = cfg[4]
    q = inputs.uniform_coords(B, d, 21)
    qids = torch.from_numpy(np.arange(40, 40 + B, dtype=np.uint64)).cuda()
    sk = S.sanns_keygen(ctx, 22)
    ct = S.sanns_encrypt_query(ctx, sk, torch.from_numpy(q).cuda(), 23, qids)
    rebuilt = S.sanns_expand_query(ctx, ct[:, :, 0].contiguous(), 23, qids)
    assert torch.equal(rebuilt, ct)
    # from the oracle's ciphertexts: their c0 alone gives back the whole
    O = Oracle(*cfg)
    _, s_hat = O.keygen(22)
    oct_ = np.stack([O.encrypt(s_hat, q[b], 23, 40 + b) for b in range(B)])
    c0 = torch.from_numpy(np.ascontiguousarray(oct_[:, :, 0])).cuda()
    assert np.array_equal(S.sanns_expand_query(ctx, c0, 23, qids).cpu().numpy(), oct_)


def test_overlapping_buffers_rejected():
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 5)
    B, d, L, N = 2, 5, 2, 256
    buf = torch.zeros(B * d * 2 * L * N, dtype=torch.uint64, device="cuda")
    c0 = buf[:B * d * L * N].view(B, d, L, N)
    qids = torch.zeros(B, dtype=torch.uint64, device="cuda")
    with pytest.raises(S.SannsError) as e:
        S.sanns_expand_query(ctx, c0, 1, qids, out=buf.view(B, d, 2, L, N))
    assert e.value.code == -1
