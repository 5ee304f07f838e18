"""Radius / lookup diagnostics (Fig. 3 and Fig. 9 analogues): the single-table
lookup count is Eq. 1, and the radii are the oracle's k-th distances."""
import math

import numpy as np
import pytest

from paper_1307_2982_gb300 import synth


def test_sht_lookups_is_the_hamming_ball():
    from paper_1307_2982_gb300.diagnostics import sht_lookups_log10

    for q in (64, 128, 256):
        for r in (0, 1, 5, 20, q):
            want = math.log10(sum(math.comb(q, d) for d in range(r + 1)))
            assert abs(sht_lookups_log10(q, np.array([r]))[0] - want) < 1e-12
        assert abs(sht_lookups_log10(q, np.array([q]))[0] - q * math.log10(2)) < 1e-9


@pytest.mark.gpu
def test_profile_radii_are_oracle_kth_distances(gpu_lib, orc):
    import torch

    from paper_1307_2982_gb300.diagnostics import search_profile

    mih = gpu_lib
    q, n = 128, 50_000
    db, qs = synth.lsh_codes(n, q, 0), synth.lsh_codes(64, q, 1)
    codes = torch.from_numpy(db.view(np.int64)).cuda()
    queries = torch.from_numpy(qs.view(np.int64)).cuda()
    ix = mih.mih_build(codes, q, 4)
    prof = search_profile(ix, queries, [1, 10, 100])
    for k in (1, 10, 100):
        _, want_dist = orc.knn(db, qs, k)
        radius = want_dist[:, k - 1]
        hist = np.bincount(radius, minlength=q + 1)
        got = prof["per_k"][str(k)]
        assert got["radius_hist"] == {str(d): int(c) for d, c in enumerate(hist) if c}
        assert abs(got["radius_mean"] - radius.mean()) < 1e-9
        assert got["linear_scan_comparisons"] == n
        assert got["mih_lookups_mean"] > 0
    ix.free()
