"""The allocation-free signing entry point gives the same hashes as pmh_minhash_sign.

pmh_minhash_sign_noalloc serves callers that cannot let a library allocate device
memory (a fixed device-memory budget reserved up front, memory owned by a caching
allocator, latency-critical loops that cannot absorb cudaFree's device-wide
synchronisation).  Its scratch is one fixed device array shared by every call, so the
test makes two calls in a row on different inputs -- the second must not see the
first one's ticket or bounding boxes -- and compares both with the ordinary entry
point.  Hashes are integers: the comparison is exact.  This file is collected last so
that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

from paper_2511_16576_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def B():
    from paper_2511_16576_gb300 import binding, build
    build.build()
    return binding


def test_noalloc_matches_sign_on_two_calls(B):
    ctx = B.Context(0)
    try:
        first = synth.star_polygons(3000, 91, (8, 300), "loguniform", (1e-3, 3e-2))
        second = synth.star_polygons(700, 92, (3, 64), "uniform", (5e-3, 5e-2))
        for ps, (K, bands, T) in ((first, (128, 16, 1 << 24)), (second, (40, 8, 5000))):
            P = B.make_params(K, bands, T)
            xy = torch.from_numpy(ps.xy).to(DEV)
            off = torch.from_numpy(ps.offsets).to(DEV)
            ref = B.minhash_sign(ctx, B.poly_upload(ctx, xy, off), P)
            got = B.minhash_sign_noalloc(xy, off, P)
            torch.cuda.synchronize()
            assert torch.equal(got, ref)
            assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())
    finally:
        ctx.close()


def test_noalloc_rejects_oversized_batches(B):
    n = B.NOALLOC_MAX_POLYS + 1
    off = torch.arange(n + 1, device=DEV, dtype=torch.int64) * 3
    xy = torch.zeros((3, 2), dtype=torch.int32, device=DEV)
    with pytest.raises(B.PmhError) as ei:
        B.minhash_sign_noalloc(xy, off, B.make_params(32, 8), out=torch.empty(1, device=DEV))
    assert "at most" in str(ei.value)


def test_noalloc_reports_invalid_polygons(B):
    xy = torch.tensor([[0, 0], [5, 0], [0, 5], [1, 1], [2, 2]], dtype=torch.int32, device=DEV)
    off = torch.tensor([0, 3, 5], dtype=torch.int64, device=DEV)   # second has 2 vertices
    with pytest.raises(B.PmhError) as ei:
        B.minhash_sign_noalloc(xy, off, B.make_params(32, 8))
    assert "fewer than 3" in str(ei.value)
