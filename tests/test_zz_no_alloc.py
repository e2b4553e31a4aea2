"""eeid_eigvals_noalloc: the entry point for callers that cannot allocate device
memory (their application's memory pool owns the device, or cudaMalloc's implicit
synchronisation is not acceptable on their path).  Its scratch is a fixed device
array inside the library, so it serves n <= 512.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.  It must pass alone in a fresh process
and after the other tests."""
import numpy as np
import pytest

from paper_2002_04989_gb300 import eeid, inputs

TOL_LAM_REL = 1e-12   # the library's eigenvalue bar (max abs error / ||A||_2)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = eeid.load()
    # no GPU work happens: the size check comes first
    st = lib.eeid_eigvals_noalloc(None, 513, 513, None, None)
    assert st == eeid.EEID_ERR_INVALID
    assert "512" in eeid.last_error()


@pytest.mark.gpu
def test_noalloc_matches_eeid_eigvals_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    ctx = eeid.Context(0)
    try:
        # two calls in a row, different sizes, so stale scratch from the first call
        # cannot leak into the second
        for n, seed in ((300, 11), (97, 12)):
            A = torch.from_numpy(inputs.goe(n, seed)).cuda()
            ref = ctx.eeid_eigvals(A)
            ctx.eeid_sync()
            lam = eeid.eeid_eigvals_noalloc(A)
            torch.cuda.synchronize()
            ref_h, lam_h = ref.cpu().numpy(), lam.cpu().numpy()
            norm = max(abs(ref_h[0]), abs(ref_h[-1]))
            assert np.all(np.diff(lam_h) >= 0)
            assert np.max(np.abs(lam_h - ref_h)) <= TOL_LAM_REL * norm, (n, np.max(np.abs(lam_h - ref_h)))
    finally:
        ctx.close()
