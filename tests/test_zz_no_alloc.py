"""eeid_eigvals_noalloc: the entry point for callers that cannot allocate device
memory (their application's memory pool owns the device, or cudaMalloc's implicit
synchronisation is not acceptable on their path).  Its scratch is a fixed device
array inside the library, so it serves n <= 512.

The first GPU test makes its first call before any context exists in this module,
so in a fresh process it exercises the entry point's own first-call set-up (the
scratch address lookup and the kernel loading).  Reference values come from the
long-double oracle (n <= 97) or from planted spectra, whose eigenvalues are known
by construction; the last test also checks two calls in a row against
eeid_eigvals.

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
    st = lib.eeid_eigvals_noalloc(None, 513, 513, None, None, None)
    assert st == eeid.EEID_ERR_INVALID
    assert "512" in eeid.last_error()


def test_binding_checks_outputs_on_the_host():
    """The binding refuses outputs the kernels could write past (wrong type or size)
    before anything reaches the library."""
    import torch
    with pytest.raises(TypeError):
        eeid._out(torch.empty(4, dtype=torch.float64), 4, torch.empty(1), "out")
    with pytest.raises(TypeError):
        eeid._hout(np.empty(4, dtype=np.float32), 4, "out")
    with pytest.raises(ValueError):
        eeid._hout(np.empty(3), 4, "out")
    with pytest.raises(TypeError):
        eeid._hout(np.empty((4, 4))[:, ::2], 4, "out")


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return torch


def _check_against(torch, A_dev, lam_ref, norm):
    """One no-alloc call with a status word pre-filled with ones; the call must clear
    it and report no size failure."""
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    lam = eeid.eeid_eigvals_noalloc(A_dev, status=status)
    torch.cuda.synchronize()
    bits = int(status.item()) & 0xffffffff
    assert bits & ~eeid.EEID_DEV_BRACKET_FALLBACK == 0, hex(bits)
    got = lam.cpu().numpy()
    assert np.all(np.diff(got) >= 0)
    err = float(np.max(np.abs(got - lam_ref))) if got.size else 0.0
    assert err <= TOL_LAM_REL * norm, (A_dev.shape[0], err)
    return got


@pytest.mark.gpu
def test_noalloc_against_oracle_and_planted_first_calls(oracle_mod):
    torch = _cuda()
    # tiny and small cases against the long-double oracle
    for n, seed in ((1, 3), (2, 4), (97, 12)):
        A = inputs.goe(n, seed)
        ref = oracle_mod.eigvals(A)
        norm = max(abs(ref[0]), abs(ref[-1]))
        _check_against(torch, torch.from_numpy(A).cuda(), ref, norm)
    # the size limit itself and a padded leading dimension, against planted spectra
    p = inputs.planted(512, 31, -1.0, 1.0, 1e-4)
    _check_against(torch, torch.from_numpy(p.A).cuda(), p.lam, 1.0)
    q = inputs.planted(300, 32, -2.0, 2.0, 1e-3)
    big = torch.zeros((300, 303), dtype=torch.float64, device="cuda")
    big[:, :300] = torch.from_numpy(q.A).cuda()
    padded = big[:, :300]
    assert padded.stride(0) == 303
    _check_against(torch, padded, q.lam, 2.0)


@pytest.mark.gpu
def test_noalloc_matches_eeid_eigvals_two_calls():
    torch = _cuda()
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
