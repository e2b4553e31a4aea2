"""Complex Hermitian A (eeid_components_herm): Sec. 2 states Eq. 1 for Hermitian
matrices.  The CUDA path reduces A and its minors with unitary Householder reflectors to
real tridiagonals; checked through the C ABI against the long-double oracle (real
symmetric embedding), the Hermitian Toeplitz closed form and planted unitary Q.
Bars as for the real path: |v_ij|^2 within 1e-10, eigenvalues within 1e-12 ||A||_2."""
import numpy as np
import pytest

from paper_2002_04989_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_VSQ = 1e-10
TOL_LAM_REL = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    from paper_2002_04989_gb300 import eeid
    c = eeid.Context(0)
    yield c
    c.close()


def herm_run(torch, ctx, A, rows=None, cols=None):
    dA = torch.from_numpy(np.ascontiguousarray(A, dtype=np.complex128)).cuda()
    lam = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    out = ctx.eeid_components_herm(dA, rows=rows, cols=cols, lam=lam)
    st = ctx.eeid_sync()
    assert st >= 0
    return out.cpu().numpy(), lam.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 3, 17, 33, 64, 100])
def test_herm_against_oracle(torch_cuda, ctx, oracle_mod, n):
    A = inputs.goe_herm(n, 600 + n)
    out, lam = herm_run(torch_cuda, ctx, A)
    ref, lam_ref = oracle_mod.components_herm(A, method=0, want_eigs=True)
    norm = max(abs(lam_ref[0]), abs(lam_ref[-1]))
    assert np.max(np.abs(lam - lam_ref)) <= TOL_LAM_REL * norm
    bar = TOL_VSQ if inputs.min_relative_gap(lam_ref) >= 1e-4 else 1e-6
    err = float(np.max(np.abs(out - ref)))
    print(f"herm n={n}: max|d vsq| = {err:.2e}")
    assert err <= bar


def test_herm_toeplitz_with_phase(torch_cuda, ctx):
    n, theta = 48, 0.9
    A = np.zeros((n, n), dtype=complex)
    idx = np.arange(n - 1)
    A[idx + 1, idx] = np.exp(1j * theta)
    A[idx, idx + 1] = np.exp(-1j * theta)
    out, lam = herm_run(torch_cuda, ctx, A)
    k = np.arange(1, n + 1)
    lam_c = np.sort(2 * np.cos(k * np.pi / (n + 1)))
    vsq_c = 2.0 / (n + 1) * np.sin(np.outer(k, k) * np.pi / (n + 1)) ** 2
    assert np.max(np.abs(lam - lam_c)) <= 1e-13
    assert np.max(np.abs(out - vsq_c)) <= TOL_VSQ


@pytest.mark.parametrize("n", [300, 1024])
def test_herm_planted(torch_cuda, ctx, n):
    p = inputs.planted_herm(n, 700 + n, -1.0, 1.0, 1e-4)
    rng = np.random.default_rng(n)
    cols = np.sort(rng.choice(n, 24, replace=False))
    out, lam = herm_run(torch_cuda, ctx, p.A, cols=cols)
    ref = (np.abs(p.Q) ** 2).T[:, cols]
    err = float(np.max(np.abs(out - ref)))
    print(f"herm planted n={n}: max|d vsq| = {err:.2e}")
    assert err <= TOL_VSQ
    assert np.max(np.abs(lam - p.lam)) <= TOL_LAM_REL


def test_herm_real_input_and_limits(torch_cuda, ctx):
    from paper_2002_04989_gb300 import eeid
    A = inputs.goe(80, 81)
    out_c, lam_c = herm_run(torch_cuda, ctx, A.astype(complex))
    out_r = ctx.eeid_components(torch_cuda.from_numpy(A).cuda()).cpu().numpy()
    ctx.eeid_sync()
    assert np.max(np.abs(out_c - out_r)) <= 1e-12
    big = torch_cuda.zeros((2049, 2049), dtype=torch_cuda.complex128, device="cuda")
    with pytest.raises(eeid.EeidError) as ei:
        ctx.eeid_components_herm(big, rows=[0], cols=[0])
    assert ei.value.status == eeid.EEID_ERR_INVALID
