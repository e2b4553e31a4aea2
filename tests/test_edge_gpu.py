"""Edge cases of the newer entry points and plans, through the C ABI: degenerate spectra
for signed eigenvectors and Hermitian A, padded leading dimensions and index subsets,
the cluster plan under a budget too small for it, and a batch mixing plans."""
import numpy as np
import pytest

from paper_2002_04989_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


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


def padded(torch, A, extra=5, dtype=None):
    """A copy of A inside a wider device array (leading dimension n + extra)."""
    n = A.shape[0]
    dtype = dtype or (torch.complex128 if np.iscomplexobj(A) else torch.float64)
    big = torch.zeros((n, n + extra), dtype=dtype, device="cuda")
    big[:, :n] = torch.from_numpy(A).cuda()
    return big[:, :n]


def test_vectors_degenerate_rows_are_nan(torch_cuda, ctx):
    """Two equal eigenvalues make Eq. 1 0/0 for those rows: their vectors are NaN, the
    call warns, and the other rows are still the right unit vectors."""
    from paper_2002_04989_gb300 import eeid
    d = np.array([1.0, 1.0, 2.0, 3.5])
    A = torch_cuda.from_numpy(np.diag(d)).cuda()
    vec = ctx.eeid_eigenvectors(A).cpu().numpy()
    assert ctx.eeid_sync() == eeid.EEID_WARN_DEGENERATE
    assert np.isnan(vec[0]).all() and np.isnan(vec[1]).all()
    assert np.allclose(vec[2], [0, 0, 1, 0], atol=1e-14)
    assert np.allclose(vec[3], [0, 0, 0, 1], atol=1e-14)


def test_vectors_padded_and_unsorted_rows(torch_cuda, ctx, oracle_mod):
    A = inputs.goe(45, 450)
    lam_ref, vec_ref = oracle_mod.eigvecs(A, convention=True)
    rows = np.array([44, 3, 20, 0])
    out = ctx.eeid_eigenvectors(padded(torch_cuda, A), rows=rows).cpu().numpy()
    ctx.eeid_sync()
    assert np.max(np.abs(out - vec_ref[rows])) <= TOL


def test_herm_padded_subsets_and_degenerate(torch_cuda, ctx, oracle_mod):
    from paper_2002_04989_gb300 import eeid
    A = inputs.goe_herm(50, 501)
    rows, cols = np.array([49, 0, 17]), np.array([3, 48, 25, 1])
    out = ctx.eeid_components_herm(padded(torch_cuda, A), rows=rows, cols=cols).cpu().numpy()
    ctx.eeid_sync()
    ref = oracle_mod.components_herm(A, rows=rows, cols=cols, method=0)
    assert np.max(np.abs(out - ref)) <= TOL
    # a Hermitian matrix with a double eigenvalue: unitary similarity of diag(1, 1, 2, 3)
    g = np.random.default_rng(3)
    Q, _ = np.linalg.qr(g.standard_normal((4, 4)) + 1j * g.standard_normal((4, 4)))
    D = (Q * np.array([1.0, 2.0, 2.0, 3.0])) @ Q.conj().T
    D = np.tril(D) + np.tril(D, -1).conj().T
    ctx.eeid_components_herm(torch_cuda.from_numpy(D).cuda())
    assert ctx.eeid_sync() in (eeid.EEID_WARN_DEGENERATE, eeid.EEID_WARN_SMALL_GAP)


def test_cluster_plan_under_small_budget(torch_cuda):
    """With a budget that holds one working slot but not the two the cluster plan needs,
    the call falls back to one CTA per matrix in more rounds: same bits, no error."""
    from paper_2002_04989_gb300 import eeid
    p = inputs.planted(1002, 31, -1.0, 1.0, 1e-4)
    A = torch_cuda.from_numpy(p.A).cuda()
    outs = []
    for budget in (0, 12 << 20):
        c = eeid.Context(0, budget)
        try:
            outs.append(c.eeid_components(A, rows=[0, 500], cols=[7]).cpu().numpy())
            assert c.eeid_sync() >= 0
        finally:
            c.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.max(np.abs(outs[0][:, 0] - p.Q[7, [0, 500]] ** 2)) <= TOL


def test_batch_mixing_plans_bitwise(torch_cuda, ctx):
    """A batch holding a large matrix with one column (alone it would take the cluster
    plan) and small full problems: every result is bitwise its single-call result."""
    torch = torch_cuda
    mats = [inputs.planted(900, 5, -1.0, 1.0, 1e-4).A, inputs.goe(40, 6), inputs.goe(130, 7)]
    cols = [[11], None, [0, 64, 129]]
    probs, singles = [], []
    for A, cl in zip(mats, cols):
        n = A.shape[0]
        dA = torch.from_numpy(A).cuda()
        nc = n if cl is None else len(cl)
        probs.append({"A": dA, "cols": cl, "out": torch.empty((n, nc), dtype=torch.float64,
                                                                device="cuda")})
        singles.append(ctx.eeid_components(dA, cols=cl).cpu().numpy())
        ctx.eeid_sync()
    ctx.eeid_components_batched(probs)
    ctx.eeid_sync()
    for pr, s in zip(probs, singles):
        assert np.array_equal(pr["out"].cpu().numpy(), s)


def test_vectors_diagonal_one_reference_each(torch_cuda, ctx):
    """A diagonal matrix (n = 300): every eigenvector is a unit vector, so each needs its
    own reference (300 of them); components whose |v_ij|^2 came out exactly 0 need no
    rotated minor.  The result is the permuted identity within the bar."""
    d = np.random.default_rng(9).permutation(np.linspace(-2.0, 3.0, 300))
    A = torch_cuda.from_numpy(np.diag(d)).cuda()
    vec = ctx.eeid_eigenvectors(A).cpu().numpy()
    ctx.eeid_sync()
    assert ctx.eeid_vector_refs() == 300
    ref = np.zeros((300, 300))
    ref[np.arange(300), np.argsort(d)] = 1.0
    assert np.max(np.abs(vec - ref)) <= TOL
