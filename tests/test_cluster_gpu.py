"""The cluster plan (latency mode, eeid_set_clusters): a call with few large reductions
(a single component, a few columns, the eigenvalues of one A) reduces each matrix on a
thread-block cluster of up to 16 CTAs, and with mode 2 the fewest largest ones on a
cooperative group of sms / nt > 16 CTAs.  The results must be bitwise those of the
one-CTA plan, and match the planted closed form Q o Q within the library's bar; the
single-component call (the paper's Table 1 task) must also be faster.  The group plan's
bounded barrier is checked by its self-test (a group with a CTA missing)."""
import time

import numpy as np
import pytest

from paper_2002_04989_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_VSQ = 1e-10


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
    c.eeid_set_clusters(2)
    c.close()


def run(torch, ctx, A, rows, cols, clusters):
    ctx.eeid_set_clusters(clusters)
    n = A.shape[0]
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    out = ctx.eeid_components(A, rows=rows, cols=cols, lam=lam)
    assert ctx.eeid_sync() >= 0
    return out.cpu().numpy(), lam.cpu().numpy()


@pytest.mark.parametrize("n,cols", [(520, [3]), (1002, [0]), (1002, [5, 400, 1001]),
                                    (700, list(range(0, 700, 35)))])
def test_cluster_bitwise_and_closed_form(torch_cuda, ctx, n, cols):
    p = inputs.planted(n, 1300 + n, -1.0, 1.0, 1e-4)
    A = torch_cuda.from_numpy(p.A).cuda()
    rows = np.unique(np.r_[0, n // 3, n - 1])
    got_c, lam_c = run(torch_cuda, ctx, A, rows, cols, True)
    got_p, lam_p = run(torch_cuda, ctx, A, rows, cols, False)
    assert np.array_equal(got_c, got_p) and np.array_equal(lam_c, lam_p)
    ref = (p.Q * p.Q).T[np.ix_(rows, cols)]
    assert np.max(np.abs(got_c - ref)) <= TOL_VSQ
    assert np.max(np.abs(lam_c - p.lam)) <= 1e-12


def test_cluster_eigvals_and_minors_bitwise(torch_cuda, ctx):
    A = torch_cuda.from_numpy(inputs.goe(1500, 77)).cuda()
    out = {}
    for cl in (True, False):
        ctx.eeid_set_clusters(cl)
        lam = ctx.eeid_eigvals(A)
        mu = ctx.eeid_minor_eigvals(A, cols=[0, 749, 1499])
        ctx.eeid_sync()
        out[cl] = (lam.cpu().numpy(), mu.cpu().numpy())
    assert np.array_equal(out[True][0], out[False][0])
    assert np.array_equal(out[True][1], out[False][1])


@pytest.mark.parametrize("n,cols", [(1600, [7]), (2100, [0, 1050, 2099])])
def test_group_plan_bitwise_and_closed_form(torch_cuda, ctx, n, cols):
    """Two or four reductions of m >= 1536: mode 2 runs each on 76 or 38 CTAs that meet at
    global-memory barriers; same bits as the one-CTA plan and the cluster plan."""
    p = inputs.planted(n, 1700 + n, -1.0, 1.0, 1e-4)
    A = torch_cuda.from_numpy(p.A).cuda()
    rows = np.unique(np.r_[0, n // 3, n - 1])
    got_g, lam_g = run(torch_cuda, ctx, A, rows, cols, 2)
    got_c, lam_c = run(torch_cuda, ctx, A, rows, cols, 1)
    got_p, lam_p = run(torch_cuda, ctx, A, rows, cols, 0)
    assert np.array_equal(got_g, got_p) and np.array_equal(lam_g, lam_p)
    assert np.array_equal(got_c, got_p)
    ref = (p.Q * p.Q).T[np.ix_(rows, cols)]
    assert np.max(np.abs(got_g - ref)) <= TOL_VSQ
    assert np.max(np.abs(lam_g - p.lam)) <= 1e-12


def test_group_plan_eigvals_bitwise(torch_cuda, ctx):
    """The eigenvalues of one n = 3000 matrix: a single group of every SM."""
    A = torch_cuda.from_numpy(inputs.goe(3000, 78)).cuda()
    out = {}
    for mode in (2, 0):
        ctx.eeid_set_clusters(mode)
        out[mode] = ctx.eeid_eigvals(A).cpu().numpy()
        assert ctx.eeid_sync() >= 0
    assert np.array_equal(out[2], out[0])


def test_group_barrier_timeout_reported(torch_cuda, ctx):
    """A group whose partner CTA never arrives gives up after the wait limit: eeid_sync
    reports EEID_ERR_TIMEOUT, and the context keeps working afterwards."""
    from paper_2002_04989_gb300 import eeid
    ctx.eeid_check_barrier_timeout()
    with pytest.raises(eeid.EeidError) as ei:
        ctx.eeid_sync()
    assert ei.value.status == eeid.EEID_ERR_TIMEOUT
    assert ctx.eeid_sync() == 0          # the word was cleared by the read
    p = inputs.planted(300, 31, -1.0, 1.0, 1e-4)
    out = ctx.eeid_components(torch_cuda.from_numpy(p.A).cuda(), cols=[4])
    assert ctx.eeid_sync() == 0
    assert np.max(np.abs(out.cpu().numpy()[:, 0] - p.Q[4] ** 2)) <= TOL_VSQ


def test_single_component_n4002(torch_cuda, ctx):
    """One component of an n = 4002 planted matrix (the largest Table 1 size the
    library's n <= 4096 limit allows near 4002): against Q o Q, and faster than the
    one-CTA plan."""
    torch = torch_cuda
    p = inputs.planted(4002, 4002, -1.0, 1.0, 1e-4)
    A = torch.from_numpy(p.A).cuda()
    i, j = 1234, 2001
    times = {}
    for cl in (2, True, False):
        ctx.eeid_set_clusters(cl)
        ctx.eeid_components(A, rows=[i], cols=[j])     # warm-up (workspace sizing)
        ctx.eeid_sync()
        t0 = time.perf_counter()
        out = ctx.eeid_components(A, rows=[i], cols=[j])
        ctx.eeid_sync()
        times[cl] = time.perf_counter() - t0
        v = float(out.cpu().numpy()[0, 0])
        assert abs(v - p.Q[j, i] ** 2) <= TOL_VSQ, (cl, v, p.Q[j, i] ** 2)
    print(f"n=4002 one component: group plan {times[2]:.3f} s, cluster plan "
          f"{times[True]:.3f} s, one CTA per matrix {times[False]:.3f} s")
    assert times[True] < 0.5 * times[False]
    assert times[2] < 0.7 * times[True]


def test_cluster_rounds_bitwise_and_closed_form(torch_cuda, ctx):
    """A uniform group with more matrices than half the SMs and a short last round
    (n = 2001 with 199 columns: 200 reductions of m = 2000/2001, one CTA per SM) runs as
    whole rounds of two-CTA clusters plus a last launch of clusters: bitwise equal to the
    one-CTA plan, and within the bar of Q o Q."""
    torch = torch_cuda
    n = 2001
    p = inputs.planted(n, 2001, -1.0, 1.0, 1e-4)
    A = torch.from_numpy(p.A).cuda()
    cols = np.sort(np.random.default_rng(7).choice(n, 199, replace=False))
    rows = np.unique(np.r_[0, 1000, n - 1, np.random.default_rng(8).choice(n, 20, replace=False)])
    got_c, lam_c = run(torch, ctx, A, rows, cols, True)
    got_p, lam_p = run(torch, ctx, A, rows, cols, False)
    assert np.array_equal(got_c, got_p) and np.array_equal(lam_c, lam_p)
    assert np.max(np.abs(got_c - (p.Q * p.Q).T[np.ix_(rows, cols)])) <= TOL_VSQ
