"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars (stated here, used everywhere below):
  * |v_ij|^2: max abs error <= 1e-10, for spectra whose minimum relative gap is
    >= 1e-4 (outside that, the error is reported and only a loose 1e-6 bar applies);
  * eigenvalues of A and of the minors: max abs error <= 1e-12 * ||A||_2.
The oracle runs in long double on the host; planted spectra are checked against
their closed form Q o Q.
"""
import numpy as np
import pytest

from invariants import grid_errors, spectrum_errors
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


def dev(torch, A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def run_components(torch, ctx, A, rows=None, cols=None):
    dA = dev(torch, A)
    n = A.shape[0]
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    out = ctx.eeid_components(dA, rows=rows, cols=cols, lam=lam)
    st = ctx.eeid_sync()
    return out.cpu().numpy(), lam.cpu().numpy(), st


def vsq_bar(lam_ref):
    return TOL_VSQ if inputs.min_relative_gap(lam_ref) >= 1e-4 else 1e-6


# ------------------------------------------------------------------ small, full oracle

SMALL = [1, 2, 3, 5, 8, 16, 31, 32, 33, 47, 63, 64, 65]


@pytest.mark.parametrize("n", SMALL)
def test_goe_small_full_grid(torch_cuda, ctx, oracle_mod, n):
    A = inputs.goe(n, 1000 + n)
    out, lam, st = run_components(torch_cuda, ctx, A)
    ref, lam_ref, mu_ref = oracle_mod.components(A, method=0, want_eigs=True)
    norm = max(abs(lam_ref[0]), abs(lam_ref[-1]))
    assert np.max(np.abs(lam - lam_ref)) <= TOL_LAM_REL * norm
    assert np.max(np.abs(out - ref)) <= vsq_bar(lam_ref), np.max(np.abs(out - ref))
    if n >= 2:
        mu = ctx.eeid_minor_eigvals(dev(torch_cuda, A)).cpu().numpy()
        assert np.max(np.abs(mu - mu_ref)) <= TOL_LAM_REL * norm


def test_goe64_workload(torch_cuda, ctx, oracle_mod):
    """One GOE matrix n = 64 from seed 0: all 64 minors and the full grid."""
    A = inputs.goe64()
    out, lam, st = run_components(torch_cuda, ctx, A)
    ref, lam_ref, mu_ref = oracle_mod.components(A, method=0, want_eigs=True)
    vv = oracle_mod.components(A, method=2)
    norm = max(abs(lam_ref[0]), abs(lam_ref[-1]))
    assert inputs.min_relative_gap(lam_ref) >= 1e-4
    assert np.max(np.abs(lam - lam_ref)) <= TOL_LAM_REL * norm
    assert np.max(np.abs(out - ref)) <= TOL_VSQ
    assert np.max(np.abs(out - vv)) <= TOL_VSQ
    mu = ctx.eeid_minor_eigvals(dev(torch_cuda, A)).cpu().numpy()
    assert np.max(np.abs(mu - mu_ref)) <= TOL_LAM_REL * norm
    g = grid_errors(A, lam, out)
    assert g["col_sum"] < 1e-11 and g["row_sum"] < 1e-11 and g["diag"] < 1e-10
    s = spectrum_errors(A, lam, mu)
    assert s["interlace"] <= 1e-13 * norm and s["minor_trace"] < 1e-10


@pytest.mark.parametrize("kind,n", [("wishart", 40), ("toeplitz", 33), ("toeplitz", 64),
                                    ("planted", 60), ("wishart", 9)])
def test_families_full_grid(torch_cuda, ctx, oracle_mod, kind, n):
    if kind == "wishart":
        A = inputs.wishart(n, 77)
    elif kind == "toeplitz":
        A = inputs.toeplitz(n, 0.0, 1.0)
    else:
        A = inputs.planted(n, 78, gap=1e-3).A
    out, lam, st = run_components(torch_cuda, ctx, A)
    ref, lam_ref, _ = oracle_mod.components(A, method=0, want_eigs=True)
    norm = max(abs(lam_ref[0]), abs(lam_ref[-1]))
    assert np.max(np.abs(lam - lam_ref)) <= TOL_LAM_REL * norm
    assert np.max(np.abs(out - ref)) <= vsq_bar(lam_ref)


# ------------------------------------------------------------------ medium: sampled oracle

@pytest.mark.parametrize("n", [96, 127, 128, 129, 160, 161, 200, 255, 256, 300])
def test_planted_medium(torch_cuda, ctx, oracle_mod, n):
    """Sizes across the shared-memory / global-memory boundary and ragged tiles:
    full grid against Q o Q, sampled minors against the secular-equation roots."""
    p = inputs.planted(n, 2000 + n, -1.0, 1.0, 1e-3)
    cols = np.array([0, n // 3, n - 1])
    out, lam, st = run_components(torch_cuda, ctx, p.A)
    assert np.max(np.abs(lam - p.lam)) <= TOL_LAM_REL * 1.0 + 1e-15
    assert np.max(np.abs(out - (p.Q * p.Q).T)) <= TOL_VSQ
    mu = ctx.eeid_minor_eigvals(dev(torch_cuda, p.A), cols=cols).cpu().numpy()
    mu_ref = oracle_mod.secular_minor_eigvals(p.lam, p.Q, cols)
    assert np.max(np.abs(mu - mu_ref)) <= TOL_LAM_REL
    g = grid_errors(p.A, lam, out)
    assert g["col_sum"] < 1e-10 and g["row_sum"] < 1e-10


@pytest.mark.parametrize("n", [100, 161])
def test_goe_medium_sampled_columns(torch_cuda, ctx, oracle_mod, n):
    A = inputs.goe(n, 3000 + n)
    rows = np.array([0, 1, n // 2, n - 2, n - 1])
    cols = np.array([n - 1, 0, n // 2])
    out, lam, st = run_components(torch_cuda, ctx, A, rows=rows, cols=cols)
    ref, lam_ref, _ = oracle_mod.components(A, rows=rows, cols=cols, method=0, want_eigs=True)
    norm = max(abs(lam_ref[0]), abs(lam_ref[-1]))
    assert np.max(np.abs(lam - lam_ref)) <= TOL_LAM_REL * norm
    assert np.max(np.abs(out - ref)) <= vsq_bar(lam_ref)


# ------------------------------------------------------------------ full-size workloads

def test_planted1024_workload(torch_cuda, ctx, oracle_mod):
    """n = 1024 planted spectrum, the full 1024 x 1024 grid against Q o Q (the launch
    configuration the benchmark times), minors sampled against the secular roots."""
    p = inputs.planted1024()
    out, lam, st = run_components(torch_cuda, ctx, p.A)
    err_lam = np.max(np.abs(lam - p.lam))
    err = np.max(np.abs(out - (p.Q * p.Q).T))
    print(f"planted1024: max|dlam| = {err_lam:.3e}, max|d vsq| = {err:.3e}")
    assert err_lam <= TOL_LAM_REL
    assert err <= TOL_VSQ
    cols = np.array([0, 511, 1023])
    mu = ctx.eeid_minor_eigvals(dev(torch_cuda, p.A), cols=cols).cpu().numpy()
    mu_ref = oracle_mod.secular_minor_eigvals(p.lam, p.Q, cols)
    assert np.max(np.abs(mu - mu_ref)) <= TOL_LAM_REL
    g = grid_errors(p.A, lam, out)
    assert g["col_sum"] < 1e-10 and g["row_sum"] < 1e-10


# ------------------------------------------------------------------ edge cases

def test_n1_and_empty(torch_cuda, ctx):
    out, lam, st = run_components(torch_cuda, ctx, np.array([[2.5]]))
    assert out[0, 0] == 1.0 and lam[0] == 2.5
    A = dev(torch_cuda, inputs.goe(5, 1))
    o = torch_cuda.zeros((0, 5), dtype=torch_cuda.float64, device="cuda")
    ctx.eeid_components(A, rows=[], cols=None, out=o)
    assert ctx.eeid_sync() == 0


def test_subset_and_order(torch_cuda, ctx, oracle_mod):
    A = inputs.goe(37, 5)
    rows, cols = [36, 0, 17], [5, 2, 30, 1]
    out, lam, st = run_components(torch_cuda, ctx, A, rows=rows, cols=cols)
    ref = oracle_mod.components(A, rows=rows, cols=cols, method=0)
    assert np.max(np.abs(out - ref)) <= TOL_VSQ


def test_lda_padding(torch_cuda, ctx, oracle_mod):
    A = inputs.goe(40, 6)
    big = np.full((40, 48), np.nan)
    big[:, :40] = A
    dA = dev(torch_cuda, big)[:, :40]
    assert dA.stride(0) == 48
    out = ctx.eeid_components(dA).cpu().numpy()
    ctx.eeid_sync()
    ref = oracle_mod.components(A, method=0)
    assert np.max(np.abs(out - ref)) <= TOL_VSQ


def test_lower_triangle_only(torch_cuda, ctx):
    A = inputs.goe(30, 9)
    B = A.copy()
    B[np.triu_indices(30, 1)] = 1e300   # garbage above the diagonal is never read
    o1, _, _ = run_components(torch_cuda, ctx, A)
    o2, _, _ = run_components(torch_cuda, ctx, B)
    assert np.array_equal(o1, o2)


def test_argument_errors(torch_cuda, ctx):
    from paper_2002_04989_gb300 import eeid
    A = dev(torch_cuda, inputs.goe(6, 2))
    for rows, cols in (([0, 0], None), ([6], None), (None, [-1]), (None, [1, 1])):
        with pytest.raises(eeid.EeidError) as ei:
            ctx.eeid_components(A, rows=rows, cols=cols)
        assert ei.value.status == eeid.EEID_ERR_INVALID


def test_size_limit_refused(torch_cuda, ctx):
    """n above the kernels' limit (4096) is refused on the host, before anything is
    queued; n = 4096 itself is the planted4096 workload (test_workloads_gpu)."""
    from paper_2002_04989_gb300 import eeid
    A = torch_cuda.zeros((4097, 4097), dtype=torch_cuda.float64, device="cuda")
    with pytest.raises(eeid.EeidError) as ei:
        ctx.eeid_components(A, rows=[0], cols=[0])
    assert ei.value.status == eeid.EEID_ERR_INVALID
    del A


def test_degenerate_warns_and_nans(torch_cuda, ctx):
    from paper_2002_04989_gb300 import eeid
    A = np.diag([1.0, 2.0, 2.0, 3.0])
    dA = dev(torch_cuda, A)
    out = ctx.eeid_components(dA).cpu().numpy()
    st = ctx.eeid_sync()
    assert st == eeid.EEID_WARN_DEGENERATE
    assert np.isnan(out[1]).all() and np.isnan(out[2]).all()
    assert np.allclose(out[0], [1, 0, 0, 0], rtol=0, atol=1e-14)
    assert np.allclose(out[3], [0, 0, 0, 1], rtol=0, atol=1e-14)


def test_diagonal_exact(torch_cuda, ctx):
    d = np.array([0.5, -2.0, 3.0, 1.25, -0.75])
    out, lam, st = run_components(torch_cuda, ctx, np.diag(d))
    order = np.argsort(d)
    expect = np.zeros((5, 5))
    expect[np.arange(5), order] = 1.0
    assert np.max(np.abs(out - expect)) <= 1e-15
    assert np.max(np.abs(lam - np.sort(d))) <= TOL_LAM_REL * 3.0


def test_eigvals_entry_point(torch_cuda, ctx, oracle_mod):
    A = inputs.wishart(70, 4)
    lam = ctx.eeid_eigvals(dev(torch_cuda, A)).cpu().numpy()
    ref = oracle_mod.eigvals(A)
    assert np.max(np.abs(lam - ref)) <= TOL_LAM_REL * ref[-1]


def test_host_entry_point_matches_device(torch_cuda, ctx):
    A = inputs.goe(50, 12)
    o_dev, lam_dev, _ = run_components(torch_cuda, ctx, A)
    lam_h = np.empty(50)
    o_host = ctx.eeid_components_host(A, lam=lam_h)
    assert np.array_equal(o_host, o_dev) and np.array_equal(lam_h, lam_dev)


def test_repeatable_bitwise(torch_cuda, ctx):
    """Repeated calls give bitwise-identical grids (no races, fixed reduction order),
    at a size where persistent CTAs process several matrices each."""
    p = inputs.planted(520, 13, -1.0, 1.0, 1e-3)
    first, _, _ = run_components(torch_cuda, ctx, p.A)
    assert np.max(np.abs(first - (p.Q * p.Q).T)) <= TOL_VSQ
    for _ in range(3):
        again, _, _ = run_components(torch_cuda, ctx, p.A)
        assert np.array_equal(first, again)


def test_batched_matches_single_bitwise(torch_cuda, ctx):
    """Uneven sizes in one batched call give bitwise the results of single calls."""
    torch = torch_cuda
    items = [inputs.batch_item(m, 8, 256)[1] for m in range(12)]
    singles, probs = [], []
    for A in items:
        o, lam, _ = run_components(torch, ctx, A)
        singles.append((o, lam))
        n = A.shape[0]
        probs.append({"A": dev(torch, A), "out": torch.empty((n, n), dtype=torch.float64, device="cuda"),
                      "lam": torch.empty(n, dtype=torch.float64, device="cuda")})
    ctx.eeid_components_batched(probs)
    ctx.eeid_sync()
    for (o, lam), p in zip(singles, probs):
        assert np.array_equal(p["out"].cpu().numpy(), o)
        assert np.array_equal(p["lam"].cpu().numpy(), lam)


def test_batched_graph_replay_reads_live_inputs(torch_cuda, ctx, oracle_mod):
    """A repeated batch replays its captured CUDA graph (same kernel count, no new
    capture) and recomputes from the current contents of the input buffers."""
    torch = torch_cuda
    mats = [inputs.goe(n, 500 + n) for n in (9, 40, 77)]
    probs = [{"A": dev(torch, A), "out": torch.empty(A.shape, dtype=torch.float64, device="cuda")}
             for A in mats]
    ctx.eeid_components_batched(probs)
    ctx.eeid_sync()
    l1 = ctx.launch_count()
    first = [p["out"].cpu().numpy().copy() for p in probs]
    ctx.eeid_components_batched(probs)          # replay
    ctx.eeid_sync()
    l2 = ctx.launch_count()
    assert l2 - l1 > 0
    for p, f in zip(probs, first):
        assert np.array_equal(p["out"].cpu().numpy(), f)
    # new matrix contents in the same buffers -> the replay must see them
    newA = inputs.wishart(40, 9)
    probs[1]["A"].copy_(torch.from_numpy(newA))
    ctx.eeid_components_batched(probs)
    ctx.eeid_sync()
    assert ctx.launch_count() - l2 == l2 - l1    # same graph, same kernel count
    ref, lam_ref, _ = oracle_mod.components(newA, method=0, want_eigs=True)
    assert np.max(np.abs(probs[1]["out"].cpu().numpy() - ref)) <= vsq_bar(lam_ref)


def test_autotune_table_and_cache(torch_cuda, tmp_path, oracle_mod):
    """The autotuner installs per-size variants, writes its table, and a second
    context that loads the table computes bitwise the same results."""
    from paper_2002_04989_gb300 import eeid
    path = str(tmp_path / "tune.txt")
    A = inputs.goe(150, 31)
    c1 = eeid.Context(0)
    c2 = eeid.Context(0)
    try:
        c1.eeid_autotune(256, path)
        lines = open(path).read().splitlines()
        assert lines[0].startswith("eeid-tune v3") and len(lines) > 3
        assert int(lines[-1].split()[1]) >= 256
        c2.eeid_autotune(256, path)              # loads the cached table
        o1 = c1.eeid_components(dev(torch_cuda, A)).cpu().numpy()
        c1.eeid_sync()
        o2 = c2.eeid_components(dev(torch_cuda, A)).cpu().numpy()
        c2.eeid_sync()
        assert np.array_equal(o1, o2)
        ref, lam_ref, _ = oracle_mod.components(A, rows=[0, 75, 149], cols=[0, 75, 149],
                                                method=0, want_eigs=True)
        assert np.max(np.abs(o1[np.ix_([0, 75, 149], [0, 75, 149])] - ref)) <= vsq_bar(lam_ref)
    finally:
        c1.close()
        c2.close()


def test_phase_times_with_graphs(torch_cuda, ctx):
    """Per-phase timing works for captured batched calls (events become graph nodes)."""
    torch = torch_cuda
    A = inputs.goe(60, 77)
    probs = [{"A": dev(torch, A), "out": torch.empty((60, 60), dtype=torch.float64, device="cuda")}]
    ctx.eeid_set_timing(True)
    try:
        for _ in range(2):
            ctx.eeid_components_batched(probs)
            ph = ctx.eeid_phase_times()
            assert ph["tridiag"] > 0 and ph["bisect_minors"] > 0 and ph["identity"] > 0
    finally:
        ctx.eeid_set_timing(False)
    ctx.eeid_sync()


def test_every_output_written_poisoned_buffers(torch_cuda, ctx):
    """Outputs pre-filled with NaN come back fully written (no entry skipped), for the
    grid, the eigenvalues and the minor eigenvalues, across tile-boundary sizes."""
    torch = torch_cuda
    for n in (31, 33, 161, 300):
        A = dev(torch, inputs.goe(n, 90 + n))
        out = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        lam = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.eeid_components(A, out=out, lam=lam)
        mu = torch.full((3, n - 1), float("nan"), dtype=torch.float64, device="cuda")
        ctx.eeid_minor_eigvals(A, cols=[0, n // 2, n - 1], out=mu)
        ctx.eeid_sync()
        assert torch.isfinite(out).all() and torch.isfinite(lam).all() and torch.isfinite(mu).all()


def test_batched_without_graphs_matches_graphs(torch_cuda, oracle_mod):
    """eeid_set_graphs(0) plans and launches directly; results are bitwise those of
    the captured-graph path."""
    from paper_2002_04989_gb300 import eeid
    torch = torch_cuda
    mats = [inputs.batch_item(m, 8, 256)[1] for m in range(20, 28)]
    outs = {}
    for graphs in (True, False):
        c = eeid.Context(0)
        try:
            c.eeid_set_graphs(graphs)
            probs = [{"A": dev(torch, A), "out": torch.empty(A.shape, dtype=torch.float64, device="cuda")}
                     for A in mats]
            for _ in range(2):
                c.eeid_components_batched(probs)
            c.eeid_sync()
            outs[graphs] = [p["out"].cpu().numpy() for p in probs]
        finally:
            c.close()
    for a, b in zip(outs[True], outs[False]):
        assert np.array_equal(a, b)


def test_autotune_rejects_foreign_cache(torch_cuda, tmp_path):
    """A cache written for another device model is ignored (re-tuned and rewritten)."""
    from paper_2002_04989_gb300 import eeid
    path = tmp_path / "tune.txt"
    path.write_text("eeid-tune v3 sms=1 name=Some Other GPU\n1 4096 1 4\n")
    c = eeid.Context(0)
    try:
        c.eeid_autotune(64, str(path))
        head = path.read_text().splitlines()[0]
        assert "Some Other GPU" not in head and head.startswith("eeid-tune v3")
    finally:
        c.close()


def test_timing_misuse_and_tuning_errors(torch_cuda):
    from paper_2002_04989_gb300 import eeid
    c = eeid.Context(0)
    try:
        with pytest.raises(eeid.EeidError):
            c.eeid_phase_times()                       # timing never enabled
        with pytest.raises(eeid.EeidError):
            c.eeid_tune_tridiag(1, 400, 0, 4)         # shared-memory variant above its limit
        with pytest.raises(eeid.EeidError):
            c.eeid_tune_tridiag(1, 100, 1, 3)         # unsupported warp count
        with pytest.raises(eeid.EeidError):
            c.eeid_autotune(0)
    finally:
        c.close()


def _tail_expected(ntasks, grid):
    """Whether a call with `ntasks` near-equal reductions on `grid` persistent CTAs splits
    off its last partial round (the rule the planner applies)."""
    r = ntasks % grid
    return ntasks > grid and r > 0 and grid - r >= max(1, grid // 16)


def test_tail_overlap_bitwise_and_launches(torch_cuda, oracle_mod):
    """n = 520: 521 near-equal reductions at one CTA per SM take several rounds.  With
    the tail overlap the last round is a second launch on another stream, bisection
    overlaps it, and the tail minors are bisected in a second launch: two more kernel
    launches, bitwise the same grid and eigenvalues as with the overlap off, in direct
    calls and in captured batched calls."""
    from paper_2002_04989_gb300 import eeid
    torch = torch_cuda
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    p = inputs.planted(520, 21, -1.0, 1.0, 1e-3)
    dA = dev(torch, p.A)
    res = {}
    for overlap in (False, True):
        c = eeid.Context(0)
        try:
            c.eeid_set_overlap(overlap)
            lam = torch.empty(520, dtype=torch.float64, device="cuda")
            l0 = c.launch_count()
            out = c.eeid_components(dA, lam=lam)
            c.eeid_sync()
            nl = c.launch_count() - l0
            probs = [{"A": dA, "out": torch.empty((520, 520), dtype=torch.float64, device="cuda"),
                      "lam": torch.empty(520, dtype=torch.float64, device="cuda")}]
            c.eeid_set_timing(True)
            for _ in range(2):                      # capture, then replay
                c.eeid_components_batched(probs)
                ph = c.eeid_phase_times()
                assert all(ph[k] > 0 for k in ("tridiag", "bisect_A", "bisect_minors", "identity"))
            c.eeid_set_timing(False)
            c.eeid_sync()
            assert np.array_equal(probs[0]["out"].cpu().numpy(), out.cpu().numpy())
            assert np.array_equal(probs[0]["lam"].cpu().numpy(), lam.cpu().numpy())
            res[overlap] = (out.cpu().numpy(), lam.cpu().numpy(), nl)
        finally:
            c.close()
    assert np.array_equal(res[True][0], res[False][0]) and np.array_equal(res[True][1], res[False][1])
    assert res[False][2] == 5
    assert res[True][2] == (7 if _tail_expected(521, sms) else 5)
    assert np.max(np.abs(res[True][0] - (p.Q * p.Q).T)) <= TOL_VSQ


def test_tail_overlap_off_when_budget_shrinks_grid(torch_cuda):
    """A budget that leaves fewer working slots than SMs changes the round structure;
    the call then runs its reductions as one launch and still matches bitwise."""
    from paper_2002_04989_gb300 import eeid
    torch = torch_cuda
    A = inputs.goe(520, 22)
    dA = dev(torch, A)
    outs, launches = [], []
    for budget in (0, 200 << 20):
        c = eeid.Context(0, budget)
        try:
            l0 = c.launch_count()
            outs.append(c.eeid_components(dA).cpu().numpy())
            c.eeid_sync()
            launches.append(c.launch_count() - l0)
        finally:
            c.close()
    assert np.array_equal(outs[0], outs[1])
    assert launches[1] == 5


@pytest.mark.parametrize("n,path,warps", [(300, 1, (1, 2, 4, 8, 12, 16)), (700, 1, (4, 8, 12, 16)),
                                          (100, 0, (1, 2, 4, 8))])
def test_warp_count_does_not_change_results(torch_cuda, n, path, warps):
    """Every instantiation of one storage variant gives bitwise the same grid: partial
    sums are kept per tile and reduced in an order fixed by the matrix size alone, so
    the scheduler may run a matrix with any warp count.  The global path runs a batch of
    six copies (1806 reductions at n = 300), enough to fill the SMs with the 1- and
    2-warp builds, which the planner keeps only for such waves."""
    from paper_2002_04989_gb300 import eeid
    torch = torch_cuda
    dA = dev(torch, inputs.goe(n, 40 + n))
    lo = 161 if path == 1 else 1
    hi = 2048 if path == 1 else 160
    copies = 6 if path == 1 else 1
    ref = None
    for W in warps:
        c = eeid.Context(0)
        try:
            c.eeid_tune_tridiag(lo, hi, path, W)
            probs = [{"A": dA, "out": torch.empty((n, n), dtype=torch.float64, device="cuda")}
                     for _ in range(copies)]
            c.eeid_components_batched(probs)
            c.eeid_sync()
            outs = [p["out"].cpu().numpy() for p in probs]
        finally:
            c.close()
        if ref is None:
            ref = outs[0]
        for o in outs:
            assert np.array_equal(o, ref), W


def test_hybrid_rounds_bitwise_at_benchmark_size(torch_cuda):
    """n = 1024, all 1024 columns: 1025 near-equal reductions are planned as rounds of two
    8-warp CTAs per SM plus a 16-warp tail overlapped with the bisection.  The grid and
    eigenvalues are bitwise those of the plain plan (overlap off: one 16-warp launch)."""
    from paper_2002_04989_gb300 import eeid
    torch = torch_cuda
    p = inputs.planted1024()
    dA = dev(torch, p.A)
    res = []
    for overlap in (True, False):
        c = eeid.Context(0)
        try:
            c.eeid_set_overlap(overlap)
            lam = torch.empty(1024, dtype=torch.float64, device="cuda")
            out = c.eeid_components(dA, lam=lam)
            c.eeid_sync()
            res.append((out.cpu().numpy(), lam.cpu().numpy()))
        finally:
            c.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert np.max(np.abs(res[0][0] - (p.Q * p.Q).T)) <= TOL_VSQ


def test_status_is_per_stream(torch_cuda, ctx):
    """Deferred warnings belong to the stream of the call that raised them: a degenerate
    matrix on one stream and a small-gap matrix on another, each eeid_sync returns its
    own stream's warning (calls ordered by an event, as the shared workspace requires)."""
    from paper_2002_04989_gb300 import eeid
    torch = torch_cuda
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    deg = torch.from_numpy(np.diag([1.0, 1.0, 2.0, 3.0])).cuda()
    gap = torch.from_numpy(np.diag([1.0, 1.0 + 1e-7, 2.0, 3.0])).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        ctx.eeid_components(deg, stream=s1)
    s2.wait_stream(s1)
    with torch.cuda.stream(s2):
        ctx.eeid_components(gap, stream=s2)
    assert ctx.eeid_sync(s2) == eeid.EEID_WARN_SMALL_GAP
    assert ctx.eeid_sync(s1) == eeid.EEID_WARN_DEGENERATE
    assert ctx.eeid_sync(s1) == eeid.EEID_OK and ctx.eeid_sync(s2) == eeid.EEID_OK


def test_high_occupancy_build_bitwise(torch_cuda):
    """The high-occupancy build of the global-slot variant (path 2: 80 registers, more
    CTAs per SM) runs the same arithmetic as path 1: bitwise the same grid."""
    from paper_2002_04989_gb300 import eeid
    torch = torch_cuda
    dA = dev(torch, inputs.goe(230, 41))
    outs = []
    for path, W in ((1, 8), (2, 8), (2, 4)):
        c = eeid.Context(0)
        try:
            c.eeid_tune_tridiag(161, 2048, path, W)
            outs.append(c.eeid_components(dA).cpu().numpy())
            c.eeid_sync()
        finally:
            c.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
