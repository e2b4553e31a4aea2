"""The serving loop (eeid_server_*): continuous batching, overlap of batches on the
device, admission by device budget, cancellation and bounded waits.  Every
failure here is made on the host (a cancelled request, a wait that runs out, a
budget refusal); no GPU fault is involved."""
import threading
import time

import numpy as np
import pytest

from paper_2002_04989_gb300 import eeid, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return torch


def solo(torch, A, cols=None):
    ctx = eeid.Context(0)
    try:
        lam = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        out = ctx.eeid_components(torch.from_numpy(A).cuda(), cols=cols, lam=lam)
        ctx.eeid_sync()
        return out.cpu().numpy(), lam.cpu().numpy()
    finally:
        ctx.close()


def test_results_same_alone_and_in_the_mix(torch_cuda):
    """Requests submitted from two threads at once are merged into shared batches;
    each result is bitwise the result of computing that matrix alone."""
    reqs = []
    for rid in range(14):
        g = np.random.default_rng(rid)
        n = int(g.integers(16, 260))
        A = inputs.goe(n, 700 + rid) if rid % 2 else inputs.planted(n, 800 + rid, gap=1e-3).A
        cols = None if rid % 3 else np.sort(g.choice(n, min(n, 1 + rid), replace=False))
        reqs.append((A, cols))
    tickets = [None] * len(reqs)
    with eeid.Server(0, max_batch=8, max_inflight=2) as srv:
        def sub(lo, hi):
            for k in range(lo, hi):
                tickets[k] = srv.eeid_server_submit(reqs[k][0], cols=reqs[k][1])
        th = [threading.Thread(target=sub, args=(0, 7)), threading.Thread(target=sub, args=(7, 14))]
        [t.start() for t in th]
        [t.join() for t in th]
        results = [srv.eeid_server_wait(t) for t in tickets]
        info = srv.eeid_server_info()
    assert info["batches_launched"] < len(reqs)          # requests were merged
    assert max(r[2]["batch_requests"] for r in results) > 1
    for (A, cols), (out, lam, st) in zip(reqs, results):
        o_ref, l_ref = solo(torch_cuda, A, cols)
        assert np.array_equal(out, o_ref) and np.array_equal(lam, l_ref)


def test_served_results_against_oracle_and_closed_form(torch_cuda, oracle_mod):
    """Served results against references that do not come from the GPU: planted
    requests (n from 40 to 1300, so the 16-warp reductions and round-sized launches
    of n > 1024 are covered) against the closed form Q o Q, GOE requests against the
    long-double oracle.  Requests go in together, so they share batches and overlap."""
    planted = [inputs.planted(n, 900 + n, -1.0, 1.0, 1e-4) for n in (40, 200, 520, 1100, 1300, 1200)]
    goes = [inputs.goe(n, 950 + n) for n in (24, 61, 90)]
    # the n = 1200 request with 199 columns has 200 reductions: whole rounds and a short
    # remainder that runs as one launch of clusters
    col_sets = [None, np.array([0, 7, 39]), None, np.array([3, 500, 1099]), np.arange(0, 1300, 97),
                np.sort(np.random.default_rng(12).choice(1200, 199, replace=False))]
    with eeid.Server(0, max_batch=8, max_inflight=2) as srv:
        tp = [srv.eeid_server_submit(p.A, cols=c) for p, c in zip(planted, col_sets)]
        tg = [srv.eeid_server_submit(A) for A in goes]
        res_p = [srv.eeid_server_wait(t) for t in tp]
        res_g = [srv.eeid_server_wait(t) for t in tg]
    for p, cols, (out, lam, st) in zip(planted, col_sets, res_p):
        n = p.A.shape[0]
        ref = (p.Q * p.Q).T if cols is None else (p.Q * p.Q).T[:, cols]
        err = float(np.max(np.abs(out - ref)))
        print(f"served planted n={n}: max|d vsq| = {err:.2e}")
        assert err <= 1e-10, (n, err)
        assert np.max(np.abs(lam - p.lam)) <= 1e-12
    for A, (out, lam, st) in zip(goes, res_g):
        ref, lam_ref, _ = oracle_mod.components(A, method=0, want_eigs=True)
        bar = 1e-10 if inputs.min_relative_gap(lam_ref) >= 1e-4 else 1e-6
        assert np.max(np.abs(out - ref)) <= bar, A.shape[0]
        assert np.max(np.abs(lam - lam_ref)) <= 1e-12 * max(abs(lam_ref[0]), abs(lam_ref[-1]))


def test_arrivals_overlap_a_running_batch(torch_cuda):
    """Small requests that arrive while a large batch runs start on the second slot
    and finish before it (continuous batching, not a FIFO queue)."""
    big = inputs.planted(1400, 5, gap=1e-4).A
    smalls = [inputs.goe(40 + 10 * k, 60 + k) for k in range(4)]
    with eeid.Server(0, max_batch=16, max_inflight=2) as srv:
        tb = srv.eeid_server_submit(big)
        time.sleep(0.05)
        ts = [srv.eeid_server_submit(A) for A in smalls]
        small_res = [srv.eeid_server_wait(t) for t in ts]
        t_small_done = time.perf_counter()
        big_res = srv.eeid_server_wait(tb)
        t_big_done = time.perf_counter()
        info = srv.eeid_server_info()
    assert info["max_overlapping_batches"] == 2
    assert t_small_done < t_big_done
    assert all(r[2]["batch_id"] != big_res[2]["batch_id"] for r in small_res)
    for A, (out, lam, st) in zip(smalls, small_res):
        o_ref, _ = solo(torch_cuda, A)
        assert np.array_equal(out, o_ref)


def test_cost_bands_and_round_launches(torch_cuda):
    """A large request and small ones queued at the same moment go to different batches
    (cost bands), and the small ones finish first although the large batch was
    launched first: its reductions run one round at a time, so the second slot's
    kernels get SMs in between."""
    big = inputs.planted(1200, 9, gap=1e-4).A
    smalls = [inputs.goe(30 + 7 * k, 90 + k) for k in range(3)]
    with eeid.Server(0, max_batch=16, max_inflight=2) as srv:
        tb = srv.eeid_server_submit(big)
        ts = [srv.eeid_server_submit(A) for A in smalls]
        small_res = [srv.eeid_server_wait(t) for t in ts]
        t_small_done = time.perf_counter()
        big_res = srv.eeid_server_wait(tb)
        t_big_done = time.perf_counter()
    assert all(r[2]["batch_id"] != big_res[2]["batch_id"] for r in small_res)
    assert t_small_done < t_big_done
    assert max(r[2]["total_ms"] for r in small_res) < 0.5 * big_res[2]["total_ms"]
    for A, (out, lam, st) in zip(smalls, small_res):
        o_ref, _ = solo(torch_cuda, A)
        assert np.array_equal(out, o_ref)


def test_cancel_and_bounded_wait(torch_cuda):
    big = inputs.planted(1200, 6, gap=1e-4).A
    small = inputs.goe(30, 3)
    with eeid.Server(0, max_batch=1, max_inflight=1) as srv:
        tb = srv.eeid_server_submit(big)
        time.sleep(0.05)
        ts = srv.eeid_server_submit(small)
        assert srv.eeid_server_cancel(ts) == 0          # still waiting for admission
        with pytest.raises(eeid.EeidError) as ei:
            srv.eeid_server_wait(ts)
        assert ei.value.status == eeid.EEID_ERR_CANCELLED
        with pytest.raises(eeid.EeidError) as ei:
            srv.eeid_server_wait(tb, timeout_ms=0)       # bounded wait runs out
        assert ei.value.status == eeid.EEID_ERR_TIMEOUT
        out, lam, st = srv.eeid_server_wait(tb)          # the request is still there
        assert out.shape == (1200, 1200) and np.isfinite(out).all()
        with pytest.raises(eeid.EeidError) as ei:
            srv.eeid_server_wait(tb)
        assert ei.value.status == eeid.EEID_ERR_NOT_FOUND


def test_budget_refusal_and_busy(torch_cuda):
    with eeid.Server(0, hbm_budget_bytes=64 << 20, max_pending=1, max_inflight=1,
                     max_batch=1) as srv:
        with pytest.raises(eeid.EeidError) as ei:       # 2 x 33.5 MB > 32 MB request budget
            srv.eeid_server_submit(inputs.goe(2048, 1))
        assert ei.value.status == eeid.EEID_ERR_NOMEM
        # a 32 MB workspace per batch still runs n = 400 (fewer persistent CTAs)
        t1 = srv.eeid_server_submit(inputs.goe(400, 2))
        t2 = srv.eeid_server_submit(inputs.goe(400, 3))  # may wait for queue room
        with pytest.raises(eeid.EeidError) as ei:
            for _ in range(50):                          # queue of one: a non-blocking
                srv.eeid_server_submit(inputs.goe(400, 4), nonblocking=True)  # submit fails
        assert ei.value.status == eeid.EEID_ERR_BUSY
        for t in (t1, t2):
            srv.eeid_server_wait(t)
