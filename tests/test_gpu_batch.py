"""Batched solves (per-item launches and the persistent kernel) and the
serving loop vs single-problem solves (GPU)."""
import os
import time

import numpy as np
import pytest

import oracle as O
from gpu_helpers import agreement
from paper_2508_09738_gb300 import binding as B
from paper_2508_09738_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_09738_gb300 import build
    build.build()


def mixed_problems(P=10, seed=0, n_scale=0.05):
    """Blob problems of uneven size and K (some ragged, some tiny) plus an image."""
    gs = W.batched_blobs(P=P - 1, n_min=300, n_max=200_000, K_min=3, K_max=10, seed=seed,
                         n_scale=n_scale)
    gs.append(W.voronoi_image(side=61, K=5, seed=seed + 99, label_frac=0.02))
    return gs


def solve_alone(g, weights, **opts):
    with B.Segmenter(g, weight_dtype=weights, **opts) as s:
        st = s.solve()
        return s.U(), s.labels(), st


@pytest.mark.parametrize("weights", ["f32", "bf16"])
@pytest.mark.parametrize("schedule,bps,lanes", [("static", 1, 0), ("dynamic", 2, 4),
                                                ("dynamic", 2, 2), ("static", 0, -1),
                                                ("items", 1, 0), ("items", 0, -1)])
def test_batch_bitwise_equals_single(weights, schedule, bps, lanes):
    """Batched solves equal single solves bit for bit when both use the same
    lanes per row (the batch's tuned or fixed count, reported by info())."""
    gs = mixed_problems(P=10, seed=3)
    iters = [30 + 7 * p for p in range(len(gs))]          # different caps per problem
    opts = [B.fw_seg_default_opts(max_iters=it, weight_dtype=weights) for it in iters]
    with B.Batch(gs, opts, weight_dtype=weights, schedule=schedule, blocks_per_sm=bps,
                 lanes_per_row=lanes) as b:
        stats = b.solve()
        info = b.info()
        assert info.graph_captured == 1 and info.graph_error == 0
        if lanes >= 0:
            assert info.lanes_per_row == lanes
        for p, g in enumerate(gs):
            U, lab, st = solve_alone(g, weights, max_iters=iters[p],
                                     lanes_per_row=info.lanes_per_row)
            assert np.array_equal(b.U(p), U), p
            assert np.array_equal(b.labels(p), lab), p
            assert stats[p].iters == st.iters and stats[p].status == st.status
            assert stats[p].gap == st.gap and stats[p].alpha == st.alpha


def test_batch_relaunch_and_reset_reproduce():
    gs = mixed_problems(P=6, seed=5)
    opts = B.fw_seg_default_opts(max_iters=40)
    with B.Batch(gs, opts, iters_per_launch=7, lanes_per_row=0) as b:
        b.solve()
        U1 = [b.U(p) for p in range(len(gs))]
        b.reset()
        b.solve()
        U2 = [b.U(p) for p in range(len(gs))]
    with B.Batch(gs, opts, iters_per_launch=0, lanes_per_row=0) as b:   # one launch
        b.solve()
        U3 = [b.U(p) for p in range(len(gs))]
    for a, c, d in zip(U1, U2, U3):
        assert np.array_equal(a, c) and np.array_equal(a, d)


def test_batch_f64_matches_oracle():
    gs = mixed_problems(P=5, seed=7, n_scale=0.01)
    with B.Batch(gs, B.fw_seg_default_opts(max_iters=25), weight_dtype="f64") as b:
        b.solve()
        for p, g in enumerate(gs):
            P = O.make_problem(g, 50.0, 1000.0, "f64")
            Uo, _ = O.gfw_solve(P, max_iters=25)
            assert np.max(np.abs(b.U(p) - Uo)) < 1e-9


def test_batch_independent_stop_rules():
    gs = mixed_problems(P=6, seed=9)
    opts = [B.fw_seg_default_opts(max_iters=400, gap_tol=1e-2, tol_mode="rel"),
            B.fw_seg_default_opts(max_iters=3),
            B.fw_seg_default_opts(max_iters=0),
            B.fw_seg_default_opts(eps=0.1, omega0=1e5, max_iters=50),      # one shot
            B.fw_seg_default_opts(max_iters=60, step_rule="armijo"),
            B.fw_seg_default_opts(max_iters=60, oracle="full")]
    with B.Batch(gs, opts, lanes_per_row=0) as b:
        stats = b.solve()
    for p, (g, o) in enumerate(zip(gs, opts)):
        with B.Segmenter(g, eps=o.eps, omega0=o.omega0, max_iters=o.max_iters,
                         gap_tol=o.gap_tol, tol_mode=o.tol_mode, step_rule=o.step_rule,
                         oracle=o.oracle) as s:
            st = s.solve()
        assert (stats[p].iters, stats[p].status) == (st.iters, st.status), p
    assert stats[1].iters == 3 and stats[2].iters == 0 and stats[3].iters == 1


def _tuned(i):
    return (i.blocks_per_sm, i.schedule, i.lanes_per_row, i.kmax, i.iters_per_launch)


def test_batch_autotune_cache(tmp_path):
    """The tuner searches blocks per SM x schedule, lanes per row, the
    kernel's class bound and iterations per launch; a second batch of the
    same sizes takes the cached choice and gives the same bits."""
    gs = mixed_problems(P=4, seed=11)
    cache = str(tmp_path / "tune.txt")
    opts = B.fw_seg_default_opts(max_iters=10)
    with B.Batch(gs, opts, tune_cache=cache) as b:
        i1 = b.info()
        b.solve()
        U1 = b.U(0)
    with B.Batch(gs, opts, tune_cache=cache) as b:
        i2 = b.info()
        b.solve()
        U2 = b.U(0)
        assert b.info().graph_captured == 1
    assert i1.tuned == 1 and i2.tuned == 2
    assert _tuned(i1) == _tuned(i2)
    assert i1.lanes_per_row in (0, 1, 2, 4, 8) and i1.iters_per_launch in (0, 64, 16)
    bounds = [4, 8, 10, 12, 16, 32]
    km = min(x for x in bounds if x >= max(g.K for g in gs))
    assert i1.kmax in (km, bounds[bounds.index(km) + 1]) and i1.tune_ms > 0
    assert np.array_equal(U1, U2)
    assert os.path.getsize(cache) > 0


@pytest.mark.parametrize("schedule", ["dynamic", "items"])
@pytest.mark.parametrize("kmax_K", [3, 10])
def test_batch_graph_capture_equals_direct_launches(kmax_K, schedule):
    """The batch's launches run from a captured CUDA graph by default
    (FW_GRAPH_REQUIRED), and give the same bits as direct launches."""
    gs = W.batched_blobs(P=5, n_min=300, n_max=20_000, K_min=kmax_K, K_max=kmax_K, seed=17,
                         n_scale=0.2)
    opts = B.fw_seg_default_opts(max_iters=45)
    kw = dict(blocks_per_sm=2, schedule=schedule, lanes_per_row=0, iters_per_launch=16)
    with B.Batch(gs, opts, use_graph="required", **kw) as a, \
            B.Batch(gs, opts, use_graph="off", **kw) as d:
        sa, sd = a.solve(), d.solve()
        ia, idd = a.info(), d.info()
        assert ia.graph_captured == 1 and ia.graph_error == 0
        assert idd.graph_captured == 0
        for p in range(len(gs)):
            assert np.array_equal(a.U(p), d.U(p)), p
            assert (sa[p].iters, sa[p].gap) == (sd[p].iters, sd[p].gap)


def test_batch_bf16_agrees_with_oracle():
    """Batched BF16 weights against the FP64 oracle on the same rounded
    weights, per problem, at reduced sizes of the batched configuration:
    label agreement and the final objective."""
    gs = W.batched_blobs(P=6, n_min=1000, n_max=200_000, K_min=3, K_max=10, label_frac=0.02,
                         seed=W.SEED0 + 3, n_scale=0.03)
    with B.Batch(gs, B.fw_seg_default_opts(max_iters=200), weight_dtype="bf16") as b:
        b.solve()
        for p, g in enumerate(gs):
            P = O.make_problem(g, 50.0, 1000.0, "bf16")
            Uo, info = O.gfw_solve(P, max_iters=200)
            assert agreement(b.labels(p), O.labels_from_U(Uo)) >= 0.999, p
            E = O.energy(b.U(p), P)
            Eo = O.energy(Uo, P)
            assert abs(E - Eo) <= 1e-4 * abs(Eo), (p, E, Eo)


def test_batch_barrier_timeout_is_reported_and_recoverable():
    """A barrier that waits for a block that never arrives runs out of its
    budget: the launch ends with FW_ERR_TIMEOUT and the context stays usable."""
    gs = mixed_problems(P=3, seed=13)
    t0 = time.time()
    with B.Batch(gs, B.fw_seg_default_opts(max_iters=5), test_barrier_extra=1,
                 spin_budget_ms=20, blocks_per_sm=1, schedule="static", lanes_per_row=0,
                 iters_per_launch=0) as b:
        with pytest.raises(B.FwError) as e:
            b.solve()
    assert e.value.status == B.FW_ERR_TIMEOUT
    assert time.time() - t0 < 30
    U, _, _ = solve_alone(gs[0], "f32", max_iters=5)   # the GPU still works
    assert np.all(np.isfinite(U))


# ------------------------------------------------------------------ serving --

def requests(seed=21):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(14):
        if i % 3 == 2:
            side = int(rng.choice([40, 64, 90]))
            g = W.voronoi_image(side=side, K=int(rng.integers(3, 9)), seed=seed + i,
                                label_frac=0.02)
            o = dict(eps=0.1, omega0=1e5, max_iters=20) if i % 2 else \
                dict(max_iters=300, gap_tol=1e-4, tol_mode="rel")
        else:
            g = W.blobs_knn(n=int(rng.integers(300, 4000)), K=int(rng.integers(3, 9)),
                            seed=seed + i, label_frac=0.02)
            o = dict(max_iters=300, gap_tol=1e-4, tol_mode="rel")
        out.append((g, o))
    return out


@pytest.mark.parametrize("schedule", ["items", "dynamic"])
def test_server_results_equal_alone(schedule):
    """Shared epochs run per-item launches (the default) or the persistent
    kernel; either way each request equals its own solve bit for bit."""
    reqs = requests()
    alone = [solve_alone(g, "f32", **o) for g, o in reqs]
    # a small pool forces queueing and reuse of freed memory
    need = max(B.fw_seg_footprint(g.n, g.nnz, 8, "f32") for g, _ in reqs)
    with B.Server(hbm_budget_bytes=3 * need, max_slots=4, max_K=8, iters_per_epoch=8,
                  schedule=schedule) as srv:
        tickets = []
        for g, o in reqs:
            tickets.append(srv.submit(g, **o))
            time.sleep(0.002)
        for (g, o), t, (U, lab, st) in zip(reqs, tickets, alone):
            rc, lab_s, st_s = srv.wait(t, g.n, timeout_ms=60_000)
            assert rc == st.status, (rc, st.status)
            assert np.array_equal(lab_s, lab)
            assert st_s.iters == st.iters and st_s.gap == st.gap
        info = srv.info()
    assert info.completed == len(reqs) and info.failed == 0 and info.admitted == len(reqs)
    assert info.epochs > 0 and info.pool_used == 0


def test_server_rejects_and_reports_errors():
    g = W.blobs_knn(n=2000, K=5, seed=1)
    small = B.fw_seg_footprint(300, 300 * 12, 8, "f32")
    with B.Server(hbm_budget_bytes=small, max_slots=2, max_K=6) as srv:
        with pytest.raises(B.FwError) as e:
            srv.submit(g)                                     # can never fit
        assert e.value.status == B.FW_ERR_NO_MEMORY
        big_k = W.blobs_knn(n=200, K=7, seed=2)
        with pytest.raises(B.FwError) as e:
            srv.submit(big_k)                                 # K above max_K
        assert e.value.status == B.FW_ERR_UNSUPPORTED
        bad = W.blobs_knn(n=200, K=3, seed=3)
        bad.w = bad.w.copy()
        bad.w[0] *= 2.0                                       # asymmetric
        t = srv.submit(bad)
        rc, _, _ = srv.wait(t, bad.n, timeout_ms=30_000)
        assert rc == B.FW_ERR_GRAPH
        ok = W.blobs_knn(n=200, K=3, seed=4)
        t = srv.submit(ok, max_iters=20)
        rc, lab, st = srv.wait(t, ok.n, timeout_ms=30_000)
        assert rc == B.FW_NOT_CONVERGED and st.iters == 20
        info = srv.info()
        assert info.rejected == 2 and info.failed == 1


def test_server_lone_requests_and_wait_any():
    """Requests submitted one at a time run alone on the server (the
    single-problem kernels); a burst then shares batched epochs.
    wait_any reports every finished ticket once, and every result equals
    the request solved alone, bit for bit."""
    reqs = requests(seed=33)[:8]
    alone = [solve_alone(g, "f32", **o) for g, o in reqs]
    with B.Server(hbm_budget_bytes=1 << 30, max_slots=8, max_K=8, iters_per_epoch=8) as srv:
        for (g, o), (U, lab, st) in zip(reqs[:4], alone[:4]):      # one at a time
            t = srv.submit(g, **o)
            rc, tk = srv.wait_any(60_000)
            assert rc == B.FW_OK and tk == t
            rc, lab_s, st_s = srv.poll(t, g.n)
            assert rc == st.status and np.array_equal(lab_s, lab)
            assert st_s.iters == st.iters and st_s.gap == st.gap
        tickets = {srv.submit(g, **o): k for k, (g, o) in enumerate(reqs[4:], start=4)}
        seen = set()
        while len(seen) < len(tickets):
            rc, tk = srv.wait_any(60_000)
            assert rc == B.FW_OK and tk in tickets and tk not in seen
            seen.add(tk)
            k = tickets[tk]
            g, _ = reqs[k]
            U, lab, st = alone[k]
            rc, lab_s, st_s = srv.poll(tk, g.n)
            assert rc == st.status and np.array_equal(lab_s, lab), k
            assert st_s.iters == st.iters and st_s.gap == st.gap, k
        assert srv.wait_any(10) == (B.FW_PENDING, None)
        info = srv.info()
    assert info.completed == len(reqs) and info.failed == 0


def test_server_lone_request_takes_class_table_form():
    """A served request large enough for the class-table pass B (scattered
    columns, more tiles than SMs) runs alone on the single-problem kernels
    with that form when it is the only resident, and equals its own solve
    bit for bit; so does it behind a small request, with which it shares
    per-item epochs (the direct pass-B code) before it finishes alone."""
    g = W.sbm(n=50_000, K=5, deg_in=16.0, deg_out=3.0, label_frac=0.01, seed=81)
    small = W.blobs_knn(n=700, K=3, seed=82)
    o = dict(max_iters=150, gap_tol=1e-4, tol_mode="rel")
    with B.Segmenter(g, weight_dtype="f32", **o) as s:
        assert s.forms().class_table == 1
    U, lab, st = solve_alone(g, "f32", **o)
    _, lab_small, st_small = solve_alone(small, "f32", **o)
    with B.Server(hbm_budget_bytes=1 << 30, max_slots=4, max_K=8, iters_per_epoch=8) as srv:
        for first in (None, small):
            tk = [srv.submit(first, **o)] if first is not None else []
            t = srv.submit(g, **o)
            rc, lab_s, st_s = srv.wait(t, g.n, timeout_ms=60_000)
            assert rc == st.status and np.array_equal(lab_s, lab)
            assert (st_s.iters, st_s.gap, st_s.objective) == (st.iters, st.gap, st.objective)
            for t2 in tk:
                rc2, lab2, st2 = srv.wait(t2, small.n, timeout_ms=60_000)
                assert rc2 == st_small.status and np.array_equal(lab2, lab_small)
        info = srv.info()
    assert info.failed == 0


@pytest.mark.parametrize("order", ["large_first", "small_first"])
def test_server_large_oldest_runs_alone_equal_results(order):
    """The oldest resident request runs alone when it has at least 2^17 rows;
    smaller residents share batched epochs without the large ones, which wait
    until they are the oldest (small_first: two small requests share epochs
    while two large ones wait).  Every result equals the request solved alone,
    bit for bit."""
    reqs = [(W.voronoi_image(side=400, K=4, seed=71, label_frac=0.005),
             dict(max_iters=120, omega0=1e5)),
            (W.blobs_knn(n=900, K=3, seed=72), dict(max_iters=90)),
            (W.voronoi_image(side=384, K=5, seed=73, label_frac=0.005),
             dict(max_iters=100, gap_tol=1e-3, tol_mode="rel", omega0=1e5)),
            (W.blobs_knn(n=1500, K=6, seed=74), dict(max_iters=150)),
            (W.voronoi_image(side=50, K=3, seed=75, label_frac=0.02), dict(max_iters=70))]
    assert reqs[0][0].n >= 1 << 17 and reqs[2][0].n >= 1 << 17
    if order == "small_first":
        reqs = [reqs[1], reqs[3], reqs[0], reqs[2], reqs[4]]
    alone = [solve_alone(g, "f32", **o) for g, o in reqs]
    with B.Server(hbm_budget_bytes=2 << 30, max_slots=8, max_K=8, iters_per_epoch=8) as srv:
        tickets = [srv.submit(g, **o) for g, o in reqs]
        for (g, o), t, (U, lab, st) in zip(reqs, tickets, alone):
            rc, lab_s, st_s = srv.wait(t, g.n, timeout_ms=120_000)
            assert rc == st.status and np.array_equal(lab_s, lab)
            assert st_s.iters == st.iters and st_s.gap == st.gap and st_s.objective == st.objective
        info = srv.info()
    assert info.completed == len(reqs) and info.failed == 0


@pytest.mark.parametrize("weights", ["f32", "bf16", "f64"])
def test_two_lane_pass_b_bitwise_equals_persistent(weights):
    """Two lanes per CSR row: the single-problem pass B (compile-time lane
    count, exact-class and 40-register forms) and the persistent kernel
    (runtime lane count) add each row's entries and lanes in the same order,
    so the iterates agree bit for bit, for exact and guarded class counts
    and every weight type."""
    gs = [W.sbm(n=307 * K, K=K, deg_in=20.0, deg_out=2.0, label_frac=0.02, seed=90 + K)
          for K in (3, 4, 7, 10, 12, 13)]
    iters = 25
    opts = B.fw_seg_default_opts(max_iters=iters, weight_dtype=weights, lanes_per_row=2)
    with B.Batch(gs, opts, weight_dtype=weights, lanes_per_row=2, blocks_per_sm=2,
                 schedule="static", iters_per_launch=0) as b:
        stats = b.solve()
        for p, g in enumerate(gs):
            U, lab, st = solve_alone(g, weights, max_iters=iters, lanes_per_row=2)
            assert np.array_equal(b.U(p), U), (p, g.K)
            assert stats[p].gap == st.gap and stats[p].objective == st.objective, (p, g.K)


@pytest.mark.parametrize("schedule", ["dynamic", "items"])
def test_batch_staggered_stops_over_several_launches(schedule):
    """Problems that stop at different iterations, in launches of 7
    iterations: the live set (and so the work list) shrinks between launches,
    and every problem still equals its single solve bit for bit."""
    gs = mixed_problems(P=7, seed=23)
    opts = [B.fw_seg_default_opts(max_iters=m, gap_tol=t, tol_mode="rel")
            for m, t in ((60, 0.0), (9, 0.0), (200, 5e-2), (33, 0.0), (0, 0.0), (50, 0.0),
                         (200, 2e-1))]
    with B.Batch(gs, opts, schedule=schedule, blocks_per_sm=2, lanes_per_row=0,
                 iters_per_launch=7) as b:
        # A problem that stops inside pass A must not leave any block waiting
        # on its bulk copies (each such wait is bounded by 2 s).
        for _ in range(3):
            b.reset()
            t0 = time.time()
            stats = b.solve()
            assert time.time() - t0 < 1.5
        assert b.info().schedule == B.SCHED[schedule]
        for p, (g, o) in enumerate(zip(gs, opts)):
            U, lab, st = solve_alone(g, "f32", max_iters=o.max_iters, gap_tol=o.gap_tol,
                                     tol_mode=o.tol_mode)
            assert np.array_equal(b.U(p), U), p
            assert (stats[p].iters, stats[p].status, stats[p].gap) == (st.iters, st.status, st.gap)
