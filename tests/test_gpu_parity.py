"""GPU path vs the FP64 oracle, through the C ABI (needs a GB300)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL, agreement, lockstep, rel
from paper_2508_09738_gb300 import binding as B
from paper_2508_09738_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_09738_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def blobs2k():
    return W.make_config_graph("blobs2k")


# ------------------------------------------------------------- lockstep --

@pytest.mark.parametrize("weights,tol", [("f64", 1e-9), ("f32", TOL), ("bf16", TOL)])
def test_lockstep_blobs2k(blobs2k, weights, tol):
    recs = lockstep(blobs2k, 60, weights=weights, tol=tol)
    assert len(recs) == 60


def test_lockstep_blobs2k_long_every10(blobs2k):
    """500 iterations, checks every 10: the L U recurrence does not drift past 1e-5."""
    recs = lockstep(blobs2k, 500, weights="f32", every=10, energy=True)
    assert len(recs) == 50


@pytest.mark.parametrize("L", [1, 2, 4, 8, 16, 32])
def test_lockstep_lanes_per_row(L):
    g = W.blobs_knn(n=1537, K=7, seed=5)       # ragged: 6 tiles of 256 + 1 row
    lockstep(g, 12, weights="f32", lanes_per_row=L)


@pytest.mark.parametrize("K", [2, 3, 4, 5, 8, 9, 12, 13, 16, 17, 32])
def test_lockstep_class_counts(K):
    g = W.blobs_knn(n=40 * K + 3, K=K, seed=100 + K, label_frac=0.1)
    lockstep(g, 8, weights="f32")
    lockstep(g, 4, weights="f64", tol=1e-9)


def test_lockstep_fp64_single_stage_multi_subtile():
    """FP64 with K > 16 keeps one staging buffer per block (two would not fit
    in shared memory), and n > 1216 * 256 gives every row tile several 256-row
    sub-tiles: each sub-tile's copy must be issued when the buffer is free."""
    g = W.sbm(n=320_000, K=20, deg_in=8.0, deg_out=1.0, label_frac=0.01, seed=7)
    recs = lockstep(g, 3, weights="f64", tol=1e-9, energy=False)
    assert len(recs) == 3


def test_lockstep_armijo(blobs2k):
    lockstep(blobs2k, 15, weights="f64", step="armijo", tol=1e-9)


def test_lockstep_full_lmo(blobs2k):
    lockstep(blobs2k, 15, weights="f64", oracle="full", tol=1e-9)


def test_lockstep_sbm200k_full_size():
    """Every 50 iterations through the 500 the benchmark times: the L U
    recurrence does not drift past the gradient bar over the whole run."""
    g = W.make_config_graph("sbm200k")
    recs = lockstep(g, 501, weights="f32", every=50, energy=True)
    assert [r["k"] for r in recs] == list(range(0, 501, 50))


@pytest.mark.parametrize("weights", ["f32", "bf16"])
def test_lockstep_voronoi2048_full_size(weights):
    """Every 50 iterations through the 200 the benchmark times, FP32 and BF16
    weights (the oracle on the same rounded weights)."""
    g = W.make_config_graph("voronoi2048")
    c = W.CONFIGS["voronoi2048"]
    recs = lockstep(g, 201, weights=weights, eps=c["eps"], omega0=c["omega0"], every=50,
                    energy=True)
    assert [r["k"] for r in recs] == list(range(0, 201, 50))


# ---------------------------------------------------------- free running --

@pytest.mark.parametrize("weights", ["f64", "f32", "bf16"])
def test_free_running_blobs2k_agreement(blobs2k, weights):
    c = W.CONFIGS["blobs2k"]
    P = O.make_problem(blobs2k, c["eps"], c["omega0"], weights)
    Uo, info = O.gfw_solve(P, max_iters=c["iters"])
    with B.Segmenter(blobs2k, eps=c["eps"], omega0=c["omega0"], weight_dtype=weights,
                     max_iters=c["iters"]) as s:
        st = s.solve()
        lab = s.labels()
        E = s.objective()
    assert st.status == B.FW_NOT_CONVERGED and st.iters == c["iters"] == info["iters"]
    a = agreement(lab, O.labels_from_U(Uo))
    assert a >= 0.999, a
    Eo = O.energy(Uo, P)
    assert rel(E, Eo) <= (1e-9 if weights == "f64" else 1e-4), (E, Eo)
    if weights == "f64":
        assert a == 1.0


def _control(workload, iters):
    """The oracle's own sensitivity to a rounding-level change of its input:
    its stored run on FP32-rounded weights against its stored run on the
    unrounded FP64 weights (relative change about 6e-8 per weight).  Returns
    the label disagreement and the largest relative change of g, q, alpha
    and E over the trajectory."""
    a = np.load(os.path.join(HERE, "golden", f"{workload}_oracle{iters}_f32.npz"))
    b = np.load(os.path.join(HERE, "golden", f"{workload}_oracle{iters}_f64.npz"))
    out = {"labels": float(np.mean(a["labels"] != b["labels"]))}
    for k in ("gap", "q", "alpha", "E"):
        out[k] = float(np.max(np.abs(a[k] - b[k]) / np.abs(b[k])))
    return out


@pytest.mark.parametrize("workload,weights", [("sbm200k", "f32"), ("voronoi2048", "f32"),
                                              ("voronoi2048", "bf16")])
def test_free_running_trajectory_vs_stored_oracle(workload, weights):
    """Whole free-running trajectories at full size against the stored FP64
    oracle run on the same rounded weights: g_k, q_k, alpha_k at every
    iteration, E_{k+1} by the recurrence, the final labels and the directly
    evaluated final objective.  The trajectory amplifies rounding-level
    differences: the oracle's own runs on FP32-rounded and on unrounded
    weights differ by 1e-3..4e-2 in q and alpha and in 0.16% of the image's
    labels.  The GPU must stay within twice that control, per quantity."""
    c = W.CONFIGS[workload]
    gold = np.load(os.path.join(HERE, "golden", f"{workload}_oracle{c['iters']}_{weights}.npz"))
    ctl = _control(workload, c["iters"])
    g = W.make_config_graph(workload)
    assert int(gold["nnz"]) == g.nnz
    with B.Segmenter(g, eps=c["eps"], omega0=c["omega0"], weight_dtype=weights,
                     max_iters=c["iters"]) as s:
        traj = []
        for _ in range(c["iters"] + 1):
            st = s.step(1)
            traj.append((st.gap, st.q, st.alpha, st.objective))
            if st.status != B.FW_PENDING:
                break
        lab = s.labels()
        E = s.objective()
    m = c["iters"]
    assert st.iters == m == int(gold["iters"]) and st.status == B.FW_NOT_CONVERGED
    t = np.array(traj[:m])
    ref = {"gap": gold["gap"][:m], "q": gold["q"][:m], "alpha": gold["alpha"][:m],
           "E": gold["E"][1:m + 1]}
    for col, k in enumerate(("gap", "q", "alpha", "E")):
        err = np.max(np.abs(t[:, col] - ref[k]) / np.abs(ref[k]))
        assert err <= 2.0 * ctl[k], (k, err, ctl[k])
    dis = float(np.mean(lab != gold["labels"]))
    assert dis <= 2.0 * max(ctl["labels"], 1e-6), (dis, ctl["labels"])
    assert rel(E, float(gold["energy"])) <= 2.0 * ctl["E"]


# ------------------------------------------------------------- one shot --

def test_voronoi2048_one_shot_closed_form():
    """eps < 1: alpha_0 = 1 and the result is the row argmin of L_s U_hat on the
    unlabelled pixels (Alg. 4 / Cor. nonconvb2); the fused one-shot kernel
    gives bitwise the labels of that GFW step."""
    c = W.CONFIGS["voronoi2048_oneshot"]
    g = W.make_config_graph("voronoi2048_oneshot")
    with B.Segmenter(g, eps=c["eps"], omega0=c["omega0"], weight_dtype="f32",
                     max_iters=c["iters"]) as s:
        lab1, _ = s.oneshot()
        st = s.solve()
        lab = s.labels()
        U = s.U()
    assert np.array_equal(lab1, lab)
    assert st.status == B.FW_OK and st.iters == 1 and st.alpha == 1.0
    assert np.all((U == 0) | (U == 1))
    P = O.make_problem(g, c["eps"], c["omega0"], "f32")
    LU0 = P.L @ P.Uhat
    target = np.argmin(LU0, axis=1)
    unl = g.labels < 0
    # rows whose two smallest entries are closer than FP32 resolution may flip
    part = np.sort(LU0, axis=1)
    safe = (part[:, 1] - part[:, 0]) > 1e-5 * np.maximum(1.0, np.abs(part[:, 0]))
    assert np.array_equal(lab[unl & safe], target[unl & safe])
    assert agreement(lab[unl], target[unl]) >= 0.999
    assert np.array_equal(lab[~unl], g.labels[~unl])


# ---------------------------------------------------------------- OSFW --

def _safe_rows(P, margin=1e-5):
    """Rows whose best two entries of L U_hat differ by more than rounding."""
    part = np.sort(P.L @ P.Uhat, axis=1)
    return (part[:, 1] - part[:, 0]) > margin * np.maximum(1.0, np.abs(part[:, 0]))


@pytest.mark.parametrize("oracle", ["greedy", "full"])
@pytest.mark.parametrize("weights", ["f64", "f32", "bf16"])
def test_oneshot_equals_first_choice(blobs2k, weights, oracle):
    """OSFW (Alg. 4): the labels are bitwise the (G)LMO choices the iteration
    makes at U_0 = U_hat, the iterate is untouched, and the oracle's OSFW
    agrees."""
    with B.Segmenter(blobs2k, eps=50.0, omega0=1000.0, weight_dtype=weights,
                     oracle=oracle) as s:
        U0 = s.U()
        lab, ms = s.oneshot()
        _, ch, _ = s.grad()
        assert np.array_equal(lab, ch)
        assert np.array_equal(s.U(), U0) and s.stats().iters == 0 and ms > 0
        assert s.step(3).iters == 3
    P = O.make_problem(blobs2k, 50.0, 1000.0, weights)
    _, s_o = O.osfw(P, oracle=oracle)
    safe = _safe_rows(P)
    assert np.array_equal(lab[safe], s_o[safe])
    assert agreement(lab, s_o) >= 0.999


@pytest.mark.parametrize("K", [2, 5, 13, 32])
def test_oneshot_class_counts_ragged(K):
    g = W.blobs_knn(n=40 * K + 3, K=K, seed=200 + K, label_frac=0.1)
    for wd in ("f32", "f64"):
        with B.Segmenter(g, weight_dtype=wd) as s:
            lab, _ = s.oneshot()
            _, ch, _ = s.grad()
            assert np.array_equal(lab, ch), (K, wd)


def test_oneshot_comb_laplacian(blobs2k):
    with B.Segmenter(blobs2k, laplacian="comb", eps=float("inf"), oracle="full",
                     weight_dtype="f64") as s:
        lab, _ = s.oneshot()
        _, ch, _ = s.grad()
        assert np.array_equal(lab, ch)


def test_oneshot_sbm200k_vs_oracle():
    c = W.CONFIGS["sbm200k"]
    g = W.make_config_graph("sbm200k")
    with B.Segmenter(g, eps=c["eps"], omega0=c["omega0"], weight_dtype=c["weights"]) as s:
        lab, _ = s.oneshot()
        _, ch, _ = s.grad()
    assert np.array_equal(lab, ch)
    P = O.make_problem(g, c["eps"], c["omega0"], c["weights"])
    _, s_o = O.osfw(P)
    safe = _safe_rows(P)
    assert np.array_equal(lab[safe], s_o[safe])
    assert agreement(lab, s_o) >= 0.999


# ---------------------------------------------------------- profile --

@pytest.mark.parametrize("weights,K", [("f32", 5), ("f32", 4), ("f64", 5)])
def test_profile_times_and_advances_like_step(weights, K):
    """fw_seg_profile times graphs of repeated passes on a copy of the
    problem's mutable arrays: positive times, and afterwards the iterate,
    the statistics and the rest of the run are bitwise those of stepping
    iters + 1 iterations."""
    import torch
    g = W.blobs_knn(n=3001, K=K, seed=60 + K, label_frac=0.03)
    stream = torch.cuda.Stream()
    with B.Segmenter(g, weight_dtype=weights, max_iters=60,
                     cuda_stream=stream.cuda_stream) as a, \
            B.Segmenter(g, weight_dtype=weights, max_iters=60) as b:
        p = a.profile(7)
        assert p["in_graph"] == 1
        assert min(p["pass_a"], p["pass_b"], p["finish"], p["per_iter"]) > 0
        b.step(8)
        assert np.array_equal(a.U(), b.U())
        sa, sb = a.stats(), b.stats()
        assert sa.iters == sb.iters == 8
        assert (sa.gap, sa.alpha, sa.objective) == (sb.gap, sb.alpha, sb.objective)
        ra, rb = a.solve(), b.solve()
        assert (ra.iters, ra.gap, ra.objective) == (rb.iters, rb.gap, rb.objective)
        assert np.array_equal(a.U(), b.U())


# ---------------------------------------------------------- LMO gap --

@pytest.mark.parametrize("weights,tol", [("f64", 1e-9), ("f32", TOL)])
def test_lmo_gap_diagnostic(blobs2k, weights, tol):
    """Classic (full-LMO) FW gap at the GPU iterate against the oracle's at
    the same U; never below the iteration's GLMO gap."""
    with B.Segmenter(blobs2k, eps=50.0, omega0=1000.0, weight_dtype=weights,
                     max_iters=10 ** 6) as s:
        for k in (0, 25):
            if k:
                s.step(k)
            gl = s.lmo_gap()
            U = s.U()
            P = O.make_problem(blobs2k, 50.0, 1000.0, weights)
            G = O.gradient(U, P)
            go = O.lmo_gap(G, U)
            assert rel(gl, go) <= tol, (k, gl, go)
            _, s_o, act_o = O.glmo(G, U)
            assert gl >= O.fw_gap(G, U, s_o, act_o) * (1 - 1e-6)


def test_lmo_gap_zero_at_one_shot_vertex():
    """eps < 1: every vertex is stationary, so after the one GFW step (alpha = 1,
    a binary U) the classic FW gap is exactly 0, as in the oracle."""
    g = W.voronoi_image(side=64, K=3, seed=9, label_frac=0.01)
    with B.Segmenter(g, eps=0.1, omega0=1e5, weight_dtype="f32", max_iters=10) as s:
        st = s.solve()
        assert st.iters == 1
        assert s.lmo_gap() == 0.0
        U = s.U()
    P = O.make_problem(g, 0.1, 1e5, "f32")
    assert O.lmo_gap(O.gradient(U, P), U) == 0.0


# ------------------------------------------------- warm start (f3) --

@pytest.mark.parametrize("weights,tol", [("f64", 1.0), ("f32", 0.999)])
def test_warm_start_inference_on_new_nodes(weights, tol):
    """Sec. 4, last paragraph: old rows start at their binary labels, added
    rows at 1/K; the old rows stay bitwise fixed, only the new rows are active,
    and their labels match the oracle's run from the same start."""
    g = W.blobs_knn(n=3000, K=5, seed=43, label_frac=0.03)
    rng = np.random.default_rng(6)
    new = np.zeros(g.n, bool)
    new[rng.choice(g.n, 300, replace=False)] = True
    new &= g.labels < 0
    U0 = np.full((g.n, g.K), 1.0 / g.K)
    U0[~new] = np.eye(g.K)[g.truth[~new]]
    with B.Segmenter(g, eps=50.0, omega0=1000.0, weight_dtype=weights, max_iters=150) as s:
        s.set_U(U0)
        st = s.solve()
        U = s.U()
        lab = s.labels()
    assert st.iters > 0 and st.active_rows <= int(new.sum())
    assert np.array_equal(U[~new], U0[~new])
    P = O.make_problem(g, 50.0, 1000.0, weights)
    Uo, info = O.gfw_solve(P, max_iters=150, U0=U0)
    assert agreement(lab[new], O.labels_from_U(Uo)[new]) >= tol


# ---------------------------------------------------------- edge cases --

def test_hand_example_path3():
    fx = json.load(open(os.path.join(HERE, "golden", "path3_tie.json")))
    g = W.Graph(fx["n"], np.array(fx["row_ptr"], np.int32), np.array(fx["col"], np.int32),
                np.array(fx["w"]), fx["K"], np.array(fx["labels"], np.int32),
                np.zeros(fx["n"], np.int32))
    for wd in ("f64", "f32"):
        with B.Segmenter(g, eps=fx["eps"], omega0=fx["omega0"], weight_dtype=wd) as s:
            Gp, ch, act = s.grad()
            want = np.array(fx["grad0"]) - 1.0 / fx["eps"]
            assert np.max(np.abs(Gp - want)) < (1e-15 if wd == "f64" else 1e-6)
            assert ch.tolist() == fx["s0"] and act.tolist() == fx["active0"]
            assert abs(s.objective() - fx["E0"]) < (1e-15 if wd == "f64" else 1e-6)
            st = s.solve()
            assert st.status == B.FW_OK and st.iters == 0 and st.gap == 0.0


def test_all_labelled_is_stationary():
    g = W.blobs_knn(n=300, K=3, seed=9)
    g.labels = g.truth.copy()
    with B.Segmenter(g) as s:
        st = s.solve()
        assert st.status == B.FW_OK and st.iters == 0 and st.active_rows == 0
        assert np.array_equal(s.labels(), g.truth)


def test_max_iters_zero_and_no_labels():
    g = W.blobs_knn(n=300, K=3, seed=9)
    with B.Segmenter(g, max_iters=0) as s:
        st = s.solve()
        assert st.status == B.FW_NOT_CONVERGED and st.iters == 0
    g.labels[:] = -1
    lockstep(g, 5, weights="f32")


def test_invalid_graphs_rejected():
    base = W.blobs_knn(n=64, K=3, seed=2)

    def mk(rp, col, w):
        return B.fw_seg_create(base.n, rp, col, w, base.K, base.labels)

    rp, col, w = base.row_ptr.copy(), base.col.copy(), base.w.copy()
    w2 = w.copy(); w2[0] *= 1.5
    cases = []
    cases.append((rp, col, w2, B.FW_ERR_GRAPH))                      # asymmetric
    c3 = col.copy(); c3[0] = base.n + 5
    cases.append((rp, c3, w, B.FW_ERR_GRAPH))                        # out of range
    w4 = w.copy(); w4[3] = -1.0
    cases.append((rp, col, w4, B.FW_ERR_GRAPH))                      # negative
    w5 = w.copy(); w5[7] = np.nan
    cases.append((rp, col, w5, B.FW_ERR_GRAPH))                      # NaN
    c6 = col.copy(); c6[rp[1]] = 1                                   # self loop in row 1
    cases.append((rp, c6, w, B.FW_ERR_GRAPH))
    for rp_, col_, w_, want in cases:
        with pytest.raises(B.FwError) as e:
            mk(rp_, col_, w_)
        assert e.value.status == want
    # isolated node: an empty row 0 (and its edges removed from the others)
    keep = np.ones(base.nnz, bool)
    rows = np.repeat(np.arange(base.n), np.diff(base.row_ptr))
    keep &= (rows != 0) & (base.col != 0)
    counts = np.bincount(rows[keep], minlength=base.n)
    rpi = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    with pytest.raises(B.FwError) as e:
        mk(rpi, base.col[keep], base.w[keep])
    assert e.value.status == B.FW_ERR_ISOLATED


def _ring(n, K):
    """Cycle graph on n nodes with unit weights (every row has 2 entries)."""
    i = np.arange(n)
    rp, col, w = W.from_edges(n, i, (i + 1) % n, np.ones(n))
    labels = np.full(n, -1, np.int32)
    labels[:: max(1, n // 64)] = (np.arange(len(labels[:: max(1, n // 64)])) % K)
    return rp, col, w, labels


def test_large_input_errors_on_upload_first_path():
    """Inputs of at least 2^20 rows start their upload before the host's
    planning pass: a bad label or a negative row length found by that pass
    still gives its error (after the queued copies drain), and a valid create
    on the same stream works afterwards."""
    torch = pytest.importorskip("torch")
    n, K = 1 << 20, 3
    rp, col, w, labels = _ring(n, K)
    stream = torch.cuda.Stream()
    o = B.fw_seg_default_opts(cuda_stream=stream.cuda_stream, max_iters=3)
    bad_lab = labels.copy()
    bad_lab[12345] = K
    with pytest.raises(B.FwError) as e:
        B.fw_seg_create(n, rp, col, w, K, bad_lab, o)
    assert e.value.status == B.FW_ERR_INVALID_ARG
    bad_rp = rp.copy()
    bad_rp[777] = bad_rp[778] + 1                    # row 777 has a negative length
    with pytest.raises(B.FwError) as e:
        B.fw_seg_create(n, bad_rp, col, w, K, labels, o)
    assert e.value.status == B.FW_ERR_GRAPH
    h = B.fw_seg_create(n, rp, col, w, K, labels, o)
    try:
        st = B.fw_seg_solve(h)
        # on a ring the first exact step has q < 0, so alpha = 1 and the run
        # stops at a vertex after one update
        assert st.status in (B.FW_OK, B.FW_NOT_CONVERGED) and 1 <= st.iters <= 3
        lab = B.fw_seg_labels(h)
        assert np.array_equal(lab[labels >= 0], labels[labels >= 0])
    finally:
        B.fw_seg_destroy(h)


@pytest.mark.parametrize("weights", ["f32", "bf16", "f64"])
def test_16bit_column_offsets_equal_32bit_indices(weights):
    """A pixel grid is banded (every |j - i| < 2^15), so its columns are stored
    as 16-bit offsets from the row by default; forcing 32-bit indices
    (index_width = 32) gives bitwise the same iterates, statistics, one-shot
    labels and SpMM refresh, on a ragged image (rows of 3, 5 and 8 entries)."""
    g = W.voronoi_image(side=333, height=97, K=5, label_frac=0.01, seed=23)
    out = []
    for iw in (0, 32):
        with B.Segmenter(g, weight_dtype=weights, max_iters=60, iters_per_launch=16,
                         index_width=iw, omega0=1e5) as s:
            lab1, _ = s.oneshot()
            st = s.solve()
            s.refresh()
            G, ch, _ = s.grad()
            out.append((s.U(), s.labels(), lab1, G, ch, st.iters, st.gap, st.objective))
    a, b = out
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_deterministic_bitwise(blobs2k):
    outs = []
    for _ in range(2):
        with B.Segmenter(blobs2k, max_iters=200, weight_dtype="f32") as s:
            s.solve()
            outs.append(s.U())
    assert np.array_equal(outs[0], outs[1])


def test_graph_launch_equals_stepwise(blobs2k):
    with B.Segmenter(blobs2k, max_iters=70, weight_dtype="f32", iters_per_launch=16) as s:
        s.solve()
        U1 = s.U()
    with B.Segmenter(blobs2k, max_iters=70, weight_dtype="f32") as s:
        for _ in range(80):
            if s.step(1).status != B.FW_PENDING:
                break
        U2 = s.U()
    assert np.array_equal(U1, U2)


@pytest.mark.parametrize("weights,laplacian", [("f32", "sym"), ("bf16", "sym"), ("f64", "comb")])
def test_lu0_from_fidelity_bytes_equals_dense_spmm(weights, laplacian):
    """Create and reset form L U_0 from the fidelity bytes (U_0 = U_hat: an
    unlabelled neighbour adds w/K to every class, a labelled one w to its
    class); a refresh recomputes L U with the dense SpMM of the stored U.  The
    two must agree bit for bit, so G' read before and after is identical."""
    g = W.blobs_knn(n=2531, K=7, seed=17, label_frac=0.04)
    with B.Segmenter(g, weight_dtype=weights, laplacian=laplacian) as s:
        G0, ch0, act0 = s.grad()
        s.refresh()
        G1, ch1, act1 = s.grad()
        assert np.array_equal(G0, G1)
        assert np.array_equal(ch0, ch1) and np.array_equal(act0, act1)
        s.step(3)
        s.reset()                                  # reinit + L U_hat again
        G2, _, _ = s.grad()
        assert np.array_equal(G0, G2)


def test_create_destroy_reuse_pooled_memory():
    """Handles take their arrays from a per-device pool that keeps freed memory
    mapped, so later handles get recycled (non-zero) memory.  Interleaved
    sizes and repeated create/solve/destroy must give the same bits every
    time (nothing may rely on fresh memory being zero)."""
    gs = [W.blobs_knn(n=1537, K=7, seed=5), W.sbm(n=20_000, K=10, deg_in=20.0, deg_out=2.0,
                                                 label_frac=0.01, seed=4)]
    first = {}
    for rep in range(4):
        for i, g in enumerate(gs if rep % 2 == 0 else gs[::-1]):
            key = g.n
            with B.Segmenter(g, weight_dtype="f32", max_iters=40, iters_per_launch=16) as s:
                st = s.solve()
                out = (s.U(), s.labels(), st.iters, st.gap, st.objective)
            if key not in first:
                first[key] = out
            else:
                ref = first[key]
                assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
                assert out[2:] == ref[2:]


def _stepwise(g, **opts):
    with B.Segmenter(g, **opts) as s:
        st = None
        for _ in range(opts["max_iters"] + 2):
            st = s.step(1)
            if st.status != B.FW_PENDING:
                break
        return s.U(), st


@pytest.mark.parametrize("case", ["blobs_f64_rel", "image_k4_f32", "sbm_k10_f32_armijo"])
@pytest.mark.parametrize("ipl", [7, 16])
def test_fused_decisions_equal_stepwise(case, ipl):
    """Inside a captured graph the step decision of each iteration but the
    last is taken by the next pass A (two accumulator banks, double-buffered
    inputs); direct launches take it in k_finish.  Same bits either way,
    including a stop that lands in the middle of a graph."""
    if case == "blobs_f64_rel":
        g = W.blobs_knn(n=3001, K=6, seed=21, label_frac=0.03)
        opts = dict(weight_dtype="f64", tol_mode="rel", gap_tol=0.075, max_iters=400)
    elif case == "image_k4_f32":
        g = W.voronoi_image(side=96, K=4, label_frac=0.01, seed=5)   # exact-4 pass A
        opts = dict(weight_dtype="f32", tol_mode="rel", gap_tol=0.49, max_iters=400,
                    omega0=1e5)
    else:
        g = W.sbm(n=20_000, K=10, deg_in=20.0, deg_out=2.0, label_frac=0.01, seed=4)
        opts = dict(weight_dtype="f32", step_rule="armijo", max_iters=90, lanes_per_row=4)
    U2, st2 = _stepwise(g, **opts)
    with B.Segmenter(g, iters_per_launch=ipl, **opts) as s:
        st1 = s.solve()
        U1 = s.U()
        assert s.stats().iters == st1.iters
    assert st1.iters == st2.iters
    assert st1.status == st2.status
    assert st1.gap == st2.gap and st1.objective == st2.objective and st1.alpha == st2.alpha
    assert np.array_equal(U1, U2)
    if case != "sbm_k10_f32_armijo":
        assert st1.status == B.FW_OK


def test_set_U_roundtrip_and_lockstep(blobs2k):
    rng = np.random.default_rng(3)
    U = rng.dirichlet(np.ones(blobs2k.K), size=blobs2k.n)
    with B.Segmenter(blobs2k, weight_dtype="f64") as s:
        s.set_U(U)
        assert np.array_equal(s.U(), U)
        P = O.make_problem(blobs2k, 50.0, 1000.0, "f64")
        Gp, ch, act = s.grad()
        assert np.max(np.abs(Gp - (O.gradient(U, P) - P.inv_eps))) < 1e-12
        assert rel(s.objective(), O.energy(U, P)) < 1e-12


def test_refresh_keeps_gradient_accurate():
    g = W.make_config_graph("blobs2k")
    P = O.make_problem(g, 50.0, 1000.0, "f32")
    with B.Segmenter(g, weight_dtype="f32", max_iters=300, refresh_every=50) as s:
        s.solve()
        U = s.U()
        Gp, _, _ = s.grad()
    Go = O.gradient(U, P) - P.inv_eps
    assert np.max(np.abs(Gp - Go)) / np.max(np.abs(Go)) < TOL


def test_linear_solve_special_case_on_gpu():
    """L = D - W, no penalty, full LMO: FW converges to (L + D_w)^-1 D_w U_hat."""
    rng = np.random.default_rng(77)
    n, K = 60, 3
    perm = rng.permutation(n)
    I = list(perm[:-1]); J = list(perm[1:])
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < 0.08:
                I.append(a); J.append(b)
    rp, col, w = W.from_edges(n, np.array(I), np.array(J), rng.uniform(0.1, 1.0, len(I)))
    labels = np.full(n, -1, np.int32)
    pick = rng.choice(n, 6, replace=False)
    labels[pick] = rng.integers(0, K, 6)
    g = W.Graph(n, rp, col, w, K, labels, np.zeros(n, np.int32))
    P = O.make_problem(g, math.inf, 5.0, kind="comb")
    A = P.L.toarray()
    M = A + np.diag(P.omega)
    Ustar = np.linalg.solve(M, np.diag(P.omega) @ P.Uhat)
    with B.Segmenter(g, eps=math.inf, omega0=5.0, weight_dtype="f64", laplacian="comb",
                     oracle="full", max_iters=3000) as s:
        s.solve()
        U = s.U()
    Uo, _ = O.gfw_solve(P, max_iters=3000, oracle="full")
    Estar = O.energy(Ustar, P)
    # FW on a convex quadratic: both trajectories approach U*, and rounding-order
    # differences between them shrink with the primal gap
    assert O.energy(U, P) - Estar < 1e-4 * (O.energy(P.Uhat, P) - Estar)
    assert abs(O.energy(U, P) - O.energy(Uo, P)) < 1e-6 * (O.energy(P.Uhat, P) - Estar)
    assert np.max(np.abs(U - Uo)) < 1e-3
    assert np.max(np.abs(U - Ustar)) < 0.02
