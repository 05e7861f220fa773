"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test names the paper passage or the textbook fact it checks.  They run
on the CPU only and are sized to finish in seconds.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2508_09738_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def random_connected_graph(n, rng, extra=0.4, wlo=0.1, whi=1.0):
    """Random weighted connected graph: a random spanning path plus extra edges."""
    perm = rng.permutation(n)
    I = list(perm[:-1])
    J = list(perm[1:])
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < extra:
                I.append(a)
                J.append(b)
    w = rng.uniform(wlo, whi, size=len(I))
    row_ptr, col, ww = W.from_edges(n, np.array(I), np.array(J), w)
    return row_ptr, col, ww


def make_graph(n, K, rng, nlab=2, extra=0.4):
    row_ptr, col, w = random_connected_graph(n, rng, extra)
    labels = np.full(n, -1, dtype=np.int32)
    pick = rng.choice(n, size=nlab, replace=False)
    labels[pick] = rng.integers(0, K, size=nlab)
    truth = np.zeros(n, dtype=np.int32)
    return W.Graph(n, row_ptr, col, w, K, labels, truth)


def dense_W(g):
    A = np.zeros((g.n, g.n))
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    A[rows, g.col] = g.w
    return A


def random_simplex_rows(n, K, rng):
    X = rng.exponential(size=(n, K))
    return X / X.sum(1, keepdims=True)


# ------------------------------------------------------------------ P1 --
# Textbook Laplacian facts (Sec. 1): L_s symmetric PSD with spectrum in
# [0, 2] and null vector D^1/2 1; L = D - W has L 1 = 0.

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_laplacian_invariants(seed):
    rng = np.random.default_rng(seed)
    g = make_graph(40, 3, rng, extra=0.2)
    Ls = O.laplacian(g, "sym").toarray()
    L = O.laplacian(g, "comb").toarray()
    assert np.array_equal(Ls, Ls.T)
    assert np.allclose(np.diag(Ls), 1.0)
    ev = np.linalg.eigvalsh(Ls)
    assert ev.min() > -1e-12 and ev.max() <= 2.0 + 1e-12
    d = dense_W(g).sum(1)
    assert np.max(np.abs(Ls @ np.sqrt(d))) < 1e-12
    assert np.max(np.abs(L @ np.ones(g.n))) < 1e-12
    for _ in range(5):
        x = rng.normal(size=g.n)
        assert x @ Ls @ x >= -1e-12
    # bipartite graph reaches lambda_max = 2 exactly (textbook)
    row_ptr, col, w = W.from_edges(4, np.array([0, 1, 2]), np.array([1, 2, 3]), np.ones(3))
    gp = W.Graph(4, row_ptr, col, w, 2, np.array([0, -1, -1, 1], np.int32), np.zeros(4, np.int32))
    assert abs(np.linalg.eigvalsh(O.laplacian(gp).toarray()).max() - 2.0) < 1e-12


def test_laplacian_sparse_graph_symmetric_and_null_vector():
    g = W.sbm(n=2000, K=4, deg_in=8, deg_out=1, seed=3)
    Ls = O.laplacian(g, "sym")
    assert (abs(Ls - Ls.T)).max() == 0.0
    d = O.degrees(g.n, g.row_ptr, g.col, g.w)
    assert np.max(np.abs(Ls @ np.sqrt(d))) < 1e-12


def test_round_weights_bf16_matches_torch():
    """bf16 storage rounding equals torch's float32->bfloat16 round-to-nearest-even."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(0, 1, 2000), rng.exponential(1e-3, 2000),
                        np.array([1.0, 0.5, 1.00390625, 1.001953125, 3.0e-30])])
    mine = O.round_weights(x, "bf16")
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mine, ref)
    assert np.array_equal(O.round_weights(x, "f32"), x.astype(np.float32).astype(np.float64))


# --------------------------------------------------------------- golden --

def test_path3_hand_derivation():
    """Worked example derived by hand (tests/golden/path3_tie.json)."""
    fx = json.load(open(os.path.join(HERE, "golden", "path3_tie.json")))
    g = W.Graph(fx["n"], np.array(fx["row_ptr"], np.int32), np.array(fx["col"], np.int32),
                np.array(fx["w"]), fx["K"], np.array(fx["labels"], np.int32),
                np.zeros(fx["n"], np.int32))
    P = O.make_problem(g, fx["eps"], fx["omega0"])
    U0 = P.Uhat
    assert abs(O.energy(U0, P) - fx["E0"]) < 1e-15
    G = O.gradient(U0, P)
    assert np.max(np.abs(G - np.array(fx["grad0"]))) < 1e-15
    _, s, active = O.glmo(G, U0)
    assert s.tolist() == fx["s0"]
    assert active.tolist() == fx["active0"]
    assert O.fw_gap(G, U0, s, active) == fx["g0"]
    U, info = O.gfw_solve(P, max_iters=10)
    assert info["status"] == "stationary" and info["iters"] == 0


# ------------------------------------------------------------------ P2 --
# Iterates stay in Sigma (eq. fs), g_k >= 0 termwise, ||D_k||^2 <= 2n
# (Prop. pr:diam).

def test_iterates_feasible_and_gap_nonnegative():
    g = W.blobs_knn(n=300, K=4, seed=11)
    P = O.make_problem(g, 50.0, 1000.0)
    U = P.Uhat.copy()
    for k in range(60):
        it = O.gfw_iteration(U, P)
        assert it.g >= 0.0
        assert it.nD <= 2 * g.n
        # termwise gap equals the definition -<G, D> on Sigma
        assert abs(it.g - (-np.sum(it.G * it.D))) <= 1e-9 * max(1.0, abs(it.g))
        if it.g <= 0:
            break
        U = U + it.alpha * it.D
        assert U.min() >= 0.0
        assert np.max(np.abs(U.sum(1) - 1.0)) < 1e-12


# ------------------------------------------------------------------ P3 --
# One-shot closed form for eps < 1 (sym-normalised L_s, labelled rows frozen):
# q <= (2 - 2/eps) ||D||^2 < 0, so alpha_0 = 1 and U_1 is the row-wise argmin of
# L_s U_hat on unlabelled rows (Alg. 4 OSFW, Cor. nonconvb2, Fig. 1 one-shot band).

@pytest.mark.parametrize("gen", ["blobs", "image"])
def test_one_shot_closed_form(gen):
    if gen == "blobs":
        g = W.blobs_knn(n=400, K=5, seed=21)
    else:
        g = W.voronoi_image(side=24, K=3, seed=22, label_frac=0.05)
    P = O.make_problem(g, 0.1, 1e5)
    # independent dense evaluation of L_s U_hat
    A = dense_W(g)
    d = A.sum(1)
    Ls = np.eye(g.n) - A / np.sqrt(np.outer(d, d))
    target = np.argmin(Ls @ P.Uhat, axis=1)
    it = O.gfw_iteration(P.Uhat, P)
    assert it.q < 0 and it.alpha == 1.0
    U, info = O.gfw_solve(P, max_iters=50)
    assert info["iters"] == 1 and info["status"] == "stationary"
    unl = g.labels < 0
    assert np.array_equal(O.labels_from_U(U)[unl], target[unl])
    assert np.array_equal(O.labels_from_U(U)[~unl], g.labels[~unl])
    assert np.all((U == 0) | (U == 1))
    # Cor. nonconvb2: for such eps GFW is OSFW (Alg. 4)
    U1, s1 = O.osfw(P)
    assert np.array_equal(U1, U) and np.array_equal(s1, O.labels_from_U(U))


# OSFW at any eps (Alg. 4): at U_hat the penalty gradient (1/eps)(1 - 2u) is
# the same for every class of an unlabelled row and the fidelity gradient is
# zero, so S_0 = GLMO(grad E(U_hat)) picks argmin_k (L_s U_hat)_ik on the
# unlabelled rows (lowest index) and keeps every labelled row; checked against
# an independent dense L_s, at an eps where GFW does not stop after one step.
@pytest.mark.parametrize("oracle", ["greedy", "full"])
def test_osfw_any_eps_closed_form(oracle):
    g = W.blobs_knn(n=350, K=4, seed=23, label_frac=0.05)
    P = O.make_problem(g, 50.0, 1000.0)
    A = dense_W(g)
    d = A.sum(1)
    Ls = np.eye(g.n) - A / np.sqrt(np.outer(d, d))
    LU = Ls @ P.Uhat
    U1, s = O.osfw(P, oracle=oracle)
    unl = g.labels < 0
    assert np.all((U1 == 0) | (U1 == 1)) and np.all(U1.sum(1) == 1)
    assert np.array_equal(s, O.labels_from_U(U1))
    assert np.array_equal(s[unl], np.argmin(LU, axis=1)[unl])
    if oracle == "greedy":
        assert np.array_equal(s[~unl], g.labels[~unl])
    else:
        # full LMO at U_hat: a labelled row adds omega_0 (u - e_c) = 0 and
        # (1/eps)(1 - 2u), which is -1/eps on its class and +1/eps elsewhere
        G = LU + (1.0 - 2.0 * P.Uhat) / 50.0
        assert np.array_equal(s[~unl], np.argmin(G, axis=1)[~unl])
    # the first GFW iteration chooses the same classes (Alg. 3 step 2)
    it = O.gfw_iteration(P.Uhat, P, oracle=oracle)
    assert np.array_equal(it.s, s)
    # and GFW at this eps does not end after that step
    assert 0.0 < it.alpha < 1.0


# ------------------------------------------------------------------ P4 --
# omega_0 invariance (Fig. 1: accuracy identical across omega_0): from
# U_0 = U_hat labelled rows never move, so the trajectory is bitwise the same.

def test_omega0_invariance():
    g = W.blobs_knn(n=300, K=3, seed=31)
    runs = []
    for w0 in (10.0, 1000.0, 1e4):
        P = O.make_problem(g, 50.0, w0)
        U, info = O.gfw_solve(P, max_iters=40, record=True)
        runs.append((U, info["hist"]["g"], info["hist"]["alpha"]))
    for U, gh, ah in runs[1:]:
        assert np.array_equal(U, runs[0][0])
        assert gh == runs[0][1] and ah == runs[0][2]


# ------------------------------------------------------------------ P5 --
# E is quadratic with constant Hessian (App. C): E(U + aD) = E(U) - a g + a^2 q / 2;
# the exact step minimises it on [0,1] and E decreases monotonically.

def test_exact_quadratic_and_line_search():
    rng = np.random.default_rng(41)
    g = W.blobs_knn(n=200, K=4, seed=41)
    P = O.make_problem(g, 5.0, 100.0)
    U = P.Uhat.copy()
    Eprev = O.energy(U, P)
    for k in range(25):
        it = O.gfw_iteration(U, P, with_energy=True)
        if it.g <= 0:
            break
        E0 = O.energy(U, P)
        for a in rng.uniform(0, 1, 5):
            lhs = O.energy(U + a * it.D, P) - E0
            rhs = -a * it.g + 0.5 * a * a * it.q
            assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(E0))
        grid = np.linspace(0, 1, 10001)
        phi = -grid * it.g + 0.5 * grid ** 2 * it.q
        phi_a = -it.alpha * it.g + 0.5 * it.alpha ** 2 * it.q
        assert phi_a <= phi.min() + 1e-12 * max(1.0, abs(E0))
        U = U + it.alpha * it.D
        Enew = O.energy(U, P)
        assert Enew <= Eprev + 1e-12 * abs(Eprev)
        Eprev = Enew


# ------------------------------------------------------------------ P6 --
# Theorem th:equivalence: for eps <= eps_bar < 2/lambda_max(L_s + D_w) every
# minimiser over Sigma is a vertex.  Brute force over all 3^n vertices.

def _batch_energy(Us, Ls, Uhat, omega, eps):
    LU = np.einsum("ij,bjk->bik", Ls, Us)
    quad = 0.5 * np.einsum("bik,bik->b", Us, LU)
    pen = np.einsum("bik->b", Us * (1 - Us)) / eps
    R = Uhat[None] - Us
    fid = 0.5 * np.einsum("i,bik->b", omega, R * R)
    return quad + pen + fid


def _vertex_min(n, K, Ls, Uhat, omega, eps):
    best = np.inf
    for chunk in itertools.islice(_chunks(itertools.product(range(K), repeat=n), 4096), None):
        lab = np.array(chunk)
        Us = np.zeros((lab.shape[0], n, K))
        Us[np.arange(lab.shape[0])[:, None], np.arange(n)[None], lab] = 1.0
        best = min(best, _batch_energy(Us, Ls, Uhat, omega, eps).min())
    return best


def _chunks(it, m):
    buf = []
    for x in it:
        buf.append(x)
        if len(buf) == m:
            yield buf
            buf = []
    if buf:
        yield buf


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_brute_force_binary_minimiser(seed):
    rng = np.random.default_rng(100 + seed)
    n, K = 7, 3
    g = make_graph(n, K, rng, nlab=1 + seed % 3)
    P0 = O.make_problem(g, 1.0, 2.0)
    Ls = P0.L.toarray()
    lam = np.linalg.eigvalsh(Ls + np.diag(P0.omega)).max()
    eps_bar = 2.0 / lam
    eps = 0.5 * eps_bar
    P = O.make_problem(g, eps, 2.0)
    Hm = Ls + np.diag(P.omega) - (2.0 / eps) * np.eye(n)
    assert np.linalg.eigvalsh(Hm).max() < 0          # strictly concave
    Vstar = _vertex_min(n, K, Ls, P.Uhat, P.omega, eps)
    Us = rng.dirichlet(np.ones(K), size=(20000, n))
    assert _batch_energy(Us, Ls, P.Uhat, P.omega, eps).min() >= Vstar - 1e-12
    # FW from many random interior starts ends at a vertex no better than V*
    for _ in range(20):
        U0 = random_simplex_rows(n, K, rng)
        U, info = O.gfw_solve(P, max_iters=200, oracle="full", U0=U0)
        assert O.energy(U, P) >= Vstar - 1e-12
    # GFW from U_hat ends at a binary GLMO-stationary vertex
    U, info = O.gfw_solve(P, max_iters=200)
    assert np.all((U == 0) | (U == 1))
    it = O.gfw_iteration(U, P)
    assert not it.active.any()


def test_brute_force_control_fractional_minimiser():
    """Control: with eps far above eps_bar a fractional point beats every vertex,
    so the brute-force test above can fail."""
    rng = np.random.default_rng(7)
    found = False
    for t in range(10):
        n, K = 6, 3
        g = make_graph(n, K, rng, nlab=1)
        P0 = O.make_problem(g, 1.0, 2.0)
        Ls = P0.L.toarray()
        eps = 100 * 2.0 / np.linalg.eigvalsh(Ls + np.diag(P0.omega)).max()
        P = O.make_problem(g, eps, 2.0)
        Vstar = _vertex_min(n, K, Ls, P.Uhat, P.omega, eps)
        U, _ = O.gfw_solve(P, max_iters=3000, oracle="full", tol=1e-12)
        if O.energy(U, P) < Vstar - 1e-6:
            found = True
            break
    assert found


# ------------------------------------------------------------------ P7 --
# Special case reducing to a linear solve: L = D - W, no penalty (eps = inf).
# E is convex and its minimiser U* = (L + D_w)^-1 D_w U_hat lies in Sigma
# (L 1 = 0 gives unit row sums; (L + D_w)^-1 >= 0 for a nonsingular M-matrix),
# so full-LMO FW (Alg. 2) from U_hat must converge to it.

def test_linear_solve_special_case():
    rng = np.random.default_rng(77)
    n, K = 60, 3
    g = make_graph(n, K, rng, nlab=6, extra=0.08)
    P = O.make_problem(g, math.inf, 5.0, kind="comb")
    A = dense_W(g)
    L = np.diag(A.sum(1)) - A
    M = L + np.diag(P.omega)
    Ustar = np.linalg.solve(M, np.diag(P.omega) @ P.Uhat)
    assert Ustar.min() >= -1e-12 and np.allclose(Ustar.sum(1), 1.0)
    Estar = O.energy(Ustar, P)
    mu = np.linalg.eigvalsh(M).min()              # strong convexity modulus
    U = P.Uhat.copy()
    E0 = O.energy(U, P) - Estar
    Eprev = np.inf
    for k in range(3000):
        it = O.gfw_iteration(U, P, oracle="full")
        Ek = O.energy(U, P) - Estar
        # convex E: the FW gap bounds the primal error; line search is monotone
        assert -1e-12 <= Ek <= it.g + 1e-10
        # with the full LMO every row is active, so g is the classic FW gap
        assert abs(O.lmo_gap(it.G, U) - it.g) <= 1e-12 * max(1.0, it.g)
        assert Ek <= Eprev + 1e-12
        Eprev = Ek
        U = U + it.alpha * it.D
    Ek = O.energy(U, P) - Estar
    assert Ek < 1e-3 * E0
    # strong convexity: ||U - U*||_F^2 <= 2 (E(U) - E*) / mu
    assert np.sum((U - Ustar) ** 2) <= 2 * Ek / mu + 1e-12
    assert np.max(np.abs(U - Ustar)) < 0.02


# ------------------------------------------------------------------ P8 --
# App. D: for eps <= eps_tilde = 1/[K (rho_max + omega_0)] the GLMO and the LMO
# agree at every point of Sigma.

def test_glmo_equals_lmo_for_small_eps():
    rng = np.random.default_rng(81)
    n, K = 50, 4
    g = make_graph(n, K, rng, nlab=5, extra=0.1)
    omega0 = 3.0
    P0 = O.make_problem(g, 1.0, omega0)
    rho = np.abs(P0.L.toarray()).sum(1).max()
    eps_t = 1.0 / (K * (rho + omega0))
    P = O.make_problem(g, 0.9 * eps_t, omega0)
    for trial in range(30):
        U = random_simplex_rows(n, K, rng)
        # zero out random entries and make some rows binary
        mask = rng.random((n, K)) < 0.3
        U = np.where(mask, 0.0, U)
        U[U.sum(1) == 0, 0] = 1.0
        U = U / U.sum(1, keepdims=True)
        rows = rng.random(n) < 0.3
        U[rows] = np.eye(K)[rng.integers(0, K, rows.sum())]
        G = O.gradient(U, P)
        Sg, sg, act = O.glmo(G, U)
        Sl, sl = O.lmo(G)
        assert np.array_equal(Sg, Sl)


# ------------------------------------------------------------------ P9 --
# Finite differences of E (eq. gradgl_vv2) against grad E (eq. gradgl_vv2g).

def test_gradient_finite_differences():
    rng = np.random.default_rng(91)
    g = make_graph(12, 3, rng, nlab=3)
    P = O.make_problem(g, 0.7, 4.0)
    U = random_simplex_rows(12, 3, rng)
    G = O.gradient(U, P)
    h = 1e-6
    for _ in range(12):
        i, k = rng.integers(12), rng.integers(3)
        E1 = U.copy(); E1[i, k] += h
        E2 = U.copy(); E2[i, k] -= h
        fd = (O.energy(E1, P) - O.energy(E2, P)) / (2 * h)
        assert abs(fd - G[i, k]) <= 5e-7 * max(1.0, abs(G[i, k]))


def test_armijo_step_satisfies_rule():
    """Armijo (eqs. eta, Armijo): the accepted delta^j passes the test and
    delta^(j-1) does not."""
    g = W.blobs_knn(n=150, K=3, seed=95)
    P = O.make_problem(g, 50.0, 1000.0)
    U = P.Uhat.copy()
    for k in range(10):
        it = O.gfw_iteration(U, P, step="armijo")
        if it.g <= 0:
            break
        E0 = O.energy(U, P)
        a = it.alpha
        assert E0 - O.energy(U + a * it.D, P) >= 1e-6 * a * it.g
        if a < 1.0:
            assert not (E0 - O.energy(U + 2 * a * it.D, P) >= 1e-6 * 2 * a * it.g)
        U = U + a * it.D


def test_labels_lowest_index_tie():
    U = np.array([[0.5, 0.5, 0.0], [0.2, 0.4, 0.4], [0.0, 0.0, 1.0]])
    assert O.labels_from_U(U).tolist() == [0, 1, 2]
    G = np.array([[1.0, 1.0, 0.0], [3.0, 2.0, 2.0], [0.0, 0.0, 0.0]])
    _, s, act = O.glmo(G, U)
    # row 0: class 2 is outside supp, tie on {0,1} -> 0; row 1: tie -> 1; row 2 binary
    assert s.tolist() == [0, 1, 2] and act.tolist() == [True, True, False]


# ------------------------------------------------------------------ f3 --
# Warm-start inference on added nodes (Sec. 4, last paragraph): start from a
# point whose old rows are the binary solution of the old data and whose new
# rows are at 1/K.  A binary row is never active under the GLMO, so the old
# rows stay exactly as they were and only the new rows move.
def test_warm_start_new_nodes_only():
    g = W.blobs_knn(n=600, K=4, seed=41, label_frac=0.05)
    rng = np.random.default_rng(5)
    new = np.zeros(g.n, bool)
    new[rng.choice(g.n, 60, replace=False)] = True
    new &= g.labels < 0
    P = O.make_problem(g, 50.0, 1000.0)
    U0 = np.full((g.n, g.K), 1.0 / g.K)
    U0[~new] = np.eye(g.K)[g.truth[~new]]
    U, info = O.gfw_solve(P, max_iters=60, U0=U0, record=True)
    assert np.array_equal(U[~new], U0[~new])
    assert max(info["hist"]["active"]) <= int(new.sum())
    assert np.any(U[new] != U0[new])
    assert info["iters"] > 0


# ------------------------------------------------------------ LMO gap --
# The classic FW gap of the full LMO is the stationarity measure over Sigma:
# (i) it is never below the GLMO gap (the GLMO minimises over the support
# only and leaves binary rows out); (ii) for eps < 1 the penalty term makes
# every vertex stationary: at a binary row with class c, G_ic carries -1/eps
# and every other class +1/eps, and 2/eps exceeds the spread of (L_s U)_i,
# whose entries lie in [-1, 2] on Sigma -- so the gap is 0 at every vertex.
def test_lmo_gap_bounds_and_vertex_stationarity():
    rng = np.random.default_rng(91)
    g = W.blobs_knn(n=300, K=4, seed=92, label_frac=0.05)
    P = O.make_problem(g, 50.0, 1000.0)
    for _ in range(5):
        U = random_simplex_rows(g.n, g.K, rng)
        G = O.gradient(U, P)
        _, s, act = O.glmo(G, U)
        assert O.lmo_gap(G, U) >= O.fw_gap(G, U, s, act) - 1e-12
    U, _ = O.gfw_solve(P, max_iters=30)
    it = O.gfw_iteration(U, P)
    assert O.lmo_gap(it.G, U) >= it.g - 1e-12
    # a binary point: GLMO gap 0 by construction, LMO gap 0 only if stationary
    Pe = O.make_problem(g, 0.1, 1000.0)
    for _ in range(3):
        V = np.eye(g.K)[rng.integers(0, g.K, g.n)]
        V[g.labels >= 0] = np.eye(g.K)[g.labels[g.labels >= 0]]
        assert O.lmo_gap(O.gradient(V, Pe), V) == 0.0
    # at eps = 50 a random vertex is not stationary
    assert O.lmo_gap(O.gradient(V, P), V) > 0.0
