"""FP64 CPU oracle of the Greedy Frank-Wolfe (GFW) segmentation method.

TEST INFRASTRUCTURE, not product code.  Only the test suite, the package
smoke check (`__graft_entry__.smoke`) and the CPU-baseline / reference leg of
`bench.py` may import or run anything under `oracle/`.  The CUDA library never
calls it and shares no code with it; the only shared module is the seeded
input generator (`paper_2508_09738_gb300.workloads`), which holds none of the
method's arithmetic.

Everything here is plain numpy / scipy.sparse in float64, written from the
paper "A Greedy Frank-Wolfe for multiclass data segmentation"
(arXiv 2508.09738) in its notation:

  * graph, degrees, Laplacians L = D - W, L_s = I - D^-1/2 W D^-1/2   (Sec. 1)
  * fidelity data  U_hat, D_omega                                      (Sec. 2)
  * penalty energy E and its gradient        (Sec. 2.1, eqs. gradgl_vv2/g)
  * Hessian I_K (x) (L_s + D_omega - (2/eps) I)              (App. C proof)
  * LMO over the simplex product Sigma                      (Sec. 4, Alg. 2)
  * GLMO, the greedy row rule                        (Sec. 4, eq. eq:LMOpr)
  * GFW iteration                                           (Sec. 4, Alg. 3)
  * One-Shot Frank-Wolfe, U_1 = GLMO(grad E(U_0))          (Sec. 4, Alg. 4)
  * FW gap g_k = -<grad E(U_k), D_k>             (Thm th:nonconvb; Sec. 5.1)
  * classic (full-LMO) FW gap, the stationarity measure        (Sec. 4, Alg. 2)
  * Armijo step (eqs. eta, Armijo; delta=0.5, gamma=1e-6 in Sec. 5.1)
  * U_0 = U_hat with unlabelled rows at 1/K                         (Sec. 5.1)

Readings where the paper is silent or where this implementation departs from
it on purpose (each is listed with its justification in the design notes):

  R1  argmin ties in LMO/GLMO go to the lowest class index.
  R2  "binary row" means every stored entry is exactly 0.0 or 1.0;
      supp(u_i) = {j : u_ij > 0}; both on the iterate's own stored values.
  R3  the gap is summed termwise, g = sum_i sum_k u_ik (G_ik - G_i,s_i); on
      Sigma (rows sum to one) this is exactly -<G, D>.
  R4  the step is the exact line search of the quadratic E along D:
      q = <D, H D>;  alpha = 1 if q <= 0 else min(1, g/q).  Armijo is kept
      as the paper-faithful alternative (`step="armijo"`).
  R5  stop when g <= tol (absolute, or relative to g_0), or no row is
      active, or g <= 0, or the iteration cap is reached; the test happens
      before the update (Alg. 3 step 4).
  R6  final labels are the row argmax of U, lowest index on ties.
  R7  eps = inf is accepted and means 1/eps = 0 (no penalty term).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse as sp

__all__ = [
    "round_weights", "degrees", "normalized_weights", "laplacian", "fidelity",
    "Problem", "make_problem", "energy", "gradient", "lmo", "glmo", "fw_gap", "lmo_gap",
    "hessian_apply", "curvature", "exact_step", "armijo_step", "Iterate",
    "gfw_iteration", "gfw_solve", "osfw", "labels_from_U",
]


# ---------------------------------------------------------------- weights --

def round_weights(x: np.ndarray, dtype: str) -> np.ndarray:
    """Round float64 values to the storage precision and widen them back.

    'f64' keeps them; 'f32' rounds to nearest-even float32; 'bf16' rounds to
    float32 (nearest-even) and then to bfloat16 (nearest-even on the upper 16
    bits of the float32 pattern).  Used so the oracle works on exactly the
    weights a lower-precision implementation stores.
    """
    x = np.asarray(x, dtype=np.float64)
    if dtype == "f64":
        return x.copy()
    f = x.astype(np.float32)
    if dtype == "f32":
        return f.astype(np.float64)
    if dtype == "bf16":
        b = f.view(np.uint32).astype(np.uint64)
        lsb = (b >> 16) & 1
        b = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
        return b.view(np.float32).astype(np.float64)
    raise ValueError(f"unknown weight dtype {dtype!r}")


def degrees(n: int, row_ptr: np.ndarray, col: np.ndarray, w: np.ndarray) -> np.ndarray:
    """d_i = sum_j w_ij, the row sums of W (Sec. 1), accumulated in CSR order."""
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    return np.bincount(rows, weights=w, minlength=n).astype(np.float64)


def normalized_weights(n, row_ptr, col, w) -> np.ndarray:
    """Entries of D^-1/2 W D^-1/2: w_ij / sqrt(d_i d_j) (Sec. 1)."""
    d = degrees(n, row_ptr, col, w)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    return w / np.sqrt(d[rows] * d[col])


def laplacian(g, kind: str = "sym", weight_dtype: str = "f64") -> sp.csr_matrix:
    """Graph Laplacian as an FP64 sparse matrix (Sec. 1).

    kind='sym':  L_s = I - D^-1/2 W D^-1/2  (unit diagonal; the paper's choice)
    kind='comb': L   = D - W
    The off-diagonal entries are rounded to `weight_dtype` storage first
    (`round_weights`), the diagonal of L_s stays exactly 1.
    """
    n, row_ptr, col, w = g.n, g.row_ptr, g.col, g.w
    if kind == "sym":
        off = round_weights(normalized_weights(n, row_ptr, col, w), weight_dtype)
        diag = np.ones(n)
    elif kind == "comb":
        off = round_weights(w, weight_dtype)
        diag = round_weights(degrees(n, row_ptr, col, w), weight_dtype)
    else:
        raise ValueError(kind)
    Woff = sp.csr_matrix((off, col.astype(np.int64), row_ptr.astype(np.int64)), shape=(n, n))
    return (sp.diags(diag) - Woff).tocsr()


def fidelity(labels: np.ndarray, K: int, omega0: float):
    """U_hat and the diagonal of D_omega (Sec. 2).

    A fidelity node i with class c gets u_hat_i = e_c and omega_i = omega0;
    every other node gets u_hat_i = (1/K) 1 (its start value, Sec. 5.1) and
    omega_i = 0.
    """
    n = labels.shape[0]
    Uhat = np.full((n, K), 1.0 / K)
    lab = labels >= 0
    Uhat[lab] = 0.0
    Uhat[np.flatnonzero(lab), labels[lab]] = 1.0
    omega = np.where(lab, float(omega0), 0.0)
    return Uhat, omega


@dataclasses.dataclass
class Problem:
    L: sp.csr_matrix       # L_s (or L), FP64
    Uhat: np.ndarray       # n x K
    omega: np.ndarray      # n
    eps: float             # penalty parameter (inf allowed: no penalty)
    K: int

    @property
    def inv_eps(self) -> float:
        return 0.0 if np.isinf(self.eps) else 1.0 / self.eps


def make_problem(g, eps: float, omega0: float, weight_dtype: str = "f64",
                 kind: str = "sym") -> Problem:
    Uhat, omega = fidelity(g.labels, g.K, omega0)
    return Problem(laplacian(g, kind, weight_dtype), Uhat, omega, float(eps), g.K)


# ---------------------------------------------------------- energy model --

def energy(U: np.ndarray, P: Problem) -> float:
    """E(U) = 1/2 tr(U^T L_s U) + 1/eps tr(U (1 - U^T)) + 1/2 ||D_w^1/2 (U_hat - U)||_F^2
    (Sec. 2.1, eq. gradgl_vv2)."""
    quad = 0.5 * float(np.sum(U * (P.L @ U)))
    pen = P.inv_eps * float(np.sum(U * (1.0 - U)))
    R = P.Uhat - U
    fid = 0.5 * float(np.sum(P.omega[:, None] * R * R))
    return quad + pen + fid


def gradient(U: np.ndarray, P: Problem) -> np.ndarray:
    """grad E(U) = L_s U + 1/eps (1 - 2U) - D_w (U_hat - U)  (eq. gradgl_vv2g)."""
    return (P.L @ U) + P.inv_eps * (1.0 - 2.0 * U) - P.omega[:, None] * (P.Uhat - U)


def hessian_apply(D: np.ndarray, P: Problem) -> np.ndarray:
    """(I_K (x) (L_s + D_w - 2/eps I)) applied to D, column by column (App. C)."""
    return (P.L @ D) + P.omega[:, None] * D - 2.0 * P.inv_eps * D


# ---------------------------------------------------------------- oracles --

def lmo(G: np.ndarray):
    """LMO over Sigma (Sec. 4): row i goes to e_{j_i}, j_i = argmin_j (g_i)_j (R1).

    Returns (S, s) with S the one-hot matrix and s the chosen class per row.
    """
    s = np.argmin(G, axis=1)
    S = np.zeros_like(G)
    S[np.arange(G.shape[0]), s] = 1.0
    return S, s


def glmo(G: np.ndarray, U: np.ndarray):
    """Greedy LMO (Sec. 4, eq. eq:LMOpr).

    Active rows I = {i : u_i not in {0,1}^K} (R2).  An active row gets
    w_i = e_{j_i} with j_i the lowest index minimising (g_i)_j over
    supp(u_i) = {j : u_ij > 0}; every other row keeps w_i = u_i.
    Returns (Wm, s, active): the GLMO output, the chosen class per row (the
    position of the 1 for inactive binary rows) and the active mask.
    """
    binary = np.all((U == 0.0) | (U == 1.0), axis=1)
    active = ~binary
    masked = np.where(U > 0.0, G, np.inf)
    s = np.argmin(masked, axis=1)
    s_inactive = np.argmax(U, axis=1)
    s = np.where(active, s, s_inactive)
    Wm = U.copy()
    rows = np.flatnonzero(active)
    Wm[rows] = 0.0
    Wm[rows, s[rows]] = 1.0
    return Wm, s, active


def fw_gap(G: np.ndarray, U: np.ndarray, s: np.ndarray, active: np.ndarray) -> float:
    """FW gap g = -<G, D> with D = S - U, summed termwise (R3):
    g = sum_{i active} sum_k u_ik (G_ik - G_{i,s_i}); every term is >= 0."""
    Gs = G[np.arange(G.shape[0]), s]
    terms = U * (G - Gs[:, None])
    return float(np.sum(terms[active]))


def lmo_gap(G: np.ndarray, U: np.ndarray) -> float:
    """Classic FW gap of the full LMO (Alg. 2): <G, U - S> with S = LMO(G),
    summed termwise as sum_i sum_k u_ik (G_ik - min_j G_ij); every term is
    >= 0, and the sum is 0 exactly at a stationary point of E over Sigma."""
    m = np.min(G, axis=1)
    return float(np.sum(U * (G - m[:, None])))


def curvature(D: np.ndarray, P: Problem) -> float:
    """q = <D, H D>: E(U + a D) = E(U) - a g + a^2 q / 2 exactly (E is quadratic)."""
    return float(np.sum(D * hessian_apply(D, P)))


def exact_step(g: float, q: float) -> float:
    """Minimiser over [0,1] of phi(a) = -a g + a^2 q / 2 with g > 0 (R4)."""
    if q <= 0.0:
        return 1.0
    return min(1.0, g / q)


def armijo_step(U, D, g, P: Problem, delta: float = 0.5, gamma: float = 1e-6,
                max_halvings: int = 60) -> float:
    """Armijo rule (eqs. eta, Armijo): alpha = delta^j for the smallest j >= 0
    with E(U) - E(U + alpha D) >= gamma * alpha * g, E evaluated directly."""
    E0 = energy(U, P)
    a = 1.0
    for _ in range(max_halvings):
        if E0 - energy(U + a * D, P) >= gamma * a * g:
            return a
        a *= delta
    return a


# ------------------------------------------------------------- iteration --

@dataclasses.dataclass
class Iterate:
    G: np.ndarray          # grad E(U_k), full formula
    s: np.ndarray          # chosen class per row
    active: np.ndarray     # rows the (G)LMO moves
    D: np.ndarray          # D_k = S_k - U_k
    g: float               # FW gap
    q: float               # <D, H D>
    alpha: float           # step
    nD: float              # ||D||_F^2
    E: Optional[float]     # E(U_k) evaluated directly (if requested)


def gfw_iteration(U: np.ndarray, P: Problem, oracle: str = "greedy",
                  step: str = "exact", with_energy: bool = False) -> Iterate:
    """One GFW iteration at U_k (Alg. 3; Alg. 2 when oracle='full')."""
    G = gradient(U, P)
    if oracle == "greedy":
        S, s, active = glmo(G, U)
    elif oracle == "full":
        S, s = lmo(G)
        active = np.ones(U.shape[0], dtype=bool)
    else:
        raise ValueError(oracle)
    D = S - U
    g = fw_gap(G, U, s, active)
    q = curvature(D, P)
    if g > 0.0:
        alpha = exact_step(g, q) if step == "exact" else armijo_step(U, D, g, P)
    else:
        alpha = 0.0
    E = energy(U, P) if with_energy else None
    return Iterate(G, s, active, D, g, q, alpha, float(np.sum(D * D)), E)


def gfw_solve(P: Problem, max_iters: int = 500, tol: float = 0.0,
              tol_mode: str = "abs", oracle: str = "greedy", step: str = "exact",
              U0: Optional[np.ndarray] = None, record: bool = False,
              with_energy: bool = False):
    """GFW from U_0 = U_hat (Sec. 5.1) with the stop rule R5.

    Returns (U, info) where info holds the iteration count, the gap history
    and, when `record`, the per-iteration (g, q, alpha, E) lists.
    """
    U = P.Uhat.copy() if U0 is None else np.array(U0, dtype=np.float64)
    hist = dict(g=[], q=[], alpha=[], E=[], active=[])
    g0 = None
    iters = 0
    status = "max_iters"
    for k in range(max_iters + 1):
        it = gfw_iteration(U, P, oracle, step, with_energy)
        if g0 is None:
            g0 = it.g
        if record:
            hist["g"].append(it.g)
            hist["q"].append(it.q)
            hist["alpha"].append(it.alpha)
            hist["E"].append(it.E)
            hist["active"].append(int(it.active.sum()))
        thr = tol if tol_mode == "abs" else tol * g0
        if not it.active.any() or it.g <= 0.0:
            status = "stationary"
            break
        if it.g <= thr:
            status = "converged"
            break
        if k == max_iters:
            break
        U = U + it.alpha * it.D
        iters += 1
    return U, dict(iters=iters, status=status, g0=g0, g=it.g, hist=hist)


def osfw(P: Problem, oracle: str = "greedy", U0: Optional[np.ndarray] = None):
    """One-Shot Frank-Wolfe (Alg. 4): from U_0 (U_hat unless given), take the
    (G)LMO vertex of the gradient at U_0 as the result, U_1 = S_0.

    Returns (U1, s): the vertex and the chosen class per row (its labels)."""
    U = P.Uhat.copy() if U0 is None else np.array(U0, dtype=np.float64)
    G = gradient(U, P)
    if oracle == "greedy":
        S, s, _ = glmo(G, U)
    elif oracle == "full":
        S, s = lmo(G)
    else:
        raise ValueError(oracle)
    return S, s


def labels_from_U(U: np.ndarray) -> np.ndarray:
    """Class per row: argmax_k u_ik, lowest index on ties (R6)."""
    return np.argmax(U, axis=1).astype(np.int32)
