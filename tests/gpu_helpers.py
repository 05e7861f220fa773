"""Helpers of the GPU parity tests: lockstep comparison with the FP64 oracle."""
import numpy as np

import oracle as O
from paper_2508_09738_gb300 import binding as B

TOL = 1e-5   # relative agreement of gradients, gap, curvature, step and objective


def rel(a, b, floor=1e-30):
    return abs(a - b) / max(abs(b), floor)


def oracle_at(U, Gp, ch, act, P, step="exact"):
    """Oracle quantities at the GPU iterate U with the GPU's (verified) choice."""
    G = O.gradient(U, P)
    S = U.copy()
    S[act] = 0.0
    S[np.flatnonzero(act), ch[act]] = 1.0
    D = S - U
    g_o = O.fw_gap(G, U, ch, act)
    q_o = O.curvature(D, P)
    if g_o > 0:
        a_o = O.exact_step(g_o, q_o) if step == "exact" else O.armijo_step(U, D, g_o, P)
    else:
        a_o = 0.0
    return G, g_o, q_o, a_o, float(np.sum(D * D))


TOL_RED = 1e-6   # the GPU's g and q against FP64 sums over its own G', U and L S


def lockstep(g, iters, weights="f32", eps=50.0, omega0=1000.0, oracle="greedy",
             step="exact", laplacian="sym", tol=TOL, every=1, energy=True, **opts):
    """Run up to `iters` GPU iterations; at every `every`-th one feed the GPU
    iterate U_k to the oracle and compare G' (relative inf-norm), the (G)LMO
    choice (bit-exact, on the GPU's own G'), g_k, q_k, alpha_k and E(U_k).

    g and q are compared twice.  (1) The GPU's reductions against FP64 sums
    over its own G', U and the oracle's L S at the GPU's choice: TOL_RED (the
    reductions themselves).  (2) Against the oracle's FP64 values: `tol`, or
    the bound the measured gradient difference implies, whichever is larger.
    g = sum_{i in I} sum_k u_ik (G'_ik - G'_is) differs from the oracle's by at
    most 2 |I| ||dG'||_inf, and q's <D, L U> term by at most 2 |I| ||dLU||_inf
    (||D_i||_1 <= 2), with ||dLU||_inf = ||dG'||_inf (U is shared); so
    rel(g) <= 2 |I| gerr ||G'||_inf / g and rel(q) <= 2 |I| gerr ||G'||_inf / |q|,
    and rel(alpha) <= rel(g) + rel(q).  Returns the per-check records."""
    P = O.make_problem(g, eps, omega0, weights, laplacian)
    red = min(TOL_RED, tol)
    recs = []
    with B.Segmenter(g, eps=eps, omega0=omega0, weight_dtype=weights, oracle=oracle,
                     step_rule=step, laplacian=laplacian, max_iters=10 ** 7, **opts) as s:
        for k in range(iters):
            if k % every:
                if s.step(1).status != B.FW_PENDING:
                    break
                continue
            U = s.U()
            Gp, ch, act = s.grad()
            # bit-exact (G)LMO on the GPU's own gradient values
            if oracle == "greedy":
                _, s_o, act_o = O.glmo(Gp, U)
            else:
                _, s_o = O.lmo(Gp)
                binary = np.all((U == 0) | (U == 1), axis=1)
                act_o = ~(binary & (U[np.arange(g.n), s_o] == 1.0))
            assert np.array_equal(s_o, ch), (k, np.flatnonzero(s_o != ch)[:10])
            assert np.array_equal(act_o, act), k
            G, g_o, q_o, a_o, nD = oracle_at(U, Gp, ch, act, P, step)
            Gp_o = G - P.inv_eps
            gnorm = max(np.max(np.abs(Gp_o)), 1e-30)
            gerr = np.max(np.abs(Gp - Gp_o)) / gnorm
            assert gerr <= tol, (k, gerr)
            rec = dict(k=k, gerr=gerr, g=(None, g_o), active=int(act.sum()))
            if energy:
                E_g = s.objective()
                E_o = O.energy(U, P)
                assert rel(E_g, E_o) <= tol, (k, E_g, E_o)
                rec["E"] = (E_g, E_o)
            st = s.step(1)
            rec["g"] = (st.gap, g_o)
            spread = 2.0 * act.sum() * gerr * gnorm
            # (1) the GPU's gap reduction against an FP64 sum over its own G' and U
            g_own = O.fw_gap(Gp, U, ch, act)
            floor = 1e-12 * max(1.0, st.gap0)
            assert rel(st.gap, g_own, floor) <= red, (k, st.gap, g_own)
            # (2) against the oracle's FP64 gradient
            bound_g = max(tol, red + spread / max(g_o, floor))
            rec["rel_g"] = (rel(st.gap, g_o, floor), bound_g)
            assert rec["rel_g"][0] <= bound_g, (k, st.gap, g_o, bound_g)
            if st.iters == k + 1:   # an update was applied: compare the step
                qfl = 1e-6 * nD
                if step == "exact":
                    # the step is the exact rule applied to the GPU's own g and q
                    a_own = 1.0 if st.q <= 0 else min(1.0, st.gap / st.q)
                    assert rel(st.alpha, a_own) <= 1e-12, (k, st.alpha, a_own)
                bound_q = max(tol, red + spread / max(abs(q_o), qfl))
                rec["rel_q"] = (rel(st.q, q_o, qfl), bound_q)
                assert rec["rel_q"][0] <= bound_q, (k, st.q, q_o, bound_q)
                # alpha = min(1, g / q): its error is at most that of g plus q
                bound_a = max(tol, bound_g + bound_q) if 0 < a_o < 1 else tol
                rec["rel_alpha"] = (rel(st.alpha, a_o), bound_a)
                if step == "exact":
                    assert rec["rel_alpha"][0] <= bound_a, (k, st.alpha, a_o, bound_a)
                else:
                    # Armijo halves until a threshold: a step of the other side of
                    # a power of two is allowed when g/q sits within the bounds
                    assert st.alpha == a_o or abs(np.log2(st.alpha / a_o)) == 1, (k, st.alpha, a_o)
                rec.update(q=(st.q, q_o), alpha=(st.alpha, a_o))
            recs.append(rec)
            if st.status != B.FW_PENDING:
                break
    return recs


def agreement(a, b):
    return float(np.mean(np.asarray(a) == np.asarray(b)))
