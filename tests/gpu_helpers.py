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


def lockstep(g, iters, weights="f32", eps=50.0, omega0=1000.0, oracle="greedy",
             step="exact", laplacian="sym", tol=TOL, every=1, energy=True, **opts):
    """Run up to `iters` GPU iterations; at every `every`-th one feed the GPU
    iterate U_k to the oracle and compare G' (relative inf-norm), the (G)LMO
    choice (bit-exact, on the GPU's own G'), g_k, q_k, alpha_k and E(U_k).
    Returns the per-check records."""
    P = O.make_problem(g, eps, omega0, weights, laplacian)
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
            gerr = np.max(np.abs(Gp - Gp_o)) / max(np.max(np.abs(Gp_o)), 1e-30)
            assert gerr <= tol, (k, gerr)
            rec = dict(k=k, gerr=gerr, g=(None, g_o), active=int(act.sum()))
            if energy:
                E_g = s.objective()
                E_o = O.energy(U, P)
                assert rel(E_g, E_o) <= tol, (k, E_g, E_o)
                rec["E"] = (E_g, E_o)
            st = s.step(1)
            rec["g"] = (st.gap, g_o)
            # the GPU's gap reduction against an FP64 sum over its own G' and U ...
            g_own = O.fw_gap(Gp, U, ch, act)
            assert rel(st.gap, g_own, 1e-9 * max(1.0, st.gap0)) <= tol, (k, st.gap, g_own)
            # ... and against the oracle's FP64 gradient: g is a sum of differences
            # G'_k - G'_s, so its relative accuracy is bounded by that of G' (checked
            # above at `tol`) times sum u|G'| / g; 10x tol covers the observed range
            assert rel(st.gap, g_o, 1e-9 * max(1.0, st.gap0)) <= 10 * tol, (k, st.gap, g_o)
            if st.iters == k + 1:   # an update was applied: compare the step
                assert rel(st.q, q_o, 1e-3 * nD) <= tol, (k, st.q, q_o)
                # the step is the exact rule applied to the GPU's own g and q ...
                if step == "exact":
                    a_own = 1.0 if st.q <= 0 else min(1.0, st.gap / st.q)
                    assert rel(st.alpha, a_own) <= 1e-12, (k, st.alpha, a_own)
                # ... and inherits their accuracy against the oracle
                assert rel(st.alpha, a_o) <= 10 * tol, (k, st.alpha, a_o)
                rec.update(q=(st.q, q_o), alpha=(st.alpha, a_o))
            recs.append(rec)
            if st.status != B.FW_PENDING:
                break
    return recs


def agreement(a, b):
    return float(np.mean(np.asarray(a) == np.asarray(b)))
