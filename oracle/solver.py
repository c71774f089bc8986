"""Line search, fixed-point map and the NGMRES family (Sec. 2.3, Algorithms 1-3).

Test infrastructure only (see oracle/__init__.py).

The accelerators are written against two callables so that the same code runs on the
transport problems and on the linear test problems of the pins:
    evaluate(v) -> (g, obj)             the reduced gradient g(v) (Eq. (3)) and obj(v)
    qmap(v, g, obj) -> (q, obj_q)       one step of the fixed-point map (Eq. (10))

Readings:
* Armijo line search (Eqs. (6)-(7)): accept rho when obj(v + rho s) < obj(v) + c rho <g, s>
  with c = 1e-4 and the L2 inner product; start from the remembered rho (1 at the first
  iteration), halve until accepted; the remembered value becomes 2 rho when the first trial
  was accepted, else the accepted rho. The paper gives no limit on the number of halvings;
  after max_backtracks halvings without acceptance the search fails (LineSearchError).
* Window (Alg. 1-3): v^{(k-i)} and g(v^{(k-i)}), i = 0..min(k, w), are the last iterates of
  the main sequence, fixed-point steps included.
* NGMRES least squares (Alg. 1 line "arg min"): plain l2 norm, solved here with
  numpy.linalg.lstsq on the explicit difference matrix with rcond = 1e-7 (the paper does not
  say how rank deficiency is treated).
* Iteration cap: the loop runs at most n_iter iterations (k = 0 .. n_iter-1).
* Mixing switch (Alg. 3): variant 1 (GA-NGMRES(w; sigma, tau)) takes a fixed-point step
  when mod(k, sigma + tau) >= sigma; variant 2 (aNGMRES(w)[sigma]-FP[tau], Sec. 3.3) when
  mod(k, sigma + tau) < tau.
"""
from __future__ import annotations

from collections import deque

import numpy as np


class LineSearchError(RuntimeError):
    pass


class ArmijoQ:
    """The fixed-point map q(v) = v + rho s, s = -(alpha L)^{-1} g(v) (Eqs. (9)-(10)),
    with the Armijo backtracking and step-size memory of Sec. 2.3."""

    def __init__(self, problem, c=1e-4, max_backtracks=20):
        self.p = problem
        self.c = c
        self.max_backtracks = max_backtracks
        self.rho_mem = 1.0
        self.trials = 0
        self.last_rho = None

    def __call__(self, v, g, obj):
        s = self.p.precond(g)
        gs = self.p.inner(g, s)
        rho = self.rho_mem
        for it in range(self.max_backtracks + 1):
            vt = v + rho * s
            ot = self.p.objective(vt)
            self.trials += 1
            if ot < obj + self.c * rho * gs:
                self.rho_mem = 2.0 * rho if it == 0 else rho
                self.last_rho = rho
                return vt, ot
            rho *= 0.5
        raise LineSearchError(f"Armijo condition not met after {self.max_backtracks} halvings")


def _is_fp_step(k, sigma, tau, variant):
    if variant == 1:
        return (k % (sigma + tau)) >= sigma
    return (k % (sigma + tau)) < tau


def ngmres_lsq(gq, gwin, rcond=1e-7):
    """beta = argmin || g_q + sum_i beta_i (g_q - g_i) ||_2 over the window gradients gwin[i]."""
    D = np.stack([(gq - gi).ravel() for gi in gwin], axis=1)
    beta, *_ = np.linalg.lstsq(D, -gq.ravel(), rcond=rcond)
    return beta


def ga_ngmres(evaluate, qmap, v0, window, sigma=1, tau=0, n_iter=200, rel_tol=1e-2,
              variant=1, rcond=1e-7, history=None):
    """GA-NGMRES(w; sigma, tau), Algorithm 3 (tau = 0 gives NGMRES(w), Algorithm 1).

    Returns (v, info) with info = dict(iters, grad_evals, rel_grad, obj, converged).
    history, if a list, receives per-iteration dicts (k, branch, rel_grad, obj, beta).
    """
    v = np.array(v0, dtype=np.float64)
    g, obj = evaluate(v)
    nge = 1
    g0 = float(np.abs(g).max())
    V = deque([v], maxlen=window + 1)
    G = deque([g], maxlen=window + 1)
    k = 0
    rel = float(np.abs(g).max()) / g0 if g0 > 0 else 0.0
    converged = rel <= rel_tol
    while not converged and k < n_iter:
        wk = min(k, window)
        qv, _ = qmap(v, g, obj)
        gq, oq = evaluate(qv)
        nge += 1
        fp = _is_fp_step(k, sigma, tau, variant)
        beta = None
        if fp:
            v, g, obj = qv, gq, oq
        else:
            gwin = [G[-1 - i] for i in range(wk + 1)]
            beta = ngmres_lsq(gq, gwin, rcond)
            vn = qv.copy()
            for i in range(wk + 1):
                vn += beta[i] * (qv - V[-1 - i])
            v = vn
            g, obj = evaluate(v)
            nge += 1
        V.append(v)
        G.append(g)
        rel = float(np.abs(g).max()) / g0 if g0 > 0 else 0.0
        converged = rel <= rel_tol
        if history is not None:
            history.append(dict(k=k, branch="fp" if fp else "ngmres", rel_grad=rel, obj=obj,
                                beta=None if beta is None else beta.copy(), v=v.copy()))
        k += 1
    return v, dict(iters=k, grad_evals=nge, rel_grad=rel, obj=obj, converged=converged)


def ga_aa(evaluate, qmap, v0, window, sigma=1, tau=0, n_iter=200, rel_tol=1e-2,
          variant=1, rcond=1e-7, history=None):
    """GA-AA(w; sigma, tau): Anderson acceleration AA(w) (Algorithm 2) with the mixing of
    Algorithm 3. r(v) = v - q(v); xi = argmin ||r_k + sum_{i>=1} xi_i (r_k - r_{k-i})||;
    v_{k+1} = q_k + sum_{i>=1} xi_i (q_k - q_{k-i})."""
    v = np.array(v0, dtype=np.float64)
    g, obj = evaluate(v)
    nge = 1
    g0 = float(np.abs(g).max())
    Q = deque(maxlen=window + 1)
    R = deque(maxlen=window + 1)
    k = 0
    rel = 1.0
    converged = g0 == 0.0
    while not converged and k < n_iter:
        wk = min(k, window)
        qv, _ = qmap(v, g, obj)
        Q.append(qv)
        R.append(v - qv)
        fp = _is_fp_step(k, sigma, tau, variant) or wk == 0
        if fp:
            vn = qv
        else:
            rk = R[-1]
            D = np.stack([(rk - R[-1 - i]).ravel() for i in range(1, wk + 1)], axis=1)
            xi, *_ = np.linalg.lstsq(D, -rk.ravel(), rcond=rcond)
            vn = qv.copy()
            for i in range(1, wk + 1):
                vn += xi[i - 1] * (qv - Q[-1 - i])
        v = vn
        g, obj = evaluate(v)
        nge += 1
        rel = float(np.abs(g).max()) / g0
        converged = rel <= rel_tol
        if history is not None:
            history.append(dict(k=k, branch="fp" if fp else "aa", rel_grad=rel, obj=obj, v=v.copy()))
        k += 1
    return v, dict(iters=k, grad_evals=nge, rel_grad=rel, obj=obj, converged=converged)


def rpgd(evaluate, qmap, v0, n_iter=200, rel_tol=1e-2, history=None):
    """Regularisation-preconditioned gradient descent (Eq. (9)): v_{k+1} = q(v_k)."""
    v = np.array(v0, dtype=np.float64)
    g, obj = evaluate(v)
    g0 = float(np.abs(g).max())
    k, rel = 0, 1.0
    converged = g0 == 0.0
    while not converged and k < n_iter:
        v, _ = qmap(v, g, obj)
        g, obj = evaluate(v)
        rel = float(np.abs(g).max()) / g0
        converged = rel <= rel_tol
        if history is not None:
            history.append(dict(k=k, branch="fp", rel_grad=rel, obj=obj, v=v.copy()))
        k += 1
    return v, dict(iters=k, grad_evals=k + 1, rel_grad=rel, obj=obj, converged=converged)


def solve_problem(problem, window, sigma, tau, n_iter=200, rel_tol=1e-2, variant=1,
                  method="ga-ngmres", c=1e-4, max_backtracks=20, history=None):
    """Alg. 3 (or RPGD / GA-AA) on a transport Problem with v^{(0)} = 0."""
    q = ArmijoQ(problem, c=c, max_backtracks=max_backtracks)
    v0 = np.zeros((problem.d,) + problem.n)
    if method == "rpgd":
        v, info = rpgd(problem.gradient, q, v0, n_iter, rel_tol, history)
    elif method == "ga-aa":
        v, info = ga_aa(problem.gradient, q, v0, window, sigma, tau, n_iter, rel_tol, variant,
                        history=history)
    else:
        v, info = ga_ngmres(problem.gradient, q, v0, window, sigma, tau, n_iter, rel_tol,
                            variant, history=history)
    info.update(obj_evals=problem.counts["obj"], line_search_trials=q.trials, rho_mem=q.rho_mem)
    return v, info


# ---------------------------------------------------------------------------
# Linear test problems for the equivalence pins (Sec. 2.3.2)
# ---------------------------------------------------------------------------

class LinearProblem:
    """g(x) = A x - b with the Richardson fixed-point map q(x) = x - rho g(x)."""

    def __init__(self, A, b, rho):
        self.A = np.asarray(A, dtype=np.float64)
        self.b = np.asarray(b, dtype=np.float64)
        self.rho = float(rho)

    def evaluate(self, x):
        return self.A @ x - self.b, None

    def qmap(self, x, g, obj):
        return x - self.rho * g, None


def gmres_iterate(A, b, x0, m):
    """x_m = argmin_{x in x0 + K_m(A, r0)} ||b - A x||_2 by a dense Arnoldi basis + lstsq."""
    r0 = b - A @ x0
    if m == 0 or np.linalg.norm(r0) == 0.0:
        return x0.copy()
    nrm = np.linalg.norm(r0)
    Q = [r0 / nrm]
    for _ in range(1, m):
        w = A @ Q[-1]
        for qv in Q:
            w = w - (qv @ w) * qv
        for qv in Q:
            w = w - (qv @ w) * qv
        nw = np.linalg.norm(w)
        if nw < 1e-14 * nrm:
            break
        Q.append(w / nw)
    Qm = np.stack(Q, axis=1)
    y, *_ = np.linalg.lstsq(A @ Qm, r0, rcond=None)
    return x0 + Qm @ y


def restarted_gmres_iterates(A, b, x0, m, steps):
    """Iterates of restarted GMRES(m) after 0..steps total inner steps."""
    out = [x0.copy()]
    xs = x0.copy()
    done = 0
    while done < steps:
        for j in range(1, m + 1):
            if done + j > steps:
                break
            out.append(gmres_iterate(A, b, xs, j))
        done += m
        xs = out[min(done, len(out) - 1)] if done <= steps else xs
    return out[: steps + 1]
