"""FP64 reference computations for finite discounted-cost MDPs (test infrastructure).

Plain numpy/scipy code that writes out the paper's definitions and algorithms in the
paper's order and notation; only the tests, the smoke check and the benchmark's CPU
baseline use it.  Library primitives used as single steps: matrix-vector products, a dense
LU solve with partial pivoting (numpy.linalg.solve, LAPACK gesv), a Householder QR
(numpy.linalg.qr, LAPACK geqrf) and a triangular solve.

Notation (paper Sec. 2): S states, A actions, p_{ss'}(a), stage cost g(s, a), discount
gamma, policy pi, P^pi, g^pi, Bellman operators T^pi and T, residual r(V) = V - TV,
Jacobian J^pi = I - gamma P^pi.  Indices are 0-based (the paper counts from 1).

Readings of the paper where it is silent (each marked "reading" below):
  * GreedyPolicy tie-break: lowest action index among exact minima.
  * Outer stop: at the top of outer iteration k, stop when ||Phi_k||_inf <= tol; return
    v = T(V_k), pi = GreedyPolicy(V_k), residual ||Phi_k||_inf.
  * Restart of GMRES(W): the new cycle starts from the current iterate (base x0 = V_{k+1},
    beta = ||g^pi - J^pi V_{k+1}||_2) and later iterates are x0 + Q y; the inner stop test
    keeps alpha * ||Phi_k||_inf from the start of the outer iteration.
  * Breakdown ("go to line 35"): leave the inner loop and go on to the next outer
    iteration; H[i+1, i] counts as zero when it is <= 1e-14 * ||J^pi Q_i||_2.
  * V_0 = 0.
  * OPI with W: W applications of T^{pi_k} per outer step, the first being the T V_k of
    the greedy step.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

BREAKDOWN_REL = 1e-14  # reading of "||q||_2 = 0" in floating point
_ROW_CHUNK = 1024      # rows of a dense P_a widened to FP64 at a time


@dataclass
class MDP:
    """Finite MDP {S, A, P, g, gamma} of paper Sec. 2.

    g[a, s] is g(s, a).  Dense storage: P[a, s, s'] = p_{ss'}(a).  ELL storage: row (a, s)
    holds the pairs (col[a, s, j], val[a, s, j]) and p_{ss'}(a) = sum of val over the j with
    col = s'.  mask[s, a] is True when a is in A(s) (None: every action allowed).
    """
    S: int
    A: int
    gamma: float
    g: np.ndarray
    kind: str
    P: np.ndarray | None = None
    col: np.ndarray | None = None
    val: np.ndarray | None = None
    mask: np.ndarray | None = None


def from_synth(m) -> MDP:
    """Build an oracle MDP from any object carrying the same field names."""
    return MDP(S=int(m.S), A=int(m.A), gamma=float(m.gamma), g=np.asarray(m.g, np.float64),
               kind=m.kind, P=m.P, col=m.col, val=m.val, mask=m.mask)


@dataclass
class Result:
    v: np.ndarray
    pi: np.ndarray
    residual: float
    status: str = "ok"
    outer: int = 0
    inner: int = 0
    restarts: int = 0
    sweeps: int = 0
    matvecs: int = 0
    history: list = field(default_factory=list)
    margin: np.ndarray | None = None


# --------------------------------------------------------------------------- operators

def transition_apply(mdp: MDP, a: int, v: np.ndarray) -> np.ndarray:
    """(P_a v)(s) = sum_{s'} p_{ss'}(a) v(s'), the expectation inside the Bellman
    equations (Sec. 2, Eqs. Bellman_eq_pi / Bellman_eq_star), in FP64."""
    v = np.asarray(v, np.float64)
    if mdp.kind == "dense":
        out = np.empty(mdp.S)
        for r0 in range(0, mdp.S, _ROW_CHUNK):
            r1 = min(mdp.S, r0 + _ROW_CHUNK)
            out[r0:r1] = mdp.P[a, r0:r1].astype(np.float64) @ v
        return out
    return (mdp.val[a].astype(np.float64) * v[mdp.col[a]]).sum(axis=1)


def q_values(mdp: MDP, v: np.ndarray) -> np.ndarray:
    """Q[a, s] = g(s, a) + gamma * sum_{s'} p_{ss'}(a) v(s') (the braces of the greedy
    policy definition, Sec. 2); +inf where a is not in A(s)."""
    Q = np.empty((mdp.A, mdp.S))
    for a in range(mdp.A):
        Q[a] = mdp.g[a] + mdp.gamma * transition_apply(mdp, a, v)
    if mdp.mask is not None:
        Q[~np.asarray(mdp.mask, bool).T] = np.inf
    return Q


def greedy_policy(Q: np.ndarray) -> np.ndarray:
    """GreedyPolicy (Sec. 2): pi(s) in argmin_a Q[a, s]; reading: lowest index on ties
    (numpy's argmin returns the first minimum)."""
    return np.argmin(Q, axis=0).astype(np.int32)


@dataclass
class Sweep:
    Q: np.ndarray
    pi: np.ndarray
    Tv: np.ndarray
    Phi: np.ndarray
    res_inf: float
    margin: np.ndarray


def bellman(mdp: MDP, v: np.ndarray) -> Sweep:
    """One Bellman sweep at v: the greedy policy, TV = min_pi {g^pi + gamma P^pi V}
    (Sec. 2), Phi = TV - v = -r(v) (Eq. Bellman_res) and ||Phi||_inf.  margin[s] is the gap
    between the two smallest Q[., s] (inf with one allowed action)."""
    v = np.asarray(v, np.float64)
    Q = q_values(mdp, v)
    pi = greedy_policy(Q)
    Tv = Q[pi, np.arange(mdp.S)]
    Phi = Tv - v
    if mdp.A >= 2:
        two = np.partition(Q, 1, axis=0)[:2]
        margin = two[1] - two[0]
        margin[~np.isfinite(margin)] = np.inf
    else:
        margin = np.full(mdp.S, np.inf)
    return Sweep(Q=Q, pi=pi, Tv=Tv, Phi=Phi, res_inf=float(np.max(np.abs(Phi))) if mdp.S else 0.0,
                 margin=margin)


def bellman_residual(mdp: MDP, v: np.ndarray) -> np.ndarray:
    """r(V) = V - TV (Eq. Bellman_res)."""
    return np.asarray(v, np.float64) - bellman(mdp, v).Tv


def policy_matrix(mdp: MDP, pi: np.ndarray):
    """[P^pi]_{ss'} = p_{ss'}(pi(s)) (Sec. 2): dense ndarray or CSR matrix, FP64."""
    pi = np.asarray(pi, np.int64)
    rows = np.arange(mdp.S)
    if mdp.kind == "dense":
        return mdp.P[pi, rows, :].astype(np.float64)
    k = mdp.col.shape[2]
    data = mdp.val[pi, rows, :].astype(np.float64).ravel()
    idx = mdp.col[pi, rows, :].astype(np.int64).ravel()
    ptr = np.arange(0, mdp.S * k + 1, k)
    return sp.csr_matrix((data, idx, ptr), shape=(mdp.S, mdp.S))


def policy_cost(mdp: MDP, pi: np.ndarray) -> np.ndarray:
    """g^pi = [g(1, pi(1)), ..., g(n, pi(n))]^T (Sec. 2)."""
    return mdp.g[np.asarray(pi, np.int64), np.arange(mdp.S)].astype(np.float64)


def jacobian(mdp: MDP, pi: np.ndarray):
    """J^pi = I - gamma P^pi (Sec. 2, Newtonian linear system Eq. Newtonian_linearsystem)."""
    Ppi = policy_matrix(mdp, pi)
    if sp.issparse(Ppi):
        return (sp.identity(mdp.S, format="csr") - mdp.gamma * Ppi).tocsr()
    J = -mdp.gamma * Ppi
    J[np.diag_indices(mdp.S)] += 1.0
    return J


def policy_evaluation(mdp: MDP, pi: np.ndarray) -> np.ndarray:
    """V^pi = (I - gamma P^pi)^{-1} g^pi (Sec. 2.1, PI's policy evaluation), by dense LU
    with partial pivoting."""
    J = jacobian(mdp, pi)
    if sp.issparse(J):
        J = J.toarray()
    return np.linalg.solve(J, policy_cost(mdp, pi))


# --------------------------------------------------------------------------- brute force

def brute_force(mdp: MDP, max_policies: int = 100000):
    """V*(s) = min over all deterministic stationary policies of V^pi(s) (Eq. optimal cost),
    by evaluating every policy with allowed actions.  Returns (V*, [(pi, V^pi), ...])."""
    allowed = [np.nonzero(mdp.mask[s])[0] if mdp.mask is not None else np.arange(mdp.A)
               for s in range(mdp.S)]
    total = int(np.prod([len(x) for x in allowed]))
    if total > max_policies:
        raise ValueError(f"{total} policies is too many to enumerate")
    table = []
    vstar = np.full(mdp.S, np.inf)
    for choice in itertools.product(*allowed):
        pi = np.array(choice, dtype=np.int32)
        vp = policy_evaluation(mdp, pi)
        table.append((pi, vp))
        vstar = np.minimum(vstar, vp)
    return vstar, table


# --------------------------------------------------------------------------- baselines

def value_iteration(mdp: MDP, v0=None, tol: float = 1e-8, max_iter: int = 100000) -> Result:
    """VI for the optimal cost, V_{k+1} = T V_k (Eq. VI_optimalcost); stops at the first k
    with ||T V_k - V_k||_inf <= tol and returns T V_k and GreedyPolicy(V_k)."""
    V = np.zeros(mdp.S) if v0 is None else np.array(v0, np.float64)
    hist = []
    for k in range(max_iter):
        b = bellman(mdp, V)
        hist.append(b.res_inf)
        if b.res_inf <= tol:
            return Result(b.Tv, b.pi, b.res_inf, "ok", outer=k, sweeps=k + 1, history=hist,
                          margin=b.margin)
        V = b.Tv
    b = bellman(mdp, V)
    return Result(b.Tv, b.pi, b.res_inf, "noconv", outer=max_iter, sweeps=max_iter + 1,
                  history=hist, margin=b.margin)


def policy_iteration(mdp: MDP, v0=None, tol: float = 1e-8, max_iter: int = 1000) -> Result:
    """PI (Sec. 2.1): pi_k = GreedyPolicy(V_k) (policy improvement), then exact policy
    evaluation V_{k+1} = (I - gamma P^{pi_k})^{-1} g^{pi_k}.  V_0 = 0, so pi_0 = GreedyPolicy(0).
    Stops when ||T V_k - V_k||_inf <= tol or when the policy repeats (then V_k = V^{pi_k}
    and pi_k is greedy for its own cost, hence optimal)."""
    V = np.zeros(mdp.S) if v0 is None else np.array(v0, np.float64)
    prev = None
    hist = []
    for k in range(max_iter):
        b = bellman(mdp, V)
        hist.append(b.res_inf)
        if b.res_inf <= tol or (prev is not None and np.array_equal(prev, b.pi)):
            return Result(b.Tv, b.pi, b.res_inf, "ok", outer=k, sweeps=k + 1, history=hist,
                          margin=b.margin)
        V = policy_evaluation(mdp, b.pi)
        prev = b.pi
    b = bellman(mdp, V)
    return Result(b.Tv, b.pi, b.res_inf, "noconv", outer=max_iter, history=hist,
                  margin=b.margin)


def optimistic_policy_iteration(mdp: MDP, W: int, v0=None, tol: float = 1e-8,
                                max_outer: int = 100000) -> Result:
    """OPI (Sec. 2.1): policy evaluation by W VI steps V <- T^{pi_k} V = g^{pi_k} +
    gamma P^{pi_k} V (Eq. VI_policyevaluation).  Reading: the first of the W steps is the
    T V_k computed with the greedy step."""
    V = np.zeros(mdp.S) if v0 is None else np.array(v0, np.float64)
    hist = []
    sweeps = 0
    matvecs = 0
    for k in range(max_outer):
        b = bellman(mdp, V)
        sweeps += 1
        hist.append(b.res_inf)
        if b.res_inf <= tol:
            return Result(b.Tv, b.pi, b.res_inf, "ok", outer=k, sweeps=sweeps,
                          matvecs=matvecs, history=hist, margin=b.margin)
        V = b.Tv
        Ppi = policy_matrix(mdp, b.pi)
        gpi = policy_cost(mdp, b.pi)
        for _ in range(W - 1):
            V = gpi + mdp.gamma * (Ppi @ V)
            matvecs += 1
    b = bellman(mdp, V)
    return Result(b.Tv, b.pi, b.res_inf, "noconv", outer=max_outer, sweeps=sweeps + 1,
                  matvecs=matvecs, history=hist, margin=b.margin)


# --------------------------------------------------------------------------- GMRES

def _lsq(H: np.ndarray, beta: float) -> np.ndarray:
    """y~ = argmin_y || beta e_1 - H y ||_2 for the (i+1) x i Hessenberg block H
    (Alg. 2, the least-squares step; Eq. GMRES_LSQ), by Householder QR."""
    rhs = np.zeros(H.shape[0])
    rhs[0] = beta
    Qh, Rh = np.linalg.qr(H, mode="reduced")
    return sla.solve_triangular(Rh, Qh.T @ rhs, lower=False)


@dataclass
class _InnerStats:
    steps: int = 0
    restarts: int = 0
    matvecs: int = 0
    breakdown: bool = False


def two_level(mdp: MDP, pi: np.ndarray, block: int):
    """Two-level preconditioner for J^pi = I - gamma P^pi (a preconditioned inner solver, the
    direction the paper names as future work in Sec. 5).  States are aggregated into consecutive
    blocks of `block` (the last one shorter); R averages a vector over each block, Pr copies a
    block value to its states (R Pr = I), and the coarse operator is the Galerkin product
    J_c = R J^pi Pr.  Returns (R, Pr, J_c, minv) with minv(q) = q + Pr J_c^{-1} R q."""
    J = jacobian(mdp, pi)
    S = mdp.S
    agg = np.arange(S) // block
    nc = int(agg[-1]) + 1
    Pr = sp.csr_matrix((np.ones(S), (np.arange(S), agg)), shape=(S, nc))
    sizes = np.bincount(agg, minlength=nc).astype(np.float64)
    R = sp.diags(1.0 / sizes) @ Pr.T.tocsr()
    JPr = J @ Pr
    Jc = np.asarray((R @ JPr).todense() if sp.issparse(JPr) else R @ JPr)
    lu = sla.lu_factor(Jc)

    def minv(q):
        return q + Pr @ sla.lu_solve(lu, R @ q)
    return R, Pr, Jc, minv


def _gmres_inner(J, g_pi: np.ndarray, V_k: np.ndarray, Phi_k: np.ndarray, threshold: float,
                 W: int, max_steps: int, st: _InnerStats, minv=None) -> np.ndarray:
    """The inner loop of Alg. 2 (GMRES(W) on J^pi V = g^pi started at V_k), run while
    ||g^pi - J^pi V_{k+1}||_inf > threshold.  Arnoldi with modified Gram-Schmidt; the true
    residual is formed at every test, as the while-condition of Alg. 2 states.  With minv
    (a preconditioner M^{-1}) the Arnoldi process runs on J M^{-1} (right preconditioning) and
    the iterate is base + M^{-1} Q y, so residuals keep their meaning."""
    mv = (lambda x: x) if minv is None else minv
    n = V_k.shape[0]
    V_next = V_k.copy()                       # V_{k+1} <- V_k
    x0 = V_k.copy()                           # base of the current cycle (reading)
    beta = float(np.linalg.norm(Phi_k))
    Q = np.zeros((n, W + 1))                  # Q <- 0_{n x (W+1)}
    H = np.zeros((W + 1, W))                  # H <- 0_{(W+1) x W}
    if beta == 0.0:
        return V_next
    Q[:, 0] = Phi_k / beta                    # [Q]_1 <- Phi_k / ||Phi_k||_2
    i = 1
    while True:
        r_true = g_pi - J @ V_next            # while-condition: true residual, inf-norm
        st.matvecs += 1
        if not (np.max(np.abs(r_true)) > threshold) or st.steps >= max_steps:
            return V_next
        q = J @ mv(Q[:, i - 1])               # q <- J^pi [Q]_i  (J^pi M^{-1} [Q]_i)
        st.matvecs += 1
        qnorm0 = float(np.linalg.norm(q))
        for j in range(1, i + 1):             # modified Gram-Schmidt
            H[j - 1, i - 1] = Q[:, j - 1] @ q
            q = q - H[j - 1, i - 1] * Q[:, j - 1]
        H[i, i - 1] = np.linalg.norm(q)       # [H]_{i+1,i} <- ||q||_2
        st.steps += 1
        if H[i, i - 1] <= BREAKDOWN_REL * qnorm0:   # ||q||_2 = 0: lucky breakdown
            y = _lsq(H[: i + 1, :i], beta)
            st.breakdown = True
            return mv(Q[:, :i] @ y) + x0
        Q[:, i] = q / H[i, i - 1]             # [Q]_{i+1} <- q / [H]_{i+1,i}
        y = _lsq(H[: i + 1, :i], beta)        # y~ <- argmin || ||Phi||_2 e_1 - H y ||_2
        V_next = mv(Q[:, :i] @ y) + x0        # V_{k+1} <- Q y~ + base  (M^{-1} Q y~)
        if i == W:                            # restart
            x0 = V_next.copy()
            r = g_pi - J @ V_next
            st.matvecs += 1
            beta = float(np.linalg.norm(r))
            Q = np.zeros((n, W + 1))
            H = np.zeros((W + 1, W))
            st.restarts += 1
            if beta == 0.0:
                return V_next
            Q[:, 0] = r / beta
            i = 1
        else:
            i += 1


def policy_eval_gmres(mdp: MDP, pi: np.ndarray, v0=None, target_inf: float = 1e-10,
                      W: int = 30, max_steps: int = 100000, precond_block: int = 0) -> Result:
    """Inexact policy evaluation alone: GMRES(W) on (I - gamma P^pi) V = g^pi started at v0
    until ||g^pi - (I - gamma P^pi) V||_inf <= target_inf (Alg. 2's inner loop with an
    absolute threshold)."""
    V0 = np.zeros(mdp.S) if v0 is None else np.array(v0, np.float64)
    J = jacobian(mdp, pi)
    g_pi = policy_cost(mdp, pi)
    Phi = g_pi - J @ V0
    st = _InnerStats()
    minv = two_level(mdp, pi, precond_block)[3] if precond_block > 0 else None
    V = _gmres_inner(J, g_pi, V0, Phi, target_inf, W, max_steps, st, minv)
    res = float(np.max(np.abs(g_pi - J @ V))) if mdp.S else 0.0
    return Result(V, np.asarray(pi, np.int32), res, "ok" if res <= target_inf else "noconv",
                  inner=st.steps, restarts=st.restarts, matvecs=st.matvecs + 2)


def inner_threshold(alpha: float, forcing_c: float, phi_inf: float, tol: float) -> float:
    """Right-hand side of the inexact stopping rule (Sec. 3), alpha_k ||Phi_k||_inf.

    forcing_c = 0: the constant alpha of Alg. 2.  forcing_c > 0: the forcing sequence
    alpha_k = min(alpha, forcing_c * ||Phi_k||_inf), which lies in [0, alpha] and tends to 0
    with the residual, so the local convergence theorem of Sec. 3 gives Q-superlinear
    convergence; the threshold is then kept at or above tol / 10 (reading: an inner solve
    more accurate than the outer tolerance cannot change the outcome, and below that the
    arithmetic's floor would stall it)."""
    if forcing_c > 0.0:
        return max(min(alpha, forcing_c * phi_inf) * phi_inf, 0.1 * tol)
    return alpha * phi_inf


def inexact_pi_vi(mdp: MDP, v0=None, alpha: float = 0.1, tol: float = 1e-8, K: int = 100,
                  max_inner: int = 100000, forcing_c: float = 0.0) -> Result:
    """Inexact Policy Iteration (Alg. 1) with VI as the inner solver (Sec. 3: OPI whose number
    of inner steps is set by the stopping rule).

    for k = 0..K-1: pi_k <- GreedyPolicy(V_k); Phi_k = g^{pi_k} - J^{pi_k} V_k (= T V_k - V_k);
    (reading: stop if ||Phi_k||_inf <= tol); W <- V_k; repeat W <- T^{pi_k} W = g^{pi_k} +
    gamma P^{pi_k} W while ||g^{pi_k} - J^{pi_k} W||_inf > alpha_k ||Phi_k||_inf; V_{k+1} <- W.
    The first inner step is taken unconditionally (the residual at V_k is Phi_k itself).
    """
    V = np.zeros(mdp.S) if v0 is None else np.array(v0, np.float64)
    res = Result(V, np.zeros(mdp.S, np.int32), np.inf)
    for k in range(K):
        b = bellman(mdp, V)                     # pi_k <- GreedyPolicy(V_k), T V_k
        res.sweeps += 1
        pi_k = b.pi
        phi_inf = b.res_inf                     # ||g^{pi_k} - J^{pi_k} V_k||_inf
        res.history.append(phi_inf)
        if phi_inf <= tol:
            res.v, res.pi, res.residual, res.outer = b.Tv, pi_k, phi_inf, k
            res.margin = b.margin
            return res
        thr = inner_threshold(alpha, forcing_c, phi_inf, tol)
        g_pi = policy_cost(mdp, pi_k)
        P_pi = policy_matrix(mdp, pi_k)
        W = b.Tv                                # first step: T^{pi_k} V_k = T V_k
        steps = 1
        while steps < max_inner:
            TW = g_pi + mdp.gamma * (P_pi @ W)  # T^{pi_k} W
            res.matvecs += 1
            if float(np.max(np.abs(TW - W))) <= thr:
                break
            W = TW
            steps += 1
        res.inner += steps
        V = W
    b = bellman(mdp, V)
    res.sweeps += 1
    res.v, res.pi, res.residual, res.outer, res.status = b.Tv, b.pi, b.res_inf, K, "noconv"
    res.margin = b.margin
    return res


def gmres_policy_iteration(mdp: MDP, v0=None, alpha: float = 0.1, W: int = 30,
                           tol: float = 1e-8, K: int = 100,
                           max_inner: int = 100000, forcing_c: float = 0.0,
                           precond_block: int = 0) -> Result:
    """GMRES(W) Policy Iteration, Alg. 2, step by step.

    for k = 0..K-1: pi_k <- GreedyPolicy(V_k); J <- I - gamma P^{pi_k}; V_{k+1} <- V_k;
    Phi_k <- g^{pi_k} - J V_k; (reading: stop here if ||Phi_k||_inf <= tol); run GMRES(W)
    from V_k while ||g^{pi_k} - J V_{k+1}||_inf > alpha_k ||Phi_k||_inf (inner_threshold:
    alpha_k = alpha unless forcing_c > 0).
    """
    V = np.zeros(mdp.S) if v0 is None else np.array(v0, np.float64)
    res = Result(V, np.zeros(mdp.S, np.int32), np.inf)
    for k in range(K):
        b = bellman(mdp, V)                   # pi_k <- GreedyPolicy(V_k)
        res.sweeps += 1
        pi_k = b.pi
        J = jacobian(mdp, pi_k)               # J^{pi_k} <- I - gamma P^{pi_k}
        g_pi = policy_cost(mdp, pi_k)
        Phi_k = g_pi - J @ V                  # Phi_k <- g^{pi_k} - J^{pi_k} V_k
        phi_inf = float(np.max(np.abs(Phi_k))) if mdp.S else 0.0
        res.history.append(phi_inf)
        if phi_inf <= tol:                    # reading: outer stop test
            res.v, res.pi, res.residual, res.outer = b.Tv, pi_k, phi_inf, k
            res.margin = b.margin
            return res
        st = _InnerStats()
        minv = two_level(mdp, pi_k, precond_block)[3] if precond_block > 0 else None
        V = _gmres_inner(J, g_pi, V, Phi_k, inner_threshold(alpha, forcing_c, phi_inf, tol),
                         W, max_inner, st, minv)
        res.inner += st.steps
        res.restarts += st.restarts
        res.matvecs += st.matvecs + 1
    b = bellman(mdp, V)
    res.sweeps += 1
    res.v, res.pi, res.residual, res.outer, res.status = b.Tv, b.pi, b.res_inf, K, "noconv"
    res.margin = b.margin
    return res
