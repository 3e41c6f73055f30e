"""Seeded synthetic MDP generators.

This module is the one source of inputs that both the CPU oracle checks and the GPU path
read.  It holds random problem data only (transition rows, stage costs, discount factors,
request traces); none of the method's arithmetic (no Bellman operator, no policy, no solve)
lives here.

Problem statement (paper Sec. 2): a finite MDP {S, A, P, g, gamma} with states 0..S-1,
actions 0..A-1 (0-based here; the paper counts from 1), row-stochastic transition rows
p_{ss'}(a) and bounded costs g(s, a).

Returned layouts (host numpy arrays):
  * dense:  P[a, s, s']            (A, S, S)   float32 or float64
  * ELL:    col[a, s, j], val[a, s, j]   (A, S, k)  int32 / float32|float64
  * costs:  g[a, s]                (A, S)      float64
  * mask:   mask[s, a]             (S, A)      bool (True = action allowed) or None

Every generator is deterministic in its seed and independent of the thread count: the work
is split into fixed blocks, each drawing from its own child of numpy's SeedSequence.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "SynthMDP", "ell_uniform", "dense_dirichlet", "ell_banded", "tiny_random",
    "batch_specs", "serving_trace", "config", "CONFIG_SEEDS",
]

# seed = 1000 + config number, one per workload
CONFIG_SEEDS = {1: 1001, 2: 1002, 3: 1003, 4: 1004, 5: 1005}

_BLOCK_ROWS = 8192  # rows per independently seeded block


@dataclass
class SynthMDP:
    """A finite discounted-cost MDP as plain arrays (see module docstring for layouts)."""
    S: int
    A: int
    gamma: float
    g: np.ndarray
    kind: str                     # "dense" or "ell"
    P: np.ndarray | None = None   # dense (A, S, S)
    col: np.ndarray | None = None  # ELL (A, S, k) int32
    val: np.ndarray | None = None  # ELL (A, S, k)
    mask: np.ndarray | None = None  # (S, A) bool
    meta: dict = field(default_factory=dict)

    @property
    def k(self) -> int:
        return 0 if self.col is None else int(self.col.shape[2])

    def nbytes(self) -> int:
        n = self.g.nbytes
        for x in (self.P, self.col, self.val, self.mask):
            if x is not None:
                n += x.nbytes
        return n


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _blocks(S: int):
    return [(b0, min(S, b0 + _BLOCK_ROWS)) for b0 in range(0, S, _BLOCK_ROWS)]


def _run_blocks(fn, jobs):
    with ThreadPoolExecutor(max_workers=_threads()) as ex:
        list(ex.map(lambda j: fn(*j), jobs))


def _distinct_columns(rng: np.random.Generator, lo: np.ndarray, width: int, k: int) -> np.ndarray:
    """For each row r draw k distinct integers uniformly from [lo[r], lo[r] + width).

    Sampling with replacement, then redrawing every row that holds a repeat, leaves each
    accepted row uniform over the k-subsets (rejection sampling).  When k > width / 4 the
    acceptance rate collapses, so such rows take the first k entries of a uniformly random
    permutation instead (also uniform over the k-subsets).
    """
    n = lo.shape[0]
    if 4 * k > width:
        # dense rows: rejection would rarely accept; take the first k of a random order
        return np.argsort(rng.random((n, width)), axis=1)[:, :k].astype(np.int64) + lo[:, None]
    out = np.empty((n, k), dtype=np.int64)
    todo = np.arange(n)
    while todo.size:
        draw = rng.integers(0, width, size=(todo.size, k))
        srt = np.sort(draw, axis=1)
        ok = np.all(srt[:, 1:] != srt[:, :-1], axis=1) if k > 1 else np.ones(todo.size, bool)
        out[todo[ok]] = draw[ok]
        todo = todo[~ok]
    return out + lo[:, None]


def ell_uniform(S: int, A: int, k: int, gamma: float, seed: int,
                val_dtype=np.float64) -> SynthMDP:
    """ELL MDP: per (a, s) k distinct columns uniform over all states, weights U(0,1)
    normalised to row sum 1 in FP64 then stored as val_dtype; costs g ~ U(0,1)."""
    if not (1 <= k <= S):
        raise ValueError("need 1 <= k <= S")
    col = np.empty((A, S, k), dtype=np.int32)
    val = np.empty((A, S, k), dtype=val_dtype)
    root = np.random.SeedSequence(seed)
    kids = root.spawn(A * len(_blocks(S)) + 1)
    jobs = []
    for a in range(A):
        for bi, (b0, b1) in enumerate(_blocks(S)):
            jobs.append((a, b0, b1, kids[a * len(_blocks(S)) + bi]))

    def work(a, b0, b1, ss):
        rng = _rng(ss)
        n = b1 - b0
        if k == S:
            c = np.tile(np.arange(S), (n, 1))
            c = rng.permuted(c, axis=1)
        else:
            c = _distinct_columns(rng, np.zeros(n, np.int64), S, k)
        w = rng.random((n, k))
        w /= w.sum(axis=1, keepdims=True)
        col[a, b0:b1] = c
        val[a, b0:b1] = w.astype(val_dtype)

    _run_blocks(work, jobs)
    g = _rng(kids[-1]).random((A, S))
    return SynthMDP(S=S, A=A, gamma=float(gamma), g=g, kind="ell", col=col, val=val,
                    meta=dict(recipe="ell_uniform", seed=seed))


def dense_dirichlet(S: int, A: int, conc: float, gamma: float, seed: int,
                    dtype=np.float32) -> SynthMDP:
    """Dense MDP: each row p_{s.}(a) ~ Dirichlet(conc) (Gamma(conc) draws normalised in
    FP64, then cast to dtype); costs g ~ U(0,1)."""
    P = np.empty((A, S, S), dtype=dtype)
    root = np.random.SeedSequence(seed)
    blocks = [(b0, min(S, b0 + 512)) for b0 in range(0, S, 512)]
    kids = root.spawn(A * len(blocks) + 1)
    jobs = [(a, b0, b1, kids[a * len(blocks) + bi])
            for a in range(A) for bi, (b0, b1) in enumerate(blocks)]

    def work(a, b0, b1, ss):
        rng = _rng(ss)
        x = rng.standard_gamma(conc, size=(b1 - b0, S), dtype=np.float32).astype(np.float64)
        s = x.sum(axis=1, keepdims=True)
        # a row whose draws all underflowed to zero: put its mass on one uniform column
        bad = (s[:, 0] <= 0)
        if bad.any():
            j = rng.integers(0, S, size=int(bad.sum()))
            x[bad] = 0.0
            x[np.nonzero(bad)[0], j] = 1.0
            s = x.sum(axis=1, keepdims=True)
        P[a, b0:b1] = (x / s).astype(dtype)

    _run_blocks(work, jobs)
    g = _rng(kids[-1]).random((A, S))
    return SynthMDP(S=S, A=A, gamma=float(gamma), g=g, kind="dense", P=P,
                    meta=dict(recipe="dense_dirichlet", conc=conc, seed=seed))


def ell_banded(S: int, A: int, k: int, halfwidth: int, shift_step: int, gamma: float,
               seed: int, noise: float = 0.1, val_dtype=np.float32) -> SynthMDP:
    """Banded ELL MDP shaped like a discretised stochastic growth model.

    Row (a, s) has k distinct columns uniform in [c - halfwidth, c + halfwidth] with centre
    c = clamp(s + (a - A//2) * shift_step, halfwidth, S - 1 - halfwidth); weights U(0,1)
    normalised in FP64, stored as val_dtype.  Cost g(s, a) = (2 s / (S-1) - 1)^2 + U(0, noise).
    """
    width = 2 * halfwidth + 1
    if width > S or k > width:
        raise ValueError("band wider than the state space or k > band width")
    col = np.empty((A, S, k), dtype=np.int32)
    val = np.empty((A, S, k), dtype=val_dtype)
    root = np.random.SeedSequence(seed)
    blocks = _blocks(S)
    kids = root.spawn(A * len(blocks) + 1)
    jobs = [(a, b0, b1, kids[a * len(blocks) + bi])
            for a in range(A) for bi, (b0, b1) in enumerate(blocks)]

    def work(a, b0, b1, ss):
        rng = _rng(ss)
        s = np.arange(b0, b1, dtype=np.int64)
        c = np.clip(s + (a - A // 2) * shift_step, halfwidth, S - 1 - halfwidth)
        cols = _distinct_columns(rng, c - halfwidth, width, k)
        w = rng.random((b1 - b0, k))
        w /= w.sum(axis=1, keepdims=True)
        col[a, b0:b1] = cols
        val[a, b0:b1] = w.astype(val_dtype)

    _run_blocks(work, jobs)
    rng = _rng(kids[-1])
    x = 2.0 * np.arange(S, dtype=np.float64) / max(S - 1, 1) - 1.0
    g = np.empty((A, S))
    for a in range(A):
        g[a] = x * x + rng.uniform(0.0, noise, size=S)
    return SynthMDP(S=S, A=A, gamma=float(gamma), g=g, kind="ell", col=col, val=val,
                    meta=dict(recipe="ell_banded", halfwidth=halfwidth,
                              shift_step=shift_step, seed=seed))


def tiny_random(S: int, A: int, seed: int, gamma: float = 0.9, kind: str = "dense",
                k: int | None = None, density: float = 1.0, mask_frac: float = 0.0,
                cost_low: float = 0.0, cost_high: float = 1.0, val_dtype=np.float64) -> SynthMDP:
    """Small random MDP for tests.  Dense rows draw U(0,1) weights on a random support of
    about density*S columns (at least one); ELL rows draw k distinct columns.  With
    mask_frac > 0 each (s, a) is disallowed with that probability, keeping >= 1 action per
    state (paper Sec. 2: A(s) is nonempty)."""
    rng = _rng(seed)
    g = rng.uniform(cost_low, cost_high, size=(A, S))
    mask = None
    if mask_frac > 0:
        mask = rng.random((S, A)) >= mask_frac
        for s in range(S):
            if not mask[s].any():
                mask[s, rng.integers(0, A)] = True
    if kind == "dense":
        w = rng.random((A, S, S))
        keep = rng.random((A, S, S)) < density
        for a in range(A):
            for s in range(S):
                if not keep[a, s].any():
                    keep[a, s, rng.integers(0, S)] = True
        w = np.where(keep, w, 0.0)
        w /= w.sum(axis=2, keepdims=True)
        return SynthMDP(S=S, A=A, gamma=float(gamma), g=g, kind="dense",
                        P=w.astype(val_dtype), mask=mask, meta=dict(recipe="tiny_random"))
    kk = k if k is not None else min(S, 3)
    col = np.empty((A, S, kk), dtype=np.int32)
    val = np.empty((A, S, kk), dtype=val_dtype)
    for a in range(A):
        for s in range(S):
            col[a, s] = rng.choice(S, kk, replace=False)
            w = rng.random(kk)
            val[a, s] = (w / w.sum()).astype(val_dtype)
    return SynthMDP(S=S, A=A, gamma=float(gamma), g=g, kind="ell", col=col, val=val,
                    mask=mask, meta=dict(recipe="tiny_random"))


def batch_specs(n: int, seed: int):
    """Descriptors of n independent MDPs for the batched workload: S log-uniform in
    [500, 50000], A uniform in {2..16}, k in {8, 16, 32} (k <= S), gamma in
    {0.9, 0.99, 0.999}; each instance j gets its own seed (seed * 100003 + j)."""
    rng = _rng(seed)
    out = []
    for j in range(n):
        S = int(round(math.exp(rng.uniform(math.log(500), math.log(50000)))))
        A = int(rng.integers(2, 17))
        k = int(rng.choice([8, 16, 32]))
        gamma = float(rng.choice([0.9, 0.99, 0.999]))
        out.append(dict(S=S, A=A, k=min(k, S), gamma=gamma, seed=seed * 100003 + j))
    return out


def serving_trace(rate: float, duration: float, seed: int):
    """Poisson request stream: exponential inter-arrival times at `rate`/s for `duration`
    seconds; each request is an ELL MDP with S log-uniform in [1e3, 2e5], A in {4, 8, 16},
    k = 16, gamma in {0.95, 0.99} and its own seed."""
    rng = _rng(seed)
    t = 0.0
    out = []
    j = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        S = int(round(math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
        out.append(dict(t=t, S=S, A=int(rng.choice([4, 8, 16])), k=16,
                        gamma=float(rng.choice([0.95, 0.99])), seed=seed * 100003 + j))
        j += 1
    return out


def instance_from_spec(spec: dict, val_dtype=np.float32) -> SynthMDP:
    """Materialise one batched/served instance descriptor as a uniform-column ELL MDP."""
    return ell_uniform(spec["S"], spec["A"], spec["k"], spec["gamma"], spec["seed"],
                       val_dtype=val_dtype)


def config(n: int, *, scale: float = 1.0) -> SynthMDP:
    """The five workloads by number (1..3 are single MDPs; 4 and 5 are described by
    batch_specs / serving_trace).  `scale` < 1 shrinks S for quick checks."""
    if n == 1:
        return ell_uniform(max(16, int(2000 * scale)), 5, 16, 0.95, CONFIG_SEEDS[1],
                           val_dtype=np.float64)
    if n == 2:
        return dense_dirichlet(max(16, int(10000 * scale)), 8, 0.1, 0.99, CONFIG_SEEDS[2],
                               dtype=np.float32)
    if n == 3:
        S = max(4096, int(1_000_000 * scale))
        return ell_banded(S, 16, 32, 512, 64, 0.999, CONFIG_SEEDS[3], val_dtype=np.float32)
    raise ValueError("configs 4 and 5 are collections: use batch_specs / serving_trace")
