"""Seeded synthetic probabilistic Boolean networks (PBNs) and states of interest.

This module only draws random network structure.  It holds none of the
steady-state method's arithmetic (no probability quantisation, no random
streams of the simulation, no statistics), so that both the CPU oracle
(`oracle/`) and the CUDA path (`paper_1508_07828_gb300`) can take their inputs
from it without sharing any of the method's code.

Network format (the PBN G(V, F) of Sec. 2.2, in CSR form):

* ``n``            number of nodes v_0 .. v_{n-1}
* ``fn_offset``    int32[n+1]; the predictor functions of node i are
                   ``fn_offset[i] .. fn_offset[i+1]-1`` (l(i) of them)
* ``par_offset``   int32[F+1]; parents of function f are
                   ``parents[par_offset[f] : par_offset[f+1]]``
* ``parents``      int32[sum k]; node indices, parent m is bit m of the
                   truth-table index
* ``tt_offset``    int32[F+1]; function f's truth table is the words
                   ``tt_words[tt_offset[f] : tt_offset[f+1]]``, max(1, 2^k / 32)
                   of them; the value of f on parent values (x_0..x_{k-1}) is
                   bit j % 32 of word j / 32, j = sum_m x_m 2^m (k <= 15)
* ``tt_words``     uint32[...]
* ``truth_table``  uint32[F]; each function's first word (its whole table
                   when k <= 5)
* ``select_prob``  float64[F]; selection probabilities c_j^(i), summing to 1
                   over the functions of each node
* ``p``            perturbation probability

The five workload recipes mirror the paper's random-PBN generator, which takes
node count, min/max functions per node and min/max parents per function
(Sec. 5.1), with the sizes of the workloads the build is measured on.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 1508078280


@dataclass
class PBN:
    n: int
    fn_offset: np.ndarray
    par_offset: np.ndarray
    parents: np.ndarray
    truth_table: np.ndarray
    select_prob: np.ndarray
    p: float
    name: str = ""
    tt_offset: Optional[np.ndarray] = None
    tt_words: Optional[np.ndarray] = None

    def __post_init__(self):
        if self.tt_offset is None:  # one word per function (every k <= 5)
            self.tt_offset = np.arange(len(self.truth_table) + 1, dtype=np.int32)
            self.tt_words = np.asarray(self.truth_table, dtype=np.uint32).copy()

    def tt_of(self, f: int) -> np.ndarray:
        return self.tt_words[self.tt_offset[f]:self.tt_offset[f + 1]]

    @property
    def n_functions(self) -> int:
        return int(self.fn_offset[-1])

    def functions_of(self, i: int) -> range:
        return range(int(self.fn_offset[i]), int(self.fn_offset[i + 1]))

    def parents_of(self, f: int) -> np.ndarray:
        return self.parents[self.par_offset[f]:self.par_offset[f + 1]]

    def density(self) -> float:
        """D(G) of Sec. 2.2: total parent count over all functions divided by n."""
        return float(len(self.parents)) / self.n


@dataclass
class StateOfInterest:
    """Meta state 1 of the two-state abstraction (Sec. 3.1): every listed node
    holds the listed value."""
    nodes: np.ndarray
    values: np.ndarray

    def __post_init__(self):
        self.nodes = np.asarray(self.nodes, dtype=np.int32)
        self.values = np.asarray(self.values, dtype=np.uint8)


def tt_words_of(tt, k: int) -> np.ndarray:
    """A truth table (Python int, or an array of 2^k bits) as max(1, 2^k/32)
    uint32 words, bit j of the table at bit j % 32 of word j / 32."""
    nw = max(1, (1 << k) >> 5)
    if isinstance(tt, (int, np.integer)):
        return np.array([(int(tt) >> (32 * w)) & 0xFFFFFFFF for w in range(nw)], dtype=np.uint32)
    bits = np.zeros(nw * 32, dtype=np.uint64)
    bits[:len(tt)] = np.asarray(tt, dtype=np.uint64)
    return (bits.reshape(nw, 32) << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)


def _assemble(n, fn_counts, fn_parents, fn_tts, fn_probs, p, name) -> PBN:
    fn_offset = np.zeros(n + 1, dtype=np.int32)
    fn_offset[1:] = np.cumsum(fn_counts)
    F = int(fn_offset[-1])
    par_offset = np.zeros(F + 1, dtype=np.int32)
    par_offset[1:] = np.cumsum([len(x) for x in fn_parents])
    parents = (np.concatenate([np.asarray(x, dtype=np.int32) for x in fn_parents])
               if F and par_offset[-1] else np.zeros(0, dtype=np.int32))
    words = [tt_words_of(tt, len(par)) for tt, par in zip(fn_tts, fn_parents)]
    tt_offset = np.zeros(F + 1, dtype=np.int32)
    tt_offset[1:] = np.cumsum([len(w) for w in words])
    tt_words = np.concatenate(words) if words else np.zeros(0, dtype=np.uint32)
    return PBN(n=n, fn_offset=fn_offset, par_offset=par_offset,
               parents=parents.astype(np.int32),
               truth_table=np.array([w[0] for w in words], dtype=np.uint32),
               select_prob=np.asarray(fn_probs, dtype=np.float64), p=float(p), name=name,
               tt_offset=tt_offset, tt_words=tt_words.astype(np.uint32))


def random_pbn(seed: int, n: int, fn_range=(1, 3), par_range=(1, 3),
               tt_bias: str = "fair", parent_weights: str = "uniform",
               p: float = 0.01, name: str = "") -> PBN:
    """Random PBN after the paper's five-parameter generator (Sec. 5.1).

    fn_range / par_range are inclusive uniform ranges for l(i) and k.  Parents
    of a function are distinct nodes (self allowed).  tt_bias 'fair' draws each
    truth-table bit as a fair coin; 'biased' draws q ~ U(0.3, 0.7) per function
    and each bit ~ Bernoulli(q).  parent_weights 'powerlaw' gives each node a
    weight w_v drawn from the discrete power law P(d) ~ d^-2.5 (d >= 1) and
    picks parents with probability proportional to w_v, so out-degrees are
    scale-free.  Selection probabilities are Dirichlet(1) over each node's
    functions.
    """
    rng = np.random.default_rng(seed)
    if parent_weights == "powerlaw":
        w = rng.zipf(2.5, size=n).astype(np.float64)
        w = np.minimum(w, 1e6)
        wp = w / w.sum()
    else:
        wp = None
    fn_counts, fn_parents, fn_tts, fn_probs = [], [], [], []
    for _ in range(n):
        l = int(rng.integers(fn_range[0], fn_range[1] + 1))
        fn_counts.append(l)
        probs = rng.dirichlet(np.ones(l)) if l > 1 else np.ones(1)
        for j in range(l):
            k = int(rng.integers(par_range[0], par_range[1] + 1))
            k = min(k, n)
            if wp is None:
                par = rng.choice(n, size=k, replace=False)
            else:
                par = rng.choice(n, size=k, replace=False, p=wp)
            if tt_bias == "fair":
                bits = rng.integers(0, 2, size=1 << k)
            else:
                q = rng.uniform(0.3, 0.7)
                bits = (rng.random(1 << k) < q).astype(np.int64)
            fn_parents.append(par)
            fn_tts.append(bits)
            fn_probs.append(float(probs[j]))
    return _assemble(n, fn_counts, fn_parents, fn_tts, fn_probs, p, name)


# ---------------------------------------------------------------------------
# Workload recipes (sizes of the five measured configurations)
# ---------------------------------------------------------------------------

def tiny_config(seed: int = BASE_SEED + 0) -> tuple:
    """n=12; 1-3 functions per node; 1-3 parents; fair truth tables; p=0.01;
    8 chains; state of interest nodes {0,1,2} all 1."""
    net = random_pbn(seed, 12, (1, 3), (1, 3), "fair", "uniform", 0.01, "tiny-n12")
    soi = StateOfInterest([0, 1, 2], [1, 1, 1])
    return net, soi, dict(omega=8, rhat=1.1, r=0.01, s=0.95, eps=1e-10)


def mid_config(seed: int = BASE_SEED + 1) -> tuple:
    """n=100; 2 functions per node; 2-5 parents; truth-table bias q~U(0.3,0.7);
    p=0.001; 1024 chains; state of interest nodes 0..4 = (1,0,1,1,0)."""
    net = random_pbn(seed, 100, (2, 2), (2, 5), "biased", "uniform", 0.001, "mid-n100")
    soi = StateOfInterest([0, 1, 2, 3, 4], [1, 0, 1, 1, 0])
    return net, soi, dict(omega=1024, rhat=1.05, r=0.005, s=0.95, eps=1e-10)


def exact_config(n: int = 16, seed: int = BASE_SEED + 16) -> tuple:
    """A network small enough for the exact solver's implicit step (n <= 16):
    1-3 functions per node, 1-3 parents, biased truth tables, p = 0.05 (fast
    mixing, so FP64 power iteration converges in a few hundred steps); 64
    chains; state of interest nodes {0,1,2} = (1,0,1); r = 0.01."""
    net = random_pbn(seed, n, (1, 3), (1, 3), "biased", "uniform", 0.05, f"exact-n{n}")
    soi = StateOfInterest([0, 1, 2], [1, 0, 1])
    return net, soi, dict(omega=64, psi0=256, rhat=1.05, r=0.01, s=0.95, eps=1e-10)


def large_config(seed: int = BASE_SEED + 2, n: int = 2000) -> tuple:
    """n=2000; 1-4 functions; 2-5 parents drawn with scale-free weights;
    biased truth tables; p=0.001; 16384 chains; Skart at relative precision
    0.01 on a 10-node state of interest (nodes 0..9; the target values are
    supplied by the caller)."""
    net = random_pbn(seed, n, (1, 4), (2, 5), "biased", "powerlaw", 0.001, f"large-n{n}")
    return net, np.arange(10, dtype=np.int32), dict(omega=16384, rhat=1.05, rel=0.01, alpha=0.05)


def wide_config(seed: int = BASE_SEED + 5, n: int = 4096) -> tuple:
    """n=4096; 4-8 functions per node; 2-5 parents with scale-free weights;
    biased truth tables; p=0.001; 16384 chains; state of interest nodes 0..9.
    About 25,000 functions (roughly 400 KB of function records): a network
    whose table does not fit one block's shared memory."""
    net = random_pbn(seed, n, (4, 8), (2, 5), "biased", "powerlaw", 0.001, f"wide-n{n}")
    return net, np.arange(10, dtype=np.int32), dict(omega=16384, rhat=1.05, rel=0.01, alpha=0.05)


# Density classes of the paper's sweep (Sec. 5.1): the density D(G) is the
# parent count of all functions over n, about (functions per node) x (parents
# per function).  Sparse ~10: 2-4 functions of 2-5 parents; in-between 50-100:
# 6-8 functions of 7-12 parents; dense 150-300: 12-16 functions of 10-15
# parents (D about 14 x 12.5 = 175; truth tables of 32-1024 words).
DENSITY_CLASSES = {"sparse": ((2, 4), (2, 5)), "in-between": ((6, 8), (7, 12)), "dense": ((12, 16), (10, 15))}


def sweep_config(n: int, density: str, seed: int = BASE_SEED + 7) -> tuple:
    """One model of the paper-shaped sweep: n nodes, the density class's
    function and parent ranges, biased truth tables, p = 0.001; state of
    interest: 3 random nodes with random values."""
    fns, pars = DENSITY_CLASSES[density]
    s = seed + 1000 * n + {"sparse": 0, "in-between": 1, "dense": 2}[density]
    net = random_pbn(s, n, fns, pars, "biased", "uniform", 0.001, f"sweep-{density}-n{n}")
    soi = random_soi(np.random.default_rng(s), n, 3, 3)
    return net, soi


def _log_uniform_int(rng, lo, hi):
    return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))


def batch_configs(seed: int = BASE_SEED + 3, count: int = 64):
    """64 networks, n log-uniform in [50, 3000], chains log-uniform in
    [256, 4096], built like the mid-size recipe; p in {0.001, 0.01}."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = _log_uniform_int(rng, 50, 3000)
        omega = _log_uniform_int(rng, 256, 4096)
        p = float(rng.choice([0.001, 0.01]))
        net = random_pbn(int(rng.integers(1 << 31)), n, (2, 2), (2, 5), "biased",
                         "uniform", p, f"batch{b}-n{n}")
        soi_nodes = rng.choice(n, size=5, replace=False).astype(np.int32)
        soi_vals = rng.integers(0, 2, size=5).astype(np.uint8)
        out.append((net, StateOfInterest(soi_nodes, soi_vals), dict(omega=omega, rhat=1.05, r=0.005, s=0.95, eps=1e-10)))
    return out


def serving_pool(seed: int = BASE_SEED + 4, count: int = 200):
    """200 networks, n log-uniform in [20, 3000], built like the large recipe."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = _log_uniform_int(rng, 20, 3000)
        out.append(random_pbn(int(rng.integers(1 << 31)), n, (1, 4), (2, 5), "biased",
                              "powerlaw", 0.001, f"pool{b}-n{n}"))
    return out


def random_soi(rng, n: int, lo: int = 1, hi: int = 10) -> StateOfInterest:
    k = int(rng.integers(lo, min(hi, n) + 1))
    nodes = np.sort(rng.choice(n, size=k, replace=False)).astype(np.int32)
    return StateOfInterest(nodes, rng.integers(0, 2, size=k).astype(np.uint8))


# ---------------------------------------------------------------------------
# Hand-built networks with known answers
# ---------------------------------------------------------------------------

def identity_node(p: float) -> PBN:
    """n=1, f(v0) = v0.  Under either perturbation reading the chain flips with
    probability p and stays otherwise (alpha = beta = p)."""
    return _assemble(1, [1], [[0]], [0b10], [1.0], p, "identity")


def constant_node(p: float, value: int = 1) -> PBN:
    """n=1, f = constant (no parents; truth-table bit 0 is the value)."""
    return _assemble(1, [1], [[]], [value & 1], [1.0], p, "constant")


def not_node(p: float) -> PBN:
    """n=1, f(v0) = NOT v0."""
    return _assemble(1, [1], [[0]], [0b01], [1.0], p, "not")


def all_identity(n: int, p: float) -> PBN:
    return _assemble(n, [1] * n, [[i] for i in range(n)], [0b10] * n, [1.0] * n, p, f"ident{n}")


def all_not(n: int, p: float) -> PBN:
    return _assemble(n, [1] * n, [[i] for i in range(n)], [0b01] * n, [1.0] * n, p, f"not{n}")


def three_node(p: float = 1.0 / 16) -> PBN:
    """Hand-built 3-node PBN:
    v0 = AND(v1, v2);  v1 = NOT v0 with probability 3/4, or v1 = v2 with 1/4;
    v2 = OR(v0, v1)."""
    return _assemble(
        3, [1, 2, 1],
        [[1, 2], [0], [2], [0, 1]],
        [0b1000, 0b01, 0b10, 0b1110],
        [1.0, 0.75, 0.25, 1.0], p, "three-node")


def from_lists(n, functions, p, name="custom") -> PBN:
    """functions: list over nodes of lists of (parents, truth_table, prob)."""
    counts, pars, tts, probs = [], [], [], []
    for fl in functions:
        counts.append(len(fl))
        for par, tt, pr in fl:
            pars.append(list(par)); tts.append(tt); probs.append(pr)
    return _assemble(n, counts, pars, tts, probs, p, name)
