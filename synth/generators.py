"""Seeded synthetic series (FP64) with the shapes and value distributions of
the workloads the RQA path is measured on.

Every generator is deterministic in its seed (numpy ``default_rng``).  Both
the CUDA path and the FP64 oracle consume the same FP64 arrays, so the RNG
choice affects nothing downstream.  Nothing here embeds, compares or counts:
these are input recipes only.

Workloads (sizes and parameters as the benchmark uses them):
  * logistic map x_{t+1} = r x_t (1 - x_t), x0 ~ U(0.1, 0.9), 500 iterates
    discarded, values in (0, 1) (not z-scored);
  * x component of the Lorenz system (sigma=10, rho=28, beta=8/3), RK4 with
    dt = 0.01 from an N(0,1)^3 initial state, 10,000 steps discarded,
    z-scored (ddof = 0);
  * AR(1) x_t = phi x_{t-1} + N(0,1), x_{-1} = 0, z-scored;
  * the paper's timing series sin(linspace(0, 1000 pi, 1000001)) (Sect. 8.2);
  * structured series whose recurrence matrices have closed forms
    (constant, period-p integer sequences, dyadic random values).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.signal import lfilter

__all__ = [
    "logistic", "lorenz_x", "ar1", "sine_paper", "constant", "periodic",
    "dyadic", "zscore", "logistic_many", "lorenz_x_many", "ar1_many",
    "SeriesSpec", "draw_spec", "batch_specs", "make_series", "serve_stream",
    "WORKLOADS", "workload",
]


def zscore(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return (x - x.mean()) / x.std()


# --------------------------------------------------------------------------
# single series
# --------------------------------------------------------------------------
def logistic(N: int, seed: int, r: float = 3.9, discard: int = 500) -> np.ndarray:
    return logistic_many([N], [r], np.random.default_rng(seed), discard)[0]


def lorenz_x(N: int, seed: int, dt: float = 0.01, discard: int = 10_000) -> np.ndarray:
    return lorenz_x_many([N], np.random.default_rng(seed), dt, discard)[0]


def ar1(N: int, seed: int, phi: float = 0.95) -> np.ndarray:
    return ar1_many([N], [phi], np.random.default_rng(seed))[0]


def sine_paper(N: int = 1_000_001) -> np.ndarray:
    """The synthetic series of the paper's runtime experiment (Sect. 8.2)."""
    return np.sin(np.linspace(0.0, 1000.0 * np.pi, N))


def constant(N: int, value: float = 0.25) -> np.ndarray:
    return np.full(N, value, dtype=np.float64)


def periodic(N: int, p: int, offset: int = 0) -> np.ndarray:
    """s_t = (t + offset) mod p as FP64 integers."""
    return ((np.arange(N, dtype=np.int64) + offset) % p).astype(np.float64)


def dyadic(N: int, seed: int, levels: int = 8, scale_log2: int = -3) -> np.ndarray:
    """Random multiples of 2**scale_log2 in [0, levels): every difference,
    square and sum of a few of them is exact in FP32 and FP64, so distance
    ties d == eps occur and are decided without rounding."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, levels, size=N).astype(np.float64) * 2.0 ** scale_log2


# --------------------------------------------------------------------------
# vectorised over many series (used for the batched and served workloads)
# --------------------------------------------------------------------------
def logistic_many(lengths, rs, rng, discard: int = 500):
    lengths = np.asarray(lengths, dtype=np.int64)
    rs = np.asarray(rs, dtype=np.float64)
    k = len(lengths)
    x = rng.uniform(0.1, 0.9, size=k)
    T = int(lengths.max()) if k else 0
    out = np.empty((k, T), dtype=np.float64)
    for _ in range(discard):
        x = rs * x * (1.0 - x)
    for t in range(T):
        out[:, t] = x
        x = rs * x * (1.0 - x)
    return [out[i, :lengths[i]].copy() for i in range(k)]


def _lorenz_rhs(v, sigma=10.0, rho=28.0, beta=8.0 / 3.0):
    x, y, z = v[:, 0], v[:, 1], v[:, 2]
    return np.stack([sigma * (y - x), x * (rho - z) - y, x * y - beta * z], axis=1)


def lorenz_x_many(lengths, rng, dt: float = 0.01, discard: int = 10_000):
    lengths = np.asarray(lengths, dtype=np.int64)
    k = len(lengths)
    v = rng.standard_normal(size=(k, 3))
    T = int(lengths.max()) if k else 0
    out = np.empty((k, T), dtype=np.float64)
    for t in range(discard + T):
        if t >= discard:
            out[:, t - discard] = v[:, 0]
        k1 = _lorenz_rhs(v)
        k2 = _lorenz_rhs(v + 0.5 * dt * k1)
        k3 = _lorenz_rhs(v + 0.5 * dt * k2)
        k4 = _lorenz_rhs(v + dt * k3)
        v = v + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return [zscore(out[i, :lengths[i]]) for i in range(k)]


def ar1_many(lengths, phis, rng):
    res = []
    for L, phi in zip(lengths, phis):
        e = rng.standard_normal(int(L))
        res.append(zscore(lfilter([1.0], [1.0, -float(phi)], e)))
    return res


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class SeriesSpec:
    """One series of a batched or served workload and its analysis
    parameters (norm: 0 = max, 1 = L2, 2 = L1)."""
    kind: str
    length: int
    m: int
    tau: int
    norm: int
    eps_rel: float          # eps = eps_rel * std(series)
    gen_param: float        # r (logistic) or phi (AR(1)); unused for Lorenz
    theiler: int = 1
    l_min: int = 2
    v_min: int = 2
    w_min: int = 2


def draw_spec(rng, length: int) -> SeriesSpec:
    """Parameters of one batched / served series (see batch_specs)."""
    kind = ("logistic", "lorenz", "ar1")[int(rng.integers(0, 3))]
    m = int(rng.integers(2, 9))
    tau = int(rng.integers(1, 5))
    norm = int(rng.integers(0, 3))
    eps_rel = float(rng.uniform(0.05, 0.5))
    if kind == "logistic":
        gp = float(rng.uniform(3.6, 4.0))
    elif kind == "ar1":
        gp = float(rng.uniform(0.5, 0.99))
    else:
        gp = 0.0
    return SeriesSpec(kind, int(length), m, tau, norm, eps_rel, gp)


def batch_specs(count: int = 4096, seed: int = 1004, lo: int = 500,
                hi: int = 20_000):
    """Uneven-length batch: lengths uniform-int in [lo, hi], generator kind
    uniform over {logistic, Lorenz-x, AR(1)}, m in [2, 8], tau in [1, 4],
    norm uniform over {max, L2, L1}, eps uniform in [0.05, 0.5] * std,
    Theiler window 1, minimum line lengths 2."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(lo, hi + 1, size=count)
    return [draw_spec(rng, int(L)) for L in lengths]


def make_series(specs, seed: int):
    """Generate the FP64 series for a list of SeriesSpec (vectorised per
    kind).  Returns (series_list, eps_list)."""
    rng = np.random.default_rng(seed)
    out = [None] * len(specs)
    idx = {"logistic": [], "lorenz": [], "ar1": []}
    for i, sp in enumerate(specs):
        idx[sp.kind].append(i)
    if idx["logistic"]:
        ii = idx["logistic"]
        ser = logistic_many([specs[i].length for i in ii],
                            [specs[i].gen_param for i in ii], rng)
        for i, s in zip(ii, ser):
            out[i] = s
    if idx["lorenz"]:
        ii = idx["lorenz"]
        ser = lorenz_x_many([specs[i].length for i in ii], rng)
        for i, s in zip(ii, ser):
            out[i] = s
    if idx["ar1"]:
        ii = idx["ar1"]
        ser = ar1_many([specs[i].length for i in ii],
                       [specs[i].gen_param for i in ii], rng)
        for i, s in zip(ii, ser):
            out[i] = s
    eps = [float(sp.eps_rel * np.std(s)) for sp, s in zip(specs, out)]
    return out, eps


def serve_stream(rate: float = 200.0, duration: float = 60.0, seed: int = 1005,
                 lo: int = 1_000, hi: int = 200_000, pool: int = 48):
    """Poisson request stream: arrival times (s), one SeriesSpec per request
    with a log-uniform length in [lo, hi], parameters drawn as for the batch.

    To keep generation fast, each generator kind draws `pool` long base
    series of length `hi` (with their own r / phi); request q takes the
    first `length` points of base series q mod pool of its kind (re-z-scored
    for the z-scored kinds).  Returns (arrivals, specs, series, eps)."""
    rng = np.random.default_rng(seed)
    arrivals = []
    t = 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        arrivals.append(t)
    k = len(arrivals)
    lengths = np.exp(rng.uniform(math.log(lo), math.log(hi), size=k)).astype(np.int64)
    specs = [draw_spec(rng, int(L)) for L in lengths]
    base_rng = np.random.default_rng(seed + 1)
    bases = {
        "logistic": logistic_many([hi] * pool, base_rng.uniform(3.6, 4.0, pool), base_rng),
        "lorenz": lorenz_x_many([hi] * pool, base_rng),
        "ar1": ar1_many([hi] * pool, base_rng.uniform(0.5, 0.99, pool), base_rng),
    }
    series, eps = [], []
    counters = {"logistic": 0, "lorenz": 0, "ar1": 0}
    for sp in specs:
        q = counters[sp.kind]
        counters[sp.kind] += 1
        s = bases[sp.kind][q % pool][:sp.length]
        if sp.kind != "logistic":
            s = zscore(s)
        series.append(np.ascontiguousarray(s))
        eps.append(float(sp.eps_rel * np.std(s)))
    return np.asarray(arrivals), specs, series, eps


# Single-series workloads with their analysis parameters.
WORKLOADS = {
    "logistic_n2000": dict(N=2_000, m=3, tau=2, norm=1, eps=0.1, theiler=1),
    "lorenz_n100k": dict(N=100_000, m=5, tau=3, norm=0, eps=0.3, theiler=5),
    "ar1_n1m": dict(N=1_048_576, m=3, tau=1, norm=1, eps=0.5, theiler=1),
    "sine_paper": dict(N=1_000_001, m=2, tau=2, norm=1, eps=1.0, theiler=0),
}


def workload(name: str, seed: int | None = None):
    """(series, params) for a named single-series workload.  Default seeds:
    1001 (logistic), 1002 (Lorenz), 1003 (AR(1))."""
    p = dict(WORKLOADS[name])
    N = p.pop("N")
    if name == "logistic_n2000":
        s = logistic(N, 1001 if seed is None else seed)
    elif name == "lorenz_n100k":
        s = lorenz_x(N, 1002 if seed is None else seed)
    elif name == "ar1_n1m":
        s = ar1(N, 1003 if seed is None else seed)
    elif name == "sine_paper":
        s = sine_paper(N)
    else:
        raise KeyError(name)
    p.update(l_min=2, v_min=2, w_min=2)
    return s, p
