"""Seeded synthetic workloads shaped like the paper's datasets.

Input synthesis only: no step of the DET-LSH method lives here.  Both the CUDA
path's tests/bench and the oracle take their inputs from these generators.

The paper evaluates on real datasets (Table 2: Msong, Deep1M, Sift10M/100M,
Deep500M, SPACEV500M, Turing500M) that are not available here; these seeded
Gaussian-mixture generators stand in for them with the same shapes:

  c1  n=1e5,  d=128 : 100 centres ~ N(0, 10^2 I), sigma = 1; 100 queries, k=10
  c2  n=1e6,  d=128 : 1000 integer centres in [0,255]^d, +N(0,20^2), rounded and
                       clipped to [0,255] (SIFT-like); 10,000 queries, k=50
  c3  n=1e6,  d=960 : 64-d latent mixture (100 centres ~ N(0,10^2 I), sigma 1)
                       mapped by W ~ N(0,1/64) (64x960) + N(0, 0.05^2); 1,000
                       queries with k uniform in {10,20,50,100}
  c4  n=1e7,  d=96  : 10,000 centres ~ N(0, I) + N(0, 0.1^2 I), L2-normalised;
                       10,000 queries, k=100
  c5  n=1e8,  d=96  : the c4 generator at seed 4; 100,000 queries in batches of
                       1..4096, k uniform in {1,10,100}

Rows are generated in fixed 65,536-row chunks, each from its own Philox stream,
so any chunk can be regenerated on its own, and the first n rows of a longer
draw are the n-row draw whenever n is a multiple of the chunk size (a partial
last chunk is drawn for its own length).
"""
import numpy as np

CHUNK = 65536

CONFIGS = {
    "c1": dict(n=100_000, d=128, m=100, k=10, seed=0, kind="gauss"),
    "c2": dict(n=1_000_000, d=128, m=10_000, k=50, seed=1, kind="sift"),
    "c3": dict(n=1_000_000, d=960, m=1_000, k=(10, 20, 50, 100), seed=2, kind="latent"),
    "c4": dict(n=10_000_000, d=96, m=10_000, k=100, seed=3, kind="sphere"),
    "c5": dict(n=100_000_000, d=96, m=100_000, k=(1, 10, 100), seed=4, kind="sphere"),
}


def _rng(seed, stream, chunk=0):
    # Philox bit generator keyed by (seed, stream, chunk): independent streams.
    return np.random.Generator(np.random.Philox(key=[(seed << 32) | stream, chunk]))


def _params(kind, d, seed):
    g = _rng(seed, 100)
    if kind == "gauss":
        return dict(centers=g.normal(0.0, 10.0, (100, d)))
    if kind == "sift":
        return dict(centers=g.integers(0, 256, (1000, d)).astype(np.float64))
    if kind == "latent":
        return dict(centers=g.normal(0.0, 10.0, (100, 64)),
                    W=g.normal(0.0, 1.0 / 8.0, (64, d)))
    if kind == "sphere":
        return dict(centers=g.normal(0.0, 1.0, (10_000, d)))
    raise ValueError(kind)


def _rows(kind, prm, d, g, cnt):
    C = prm["centers"]
    lab = g.integers(0, C.shape[0], cnt)
    if kind == "gauss":
        X = C[lab] + g.normal(0.0, 1.0, (cnt, d))
    elif kind == "sift":
        X = np.clip(np.rint(C[lab] + g.normal(0.0, 20.0, (cnt, d))), 0, 255)
    elif kind == "latent":
        z = C[lab] + g.normal(0.0, 1.0, (cnt, 64))
        X = z @ prm["W"] + g.normal(0.0, 0.05, (cnt, d))
    elif kind == "sphere":
        X = C[lab] + g.normal(0.0, 0.1, (cnt, d))
        X /= np.linalg.norm(X, axis=1, keepdims=True)
    return X.astype(np.float32)


def generate(kind, n, d, seed, stream, rows=None):
    """Rows [0, n) (or the listed row ids) of a workload; stream 0 = data, 1 = queries."""
    prm = _params(kind, d, seed)
    if rows is None:
        out = np.empty((n, d), np.float32)
        for c0 in range(0, n, CHUNK):
            cnt = min(CHUNK, n - c0)
            out[c0:c0 + cnt] = _rows(kind, prm, d, _rng(seed, stream, c0 // CHUNK), cnt)
        return out
    rows = np.asarray(rows, np.int64)
    out = np.empty((rows.size, d), np.float32)
    for ch in np.unique(rows // CHUNK):
        c0 = int(ch) * CHUNK
        cnt = min(CHUNK, n - c0)
        blk = _rows(kind, prm, d, _rng(seed, stream, int(ch)), cnt)
        sel = rows // CHUNK == ch
        out[sel] = blk[rows[sel] - c0]
    return out


def workload(name, n=None, m=None):
    """(X, Q, k) for a named config; n and m may be reduced for small cases."""
    cfg = CONFIGS[name]
    n = cfg["n"] if n is None else n
    m = cfg["m"] if m is None else m
    X = generate(cfg["kind"], n, cfg["d"], cfg["seed"], 0)
    Q = generate(cfg["kind"], m, cfg["d"], cfg["seed"], 1)
    k = cfg["k"]
    if isinstance(k, tuple):
        k = _rng(cfg["seed"], 4).choice(np.asarray(k, np.int32), m)
    return X, Q, k


def batch_sizes(total, seed=4, lo=1, hi=4096):
    """Uneven query batches: sizes floor(exp(U[0, ln(hi+1)])) clipped to [lo, hi]."""
    g = _rng(seed, 5)
    out, left = [], total
    while left > 0:
        s = int(np.clip(np.floor(np.exp(g.uniform(0.0, np.log(hi + 1)))), lo, hi))
        s = min(s, left)
        out.append(s)
        left -= s
    return out
