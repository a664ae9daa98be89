"""Measurements beyond the benchmark line: the other workload configurations,
the recall knobs, the paper's query variants and the encoding ablation.

  python -m paper_2603_24920_gb300.experiments configs    # c1, c3, c4 (c5: --c5-n)
  python -m paper_2603_24920_gb300.experiments sweep      # beta x max_size on c2
  python -m paper_2603_24920_gb300.experiments lk         # L x K on c2
  python -m paper_2603_24920_gb300.experiments variants   # r_min policy, (r,c)-ANN,
                                                          # static vs dynamic encoding
  python -m paper_2603_24920_gb300.experiments stream     # c5: uneven batches through
                                                          # captured CUDA graphs

Every number is device time from CUDA events (the library's own timings) on
device-resident inputs, after one warm-up call.  Recall@10 (or recall@k for
k < 10) is measured against exact FP64 brute force on the GPU (plain PyTorch)
for up to 200 queries.  Inputs are the seeded synthetic workloads of
`workloads`; nothing here is on the benchmark's timed path.
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _torch():
    import torch
    return torch


def exact_knn(Xd, Q, k, nq=200):
    torch = _torch()
    Qd = torch.from_numpy(Q[:nq]).to(Xd.device, torch.float64)
    ids = []
    for i in range(0, Qd.shape[0], 8):
        best_d, best_i = None, None
        for c0 in range(0, Xd.shape[0], 2_000_000):
            xb = Xd[c0:c0 + 2_000_000].double()
            dd = torch.cdist(Qd[i:i + 8], xb, compute_mode="donot_use_mm_for_euclid_dist")
            v, ix = torch.topk(dd, min(k, xb.shape[0]), largest=False)
            ix = ix + c0
            if best_d is None:
                best_d, best_i = v, ix
            else:
                v2 = torch.cat([best_d, v], 1)
                i2 = torch.cat([best_i, ix], 1)
                o = torch.topk(v2, k, largest=False)
                best_d, best_i = o.values, torch.gather(i2, 1, o.indices)
            del xb
        ids.append(best_i.cpu())
    return torch.cat(ids).numpy()


def recall(ids, gt, kk):
    kk = np.asarray(kk)
    out = []
    for i in range(gt.shape[0]):
        r = int(min(10, kk[i] if kk.ndim else kk))
        out.append(len(set(ids[i, :r].tolist()) & set(gt[i, :r].tolist())) / r)
    return float(np.mean(out))


def run_query(D, h, Qd, k, kq=None, reps=2, **kw):
    for _ in range(reps):
        ids, dists = D.detlsh_query_ex(h, Qd, k, k_per_query=kq, **kw)
    t = D.detlsh_get_timings(h)
    return ids, dists, t


def row(*cols):
    print("| " + " | ".join(str(c) for c in cols) + " |", flush=True)


def cmd_configs(a):
    torch = _torch()
    import workloads
    from paper_2603_24920_gb300 import detlsh as D
    row("config", "n x d", "queries", "k", "beta", "build ms", "Mpts/s", "query kernel ms",
        "queries/s (BF16)", "queries/s (FP32)", "recall@10 BF16 / FP32", "S per query")
    todo = [("c1", None, (0.01, 0.002)), ("c3", None, (0.002, 0.01, 0.05)),
            ("c4", None, (0.0015, 0.0003, 0.0001))]
    if a.c5_n:
        todo.append(("c5", a.c5_n, (0.0003, 0.0001, 0.00003)))
    for name, n, betas in todo:
        cfg = workloads.CONFIGS[name]
        nn = n or cfg["n"]
        m = min(cfg["m"], 10_000)
        t0 = time.time()
        X, Q, k = workloads.workload(name, n=nn, m=m)
        gen_s = time.time() - t0
        Xd = torch.from_numpy(X).cuda()
        Qd = torch.from_numpy(Q).cuda()
        del X
        kq = None if np.isscalar(k) else np.asarray(k, np.int32)
        kmax = int(k) if kq is None else int(kq.max())
        h = D.detlsh_build(Xd, L=4, K=16, N_r=256, seed=0, max_size=64)
        D.detlsh_free(h)
        h = D.detlsh_build(Xd, L=4, K=16, N_r=256, seed=0, max_size=64)
        tb = D.detlsh_get_timings(h)
        gt = exact_knn(Xd, Q, max(10, kmax) if kq is None else 10)
        for beta in betas:
            res = {}
            for prec, pname in ((D.PREC_BF16_REFINE, "bf16"), (D.PREC_FP32, "fp32")):
                ids, _, t = run_query(D, h, Qd, kmax, kq, beta=beta, precision=prec)
                ids = ids.cpu().numpy()[:gt.shape[0]]
                res[pname] = (t.query_kernel_ms, t.query_ms,
                              recall(ids, gt, kq[:gt.shape[0]] if kq is not None else kmax),
                              t.query_candidates / max(1, t.query_count))
            row(name + (" (first %d)" % nn if n else ""), "%d x %d" % (nn, cfg["d"]), m,
                kmax if kq is None else "mixed %s" % sorted(set(kq.tolist())), beta,
                "%.2f" % tb.build_ms, "%.1f" % (nn / tb.build_ms / 1e3),
                "%.2f / %.2f" % (res["bf16"][0], res["fp32"][0]),
                "%.0f" % (m / res["bf16"][1] * 1e3), "%.0f" % (m / res["fp32"][1] * 1e3),
                "%.3f / %.3f" % (res["bf16"][2], res["fp32"][2]), "%.0f" % res["fp32"][3])
        print("  (data generated on the host in %.0f s)" % gen_s, flush=True)
        D.detlsh_free(h)
        del Xd, Qd
        torch.cuda.empty_cache()


def _c2():
    torch = _torch()
    import workloads
    X, Q, k = workloads.workload("c2")
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    gt = exact_knn(Xd, Q, 10)
    return Xd, Qd, Q, gt


def cmd_sweep(a):
    from paper_2603_24920_gb300 import detlsh as D
    Xd, Qd, Q, gt = _c2()
    Qs = Qd[:1000].contiguous()  # large beta gathers ~beta*n rows per query
    print("c2, first 1,000 queries, k = 50; kernel ms per 1,000 queries")
    row("max_size", "beta", "build ms", "kernel ms FP32", "kernel ms BF16", "recall@10", "S per query")
    for M in (16, 64, 256):
        h = D.detlsh_build(Xd, L=4, K=16, N_r=256, seed=0, max_size=M)
        tb = D.detlsh_get_timings(h).build_ms
        for beta in (0.1, 0.05, 0.02, 0.01, 0.005, 0.002, 0.0015, 0.001):
            reps = 1 if beta >= 0.01 else 2
            ids, _, t = run_query(D, h, Qs, 50, reps=reps, beta=beta, precision=D.PREC_FP32)
            _, _, tb16 = run_query(D, h, Qs, 50, reps=reps, beta=beta, precision=D.PREC_BF16_REFINE)
            rec = recall(ids.cpu().numpy()[:gt.shape[0]], gt, 10)
            row(M, beta, "%.2f" % tb, "%.2f" % t.query_kernel_ms, "%.2f" % tb16.query_kernel_ms,
                "%.3f" % rec, "%.0f" % (t.query_candidates / t.query_count))
        D.detlsh_free(h)


def cmd_lk(a):
    from paper_2603_24920_gb300 import detlsh as D
    Xd, Qd, Q, gt = _c2()
    row("L", "K", "eps^2", "build ms", "kernel ms (beta 0.0015)", "recall@10", "S per query")
    for L, K in ((2, 16), (4, 16), (8, 16), (4, 8), (8, 8), (4, 12)):
        h = D.detlsh_build(Xd, L=L, K=K, N_r=256, seed=0, max_size=64)
        tb = D.detlsh_get_timings(h).build_ms
        ids, _, t = run_query(D, h, Qd, 50, beta=0.0015, precision=D.PREC_FP32)
        rec = recall(ids.cpu().numpy()[:gt.shape[0]], gt, 10)
        row(L, K, "%.3f" % D.detlsh_get_info(h).eps2, "%.2f" % tb, "%.2f" % t.query_kernel_ms,
            "%.3f" % rec, "%.0f" % (t.query_candidates / t.query_count))
        D.detlsh_free(h)


def cmd_variants(a):
    torch = _torch()
    import workloads
    from paper_2603_24920_gb300 import detlsh as D
    Xd, Qd, Q, gt = _c2()
    h = D.detlsh_build(Xd, L=4, K=16, N_r=256, seed=0, max_size=64, keep_projections=1)
    print("r_min policy (Alg. 5), c2, beta = 0.0015, k = 50, FP32 path:")
    row("r_min", "kernel ms", "recall@10", "S per query")
    ids, _, t = run_query(D, h, Qd, 50, beta=0.0015)
    row("magic grid", "%.2f" % t.query_kernel_ms, "%.3f" % recall(ids.cpu().numpy()[:200], gt, 10),
        "%.0f" % (t.query_candidates / t.query_count))
    for r0 in (1.0, 10.0, 100.0, 400.0):
        ids, _, t = run_query(D, h, Qd, 50, beta=0.0015, r_min=r0)
        row("fixed %g" % r0, "%.2f" % t.query_kernel_ms,
            "%.3f" % recall(ids.cpu().numpy()[:200], gt, 10),
            "%.0f" % (t.query_candidates / t.query_count))
    # (r,c)-ANN at r = the true nearest-neighbour distance times a factor
    Qn = Q[:200]
    nn = []
    for i in range(0, 200, 8):
        dd = torch.cdist(torch.from_numpy(Qn[i:i + 8]).cuda().double(), Xd.double(),
                         compute_mode="donot_use_mm_for_euclid_dist")
        nn.append(dd.min(1).values.cpu().numpy())
    nn = np.concatenate(nn)
    print("Alg. 5 with and without the priority queue of Sec. VI-B2, c2, beta = 0.0015, k = 50:")
    row("budget check", "kernel ms", "recall@10", "S per query")
    for pt in (False, True):
        ids, _, t = run_query(D, h, Qd, 50, beta=0.0015, per_tree=pt)
        row("after each tree (as printed)" if pt else "after each leaf (priority queue)",
            "%.2f" % t.query_kernel_ms, "%.3f" % recall(ids.cpu().numpy()[:200], gt, 10),
            "%.0f" % (t.query_candidates / t.query_count))
    print("(r,c)-ANN (Alg. 4), c2, c = 1.5, 200 queries: Alg. 3 as printed vs optimisation (1)"
          " of Sec. VI-B2 (whole leaves):")
    row("range query", "r / NN distance", "beta", "kernel ms per query", "answered within c*r",
        "returns the true NN", "mean S size")
    r_med = float(np.median(nn))
    nn_id = exact_knn(Xd, Qn, 1, nq=200)[:, 0]
    for opt in (False, True):
        for f in (1.0, 1.5):
            for beta in (0.0015, 0.01):
                r = f * r_med
                D.detlsh_rc_ann(h, Qn, r, beta=beta, optimised=opt)
                ids, dists, stop, ssz, _ = D.detlsh_rc_ann(h, Qn, r, beta=beta, optimised=opt)
                t = D.detlsh_get_timings(h)
                ok = np.mean((ids >= 0) & (dists <= 1.5 * r * (1 + 1e-6)))
                row("whole leaves" if opt else "as printed", "%.1f x median (r = %.1f)" % (f, r),
                    beta, "%.4f" % (t.query_kernel_ms / 200), "%.3f" % ok,
                    "%.3f" % np.mean(ids == nn_id), "%.0f" % ssz.mean())
    D.detlsh_free(h)
    del Xd, Qd
    torch.cuda.empty_cache()
    print("encoding scheme (Sec. III-A), 1e6 points, beta = 0.0015, FP32 path:")
    row("data", "encoding", "build ms", "max leaf", "kernel ms", "recall@10", "S per query")
    for name in ("c4", "c2"):
        X, Qx, k = workloads.workload(name, n=1_000_000, m=2000)
        Xd = torch.from_numpy(X).cuda()
        Qd = torch.from_numpy(Qx).cuda()
        g = exact_knn(Xd, Qx, 10)
        for enc in (D.ENC_DYNAMIC, D.ENC_STATIC):
            h = D.detlsh_build(Xd, L=4, K=16, N_r=256, seed=0, max_size=64, encoding=enc)
            tb = D.detlsh_get_timings(h).build_ms
            info = D.detlsh_get_info(h)
            ids, _, t = run_query(D, h, Qd, 10, beta=0.0015)
            row(name, "static" if enc else "dynamic", "%.2f" % tb, info.max_leaf_size,
                "%.2f" % t.query_kernel_ms, "%.3f" % recall(ids.cpu().numpy()[:200], g, 10),
                "%.0f" % (t.query_candidates / t.query_count))
            D.detlsh_free(h)
        del Xd, Qd
        torch.cuda.empty_cache()


def cmd_stream(a):
    """c5's serving pattern: a stream of 100,000 queries in uneven batches
    (sizes 1..4096), k in {1, 10, 100}, answered by detlsh_query_async replayed
    from CUDA graphs (one per power-of-two batch bucket, captured on first use;
    a batch is padded to its bucket with copies of its last query).  Each batch
    is copied in from pinned host memory and its results copied back."""
    torch = _torch()
    import workloads
    from paper_2603_24920_gb300 import detlsh as D
    cfg = workloads.CONFIGS["c5"]
    n = a.n or cfg["n"]
    t0 = time.time()
    X = workloads.generate(cfg["kind"], n, cfg["d"], cfg["seed"], 0)
    Q = workloads.generate(cfg["kind"], cfg["m"], cfg["d"], cfg["seed"], 1)
    kq = np.asarray(workloads._rng(cfg["seed"], 4).choice(np.asarray(cfg["k"], np.int32), cfg["m"]),
                    np.int32)
    sizes = workloads.batch_sizes(cfg["m"])
    gen_s = time.time() - t0
    Xd = torch.from_numpy(X).cuda()
    del X
    h = D.detlsh_build(Xd, L=4, K=16, N_r=256, seed=0, max_size=64)
    D.detlsh_free(h)
    h = D.detlsh_build(Xd, L=4, K=16, N_r=256, seed=0, max_size=64)
    tb = D.detlsh_get_timings(h).build_ms
    kmax = int(kq.max())
    D.detlsh_query_reserve(h, 4096, kmax, beta=a.beta, precision=D.PREC_BF16_REFINE)
    st = torch.cuda.Stream()
    Qh = torch.from_numpy(Q).pin_memory()
    Kh = torch.from_numpy(kq).pin_memory()
    ids_h = torch.empty((cfg["m"], kmax), dtype=torch.int64).pin_memory()
    d_h = torch.empty((cfg["m"], kmax), dtype=torch.float32).pin_memory()
    graphs = {}

    def bucket(s):
        b = 1
        while b < s:
            b *= 2
        return b

    def get_graph(B):
        if B not in graphs:
            qb = torch.zeros((B, cfg["d"]), dtype=torch.float32, device="cuda")
            kb = torch.ones(B, dtype=torch.int32, device="cuda")
            ib = torch.empty((B, kmax), dtype=torch.int64, device="cuda")
            db = torch.empty((B, kmax), dtype=torch.float32, device="cuda")
            sb = torch.zeros(1, dtype=torch.int32, device="cuda")
            with torch.cuda.stream(st):
                D.detlsh_query_async(h, qb, kmax, ib, db, sb, k_per_query=kb, stream=st)
            st.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                D.detlsh_query_async(h, qb, kmax, ib, db, sb, k_per_query=kb, stream=st)
            graphs[B] = (g, qb, kb, ib, db, sb)
        return graphs[B]

    def run_stream():
        pos = 0
        with torch.cuda.stream(st):
            for s in sizes:
                g, qb, kb, ib, db, sb = get_graph(bucket(s))
                B = qb.shape[0]
                qb[:s].copy_(Qh[pos:pos + s], non_blocking=True)
                kb[:s].copy_(Kh[pos:pos + s], non_blocking=True)
                if B > s:
                    qb[s:].copy_(qb[s - 1:s].expand(B - s, -1))
                    kb[s:].fill_(1)
                g.replay()
                ids_h[pos:pos + s].copy_(ib[:s], non_blocking=True)
                d_h[pos:pos + s].copy_(db[:s], non_blocking=True)
                pos += s
        st.synchronize()

    run_stream()  # captures the graphs, warms up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    e0.record(st)
    run_stream()
    e1.record(st)
    st.synchronize()
    wall = time.time() - w0
    ms = e0.elapsed_time(e1)
    gt = exact_knn(Xd, Q, 10, nq=200)
    rec = recall(ids_h.numpy()[:200], gt, kq[:200])
    print("c5 stream: n = %d x %d (data generated on the host in %.0f s), build %.1f ms "
          "(%.0f M points/s)" % (n, cfg["d"], gen_s, tb, n / tb / 1e3))
    row("queries", "batches", "graphs", "beta", "stream ms (device)", "queries/s",
        "wall s", "recall@min(k,10)")
    row(cfg["m"], len(sizes), len(graphs), a.beta, "%.1f" % ms, "%.0f" % (cfg["m"] / ms * 1e3),
        "%.2f" % wall, "%.3f" % rec)
    D.detlsh_free(h)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["configs", "sweep", "lk", "variants", "stream"])
    ap.add_argument("--c5-n", type=int, default=0, help="also run the first N points of c5")
    ap.add_argument("--n", type=int, default=0, help="stream: points of c5 (0 = all 1e8)")
    ap.add_argument("--beta", type=float, default=5e-5, help="stream: beta")
    a = ap.parse_args()
    {"configs": cmd_configs, "sweep": cmd_sweep, "lk": cmd_lk, "variants": cmd_variants,
     "stream": cmd_stream}[a.what](a)


if __name__ == "__main__":
    main()
