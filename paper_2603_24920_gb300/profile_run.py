"""Runs one workload's build and query calls a fixed number of times.

A plain driver for kernel profilers: the same calls bench.py times (build from
device-resident data, then one BF16+refine and one FP32 query call per
repetition), without the recall check, the end-to-end pass or the CPU timing,
so that a profiler sees few launches and little device memory.

  python -m paper_2603_24920_gb300.profile_run --config c2 --reps 2 --beta 0.0015

Launch order per repetition: the build's kernels, then k_query (BF16+refine),
then k_query (FP32).
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c2")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--beta", type=float, default=0.0015)
    ap.add_argument("--c", type=float, default=1.5)
    ap.add_argument("--queries", type=int, default=0, help="first m queries (0 = all)")
    a = ap.parse_args()

    import torch
    import workloads
    from paper_2603_24920_gb300 import detlsh as D

    cfg = workloads.CONFIGS[a.config]
    X = workloads.generate(cfg["kind"], cfg["n"], cfg["d"], cfg["seed"], 0)
    Q = workloads.generate(cfg["kind"], cfg["m"], cfg["d"], cfg["seed"], 1)
    if a.queries:
        Q = Q[:a.queries]
    k = cfg["k"] if isinstance(cfg["k"], int) else max(cfg["k"])
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    st = torch.cuda.current_stream()
    for _ in range(a.reps):
        h = D.detlsh_build(Xd, L=4, K=16, N_r=256, seed=0, max_size=64, stream=st)
        D.detlsh_query_ex(h, Qd, k, beta=a.beta, c=a.c, precision=D.PREC_BF16_REFINE, stream=st)
        D.detlsh_query_ex(h, Qd, k, beta=a.beta, c=a.c, precision=D.PREC_FP32, stream=st)
        torch.cuda.synchronize()
        t = D.detlsh_get_timings(h)
        print("build %.3f ms (sample %.3f, breakpoints %.3f, encode %.3f, trees %.3f)  "
              "query kernel %.3f ms  |S|/q %.0f" %
              (t.build_ms, t.sample_ms, t.breakpoints_ms, t.encode_ms, t.trees_ms,
               t.query_kernel_ms, t.query_candidates / max(1, t.query_count)),
              flush=True)
        D.detlsh_free(h)


if __name__ == "__main__":
    main()
