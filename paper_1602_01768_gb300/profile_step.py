"""Per-phase timing of AdaRBFGS steps on the n x n workload (CUDA events).

    python -m paper_1602_01768_gb300.profile_step --n 16384 --q 128 --prec mixed --steps 5

prints one JSON line per precision form with the median device time of each
phase of a step (sketch draw, S = L S~, G = A S, Gram products, q x q core,
W = L^T G, V and S^, update of L).  With --plain it only runs --warmup plus
--steps steps without events, which is the form to put under a profiler.
"""
import argparse
import json
import os
import statistics
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--q", type=int, default=128)
    ap.add_argument("--prec", default="mixed")
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--plain", action="store_true")
    args = ap.parse_args()

    import torch

    import paper_1602_01768_gb300._binding as B
    from paper_1602_01768_gb300 import workloads as wl

    A = wl.c3_matrix(n=args.n, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for pn in args.prec.split(","):
        o = B.make_opts(method=B.RB_METHOD_ADARBFGS, sketch=B.RB_SKETCH_GAUSS, q=args.q, prec=B.PREC[pn], seed=1)
        h = B.rbfgs_init(args.n, A.data_ptr(), args.n, False, o, st)
        B.adarbfgs_step(h, args.warmup)
        if args.plain:
            B.adarbfgs_step(h, args.steps)
            B.rbfgs_sync(h)
            print(json.dumps({"prec": pn, "n": args.n, "q": args.q, "steps": args.steps}), flush=True)
        else:
            prof = {}
            for _ in range(args.steps):
                for name, ms in B.rbfgs_profile_step(h):
                    prof.setdefault(name, []).append(ms)
            ph = {k: round(statistics.median(v), 4) for k, v in prof.items()}
            print(json.dumps({"prec": pn, "n": args.n, "q": args.q, "phases_ms": ph,
                              "step_ms": round(sum(ph.values()), 4)}), flush=True)
        B.rbfgs_destroy(h)


if __name__ == "__main__":
    main()
