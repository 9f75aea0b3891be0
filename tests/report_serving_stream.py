"""Report: one served stream of mixed requests, offered at once, through the
continuous-batching server (n uniform in {3..8}, 2d in {4, 6, 8}, r = N;
even request ids SOS targets, odd ones made negative at a point).  Prints the
wall time; meant to run under an ncu launch list, whose kernel shares show
where a served stream spends its GPU time.

    python tests/report_serving_stream.py [--requests 256]
"""
import argparse
import os
import sys
import time

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2410_19844_gb300.server import Server  # noqa: E402
from paper_2410_19844_gb300.workloads import build_jobs  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=256)
    args = ap.parse_args()
    jobs = build_jobs(args.requests, 1.0, seed=0, arrivals=False)
    srv = Server(capacity=512, steps_per_tick=32)
    t0 = time.perf_counter()
    out = srv.run(jobs)
    torch.cuda.synchronize()
    print("served", len(out), "in", round(time.perf_counter() - t0, 3), "s")
    srv.close()


if __name__ == "__main__":
    main()
