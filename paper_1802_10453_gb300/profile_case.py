"""One factorisation of a planted matrix, for profiling under ncu.

    python -m paper_1802_10453_gb300.profile_case N [p] [path]

Draws A = T R T^T (n = N, rank N/2, a quarter of R's non-zeros in 2x2 pairs)
on the GPU, factors it once through the C ABI and prints rank and status.
"""
import sys

import torch

import paper_1802_10453_gb300 as lr
from paper_1802_10453_gb300 import inputs_gpu


def main(argv):
    n = int(argv[1]) if len(argv) > 1 else 8192
    p = int(argv[2]) if len(argv) > 2 else 67108859
    path = lr.PATH_FP64 if (len(argv) > 3 and argv[3] == "fp64") else lr.PATH_TC
    r = n // 2
    A, _ = inputs_gpu.planted_matrix(n, r, r // 4, p, 12345)
    res = lr.factor(A, p, path=path)
    torch.cuda.synchronize()
    print("n", n, "p", p, "rank", int(res["rank"].item()), "status", int(res["status"].item()))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
