"""One factorisation (or one batched call) for profiling under ncu.

    python -m paper_1802_10453_gb300.profile_case N [p] [fp64] [host]
    python -m paper_1802_10453_gb300.profile_case WORKLOAD_NAME [host]
    python -m paper_1802_10453_gb300.profile_case batch COUNT
    python -m paper_1802_10453_gb300.profile_case trss N [p]

The first form draws A = T R T^T (n = N, rank N/2, a quarter of R's non-zeros
in 2x2 pairs, p = 2^26 - 5 unless given) on the GPU; the second draws the named
workload of inputs.WORKLOADS exactly as bench.py does; both factor it once
through the C ABI, as one CUDA graph, or with `host` from the profiling host
loop (the same kernels launched one by one from the host, one readback per
panel), which is what the ncu captures of single kernels use; it also prints
the algorithmic bytes of the level-3 update launches.  The third draws the first COUNT matrices of the batch
workload (n in [32, 512], p = 65521) and factors them in one batched call.
The fourth solves one TRSS (Algorithm 1) of order N (random upper triangular
U with a non-zero diagonal, random symmetric C; p = 8388593 unless given).
Prints rank(s) and status.
"""
import sys

import torch

import paper_1802_10453_gb300 as lr
from paper_1802_10453_gb300 import inputs, inputs_gpu


def main(argv):
    arg = argv[1] if len(argv) > 1 else "8192"
    if arg == "batch":
        count = int(argv[2]) if len(argv) > 2 else 1024
        _, n_lo, n_hi, p = inputs.BATCH_WORKLOADS["batch4096_n32to512_p65521"]
        seed = inputs.SEED_BASE + 3
        ns, rs = inputs.batch_shapes(4096, n_lo, n_hi, seed)
        ns, rs = ns[:count], rs[:count]
        batch = lr.Batch(ns)
        inputs_gpu.planted_batch(batch, rs, p, seed)
        lr.factor_batched(batch, p)
        ok = bool((batch.rank[:count].cpu() == torch.from_numpy(rs)).all())
        print("batch", count, "p", p, "ranks as planted", ok)
        return 0 if ok else 1
    if arg == "trss":
        n = int(argv[2]) if len(argv) > 2 else 2048
        p = int(argv[3]) if len(argv) > 3 else 8388593
        g = torch.Generator(device="cuda")
        g.manual_seed(1802)
        U = torch.randint(0, p, (n, n), dtype=torch.int32, device="cuda", generator=g).triu_()
        U.diagonal().copy_(torch.randint(1, p, (n,), dtype=torch.int32, device="cuda", generator=g))
        C = torch.randint(0, p, (n, n), dtype=torch.int32, device="cuda", generator=g)
        st = lr.trss(U, C, p, check=False)
        torch.cuda.synchronize()
        print("trss n", n, "p", p, "status", int(st.item()))
        return 0 if int(st.item()) == 0 else 1
    host = "host" in argv[2:]
    argv = [a for a in argv if a != "host"]
    if arg in inputs.WORKLOADS:
        A, n, _, p, _ = inputs_gpu.workload_matrix(arg)
        path = lr.PATH_TC
    else:
        n = int(arg)
        p = int(argv[2]) if len(argv) > 2 else 67108859
        path = lr.PATH_FP64 if (len(argv) > 3 and argv[3] == "fp64") else lr.PATH_TC
        r = n // 2
        A, _ = inputs_gpu.planted_matrix(n, r, r // 4, p, 12345)
    if host:
        lr.lib().ldlt_rpm_profile_reset()
        lr.lib().ldlt_rpm_profile_enable(1)
    res = lr.factor(A, p, path=path)
    torch.cuda.synchronize()
    if host:
        lr.lib().ldlt_rpm_profile_enable(0)
    print("n", n, "p", p, "rank", int(res["rank"].item()), "status", int(res["status"].item()))
    if host:
        import ctypes
        hb = (ctypes.c_double * 16)()
        lr.lib().ldlt_rpm_profile_read_hbm(hb)
        # the level-3 updates' algorithmic bytes (old lower triangle read, new
        # one written, operands once) and their launches, for the ncu traffic ratio
        print("update_alg_bytes %.6e update_launches %d first_three_alg_bytes %.6e"
              % (hb[12], int(hb[13]), hb[14]))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
