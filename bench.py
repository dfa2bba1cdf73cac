#!/usr/bin/env python3
"""Benchmark: effective field-ops/s of the rank-profile-revealing PLDL^T mod p.

One step = one whole factorisation P^T A P = L D L^T of the n = 16384 planted
matrix (r = 8192, p = 2^26 - 5 = 67108859, A = T R T^T with 2048 pairs and
4096 fixed points), through the C ABI, inputs resident in HBM.  The operation
count is the paper's (Section 6): r^3/3 + n^2 r - r^2 n per factorisation.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  Multi-GPU runs are independent replicas (the
factorisation of one matrix does not shard); value = all ranks' ops / max time.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "effective Gfops/s of PLDL^T mod p, n=16384: INT8-limb vs FP64 form, bit-exact"
UNIT = "Gfops/s"
WORKLOAD = "planted_n16384_r8192_p67108859"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-form comparison line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-schedule line")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the n = 4096 uniform and n = 32768 all-pairs lines")
    return ap.parse_args()


def dist_env():
    from paper_1802_10453_gb300.replicas import dist_env as _env
    return _env()


def tc_digits(p):
    """Digit counts of the tensor-core update (csrc/syrdk_tc.cu): L_B signed
    base-256 digits with a top digit of magnitude <= 128 on the B side; on the
    A side base 512 (digits <= 256, at most 3) when that needs fewer digits."""
    h = (p - 1) // 2

    def count(base, half, top, lmax):
        for L in range(1, lmax + 1):
            low = sum(half * base ** u for u in range(L - 1))
            if (h + low) // base ** (L - 1) <= top:
                return L
        return None

    lb = count(256, 128, 128, 4)
    la = count(512, 256, 256, min(3, lb - 1)) if lb > 1 else None
    return lb, (la if la is not None else lb)


def effective_ops(n, r):
    n, r = float(n), float(r)
    return r ** 3 / 3.0 + n * n * r - r * r * n


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(A_host, p, seconds, draws=3):
    """The CPU oracle as it stands, on the same matrix, stopped after a number
    of pivots chosen so that `draws` runs take about `seconds` together; rate =
    sum over its pivot steps of m^2 (the per-step term of the Section 6
    operation count) / time.  value = the median draw; min and max give the
    spread."""
    from oracle import oracle as o
    t0 = time.perf_counter()
    o.ldlt_rpm(A_host, p, want_L=False, stop_after=8)
    t_cal = time.perf_counter() - t0
    per = max(t_cal / 8.0, 1e-4)
    k = int(max(8, min(4096, seconds / max(draws, 1) / per)))
    rates, total = [], 0.0
    for _ in range(max(draws, 1)):
        t0 = time.perf_counter()
        res = o.ldlt_rpm(A_host, p, want_L=False, stop_after=k)
        dt = time.perf_counter() - t0
        total += dt
        rates.append(res["ops"] / dt / 1e9)
    return {"value": statistics.median(rates), "unit": UNIT, "cores": o.max_threads(), "kind": "oracle",
            "sample": "first %d pivots of the same n=%d matrix (CPU oracle, right-looking Algorithm 4 "
                      "pivoting), %d draws; ops = sum of m^2 over those pivot steps; %.1f s in all"
                      % (k, A_host.shape[0], len(rates), total),
            "spread": {"min": min(rates), "max": max(rates), "draws": len(rates)},
            "seconds": total}


def cpu_one_core(seconds=3.0):
    """The oracle on one host core: the whole factorisation of the n = 256
    planted matrix, and a bounded sample (the first pivots, about `seconds`)
    of the n = 4096 uniform matrix; host-generated inputs of those workloads."""
    from oracle import oracle as o
    out = {}
    A0 = _host_matrix("planted_n256_r192_p65521")
    t0 = time.perf_counter()
    r0 = o.ldlt_rpm(A0, 65521, want_L=False, nthreads=1)
    dt = time.perf_counter() - t0
    out["planted_n256_r192_p65521"] = {"seconds": dt, "value": effective_ops(256, r0["rank"]) / dt / 1e9,
                                       "unit": UNIT, "sample": "whole factorisation"}
    A1 = _host_matrix("uniform_n4096_p8388593")
    t0 = time.perf_counter()
    o.ldlt_rpm(A1, 8388593, want_L=False, stop_after=8, nthreads=1)
    per = max((time.perf_counter() - t0) / 8.0, 1e-4)
    k = int(max(8, min(4096, seconds / per)))
    t0 = time.perf_counter()
    r1 = o.ldlt_rpm(A1, 8388593, want_L=False, stop_after=k, nthreads=1)
    dt = time.perf_counter() - t0
    out["uniform_n4096_p8388593"] = {"seconds": dt, "value": r1["ops"] / dt / 1e9, "unit": UNIT,
                                     "sample": "first %d pivots; ops = sum of m^2 over those steps" % k}
    out["cores"] = 1
    return out


def profile_traffic(kernel_src):
    """DRAM bytes (read + write) of SYRDK launches over their algorithmic
    bytes, from the committed ncu summary (the first three update launches of
    the bench workload, the largest ones, one ncu pass), if it was taken on the
    current kernel source (else None).  The bench scales it to its own
    launches by their algorithmic bytes."""
    path = os.path.join(ROOT, "profiles", "syrdk_tc_traffic_n16384.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    src = open(kernel_src, "rb").read()
    h = hashlib.sha256(src).hexdigest()[:16]
    m1 = re.search(r"kernel source sha256\[:16\]:\s*([0-9a-f]{16})", txt)
    m2 = re.search(r"traffic over algorithmic bytes:\s*([0-9.eE+]+)", txt)
    if not m1 or not m2 or m1.group(1) != h:
        return None
    return float(m2.group(1))


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_1802_10453_gb300 import inputs
    kind, n, r, p, all_pairs = inputs.WORKLOADS[args.workload]
    seed = inputs.SEED_BASE + list(inputs.WORKLOADS).index(args.workload)
    A_host = _host_matrix(args.workload)
    vals = []
    per_step_s = min(20.0, max(3.0, 90.0 / max(1, args.steps)))
    for s in range(args.steps):
        b = cpu_oracle_sample(A_host, p, per_step_s, draws=1)
        vals.append(b)
    v = statistics.median(x["value"] for x in vals)
    spread = {"min": min(x["value"] for x in vals), "max": max(x["value"] for x in vals), "draws": len(vals)}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32 (uint64 products, % p)",
            "data": "synthetic (seeded A = T R T^T)",
            "config": {"workload": args.workload, "n": n, "rank": r, "p": p},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"] + "; one draw per step", "spread": spread},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


_HOST_CACHE = {}


def _host_matrix(name):
    """The workload matrix on the host (drawn on the GPU when one is present)."""
    if name in _HOST_CACHE:
        return _HOST_CACHE[name]
    import numpy as np
    from paper_1802_10453_gb300 import inputs
    kind, n, r, p, all_pairs = inputs.WORKLOADS[name]
    seed = inputs.SEED_BASE + list(inputs.WORKLOADS).index(name)
    try:
        import torch
        if torch.cuda.is_available():
            from paper_1802_10453_gb300 import inputs_gpu
            A, _, _, _, _ = inputs_gpu.workload_matrix(name)
            out = np.tril(A.cpu().numpy()).astype(np.uint32)
            del A
            _HOST_CACHE[name] = out
            return out
    except Exception:
        pass
    if kind == "planted":
        A, _, _ = inputs.planted_matrix(n, r, inputs.default_pairs(r, all_pairs), p, seed)
    else:
        A = inputs.uniform_symmetric(n, p, seed)
    _HOST_CACHE[name] = A
    return A


def batched_bench(lr, inputs, inputs_gpu, dev, steps):
    """The batched schedule on the batch workload (4096 planted matrices, n in
    [32, 512]): one ldlt_rpm_factor_batched call per step, timed with CUDA
    events around the call (the inputs are restored from a device copy before
    each step, outside the events); the same call replayed from a captured CUDA
    graph; and the per-matrix loop of ldlt_rpm_factor on the first 256 matrices,
    scaled to the batch by effective operations."""
    import numpy as np
    import torch
    name = "batch4096_n32to512_p65521"
    count, n_lo, n_hi, p = inputs.BATCH_WORKLOADS[name]
    seed = inputs.SEED_BASE + 3
    ns, rs = inputs.batch_shapes(count, n_lo, n_hi, seed)
    batch = lr.Batch(ns, device=dev)
    partners = inputs_gpu.planted_batch(batch, rs, p, seed)
    src = batch.arena.clone()
    ops = float(sum(effective_ops(int(a), int(b)) for a, b in zip(ns, rs)))
    stream = torch.cuda.current_stream(dev)
    ws = torch.empty(lr.batched_workspace_bytes(count, p), dtype=torch.uint8, device=dev)

    def run_once():
        lr.factor_batched(batch, p, workspace=ws, stream=stream, check=False)

    tuned = lr.tune_batched(batch, p, reps=1, workspace=ws)  # restores the inputs

    for _ in range(2):
        batch.arena.copy_(src)
        run_once()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        batch.arena.copy_(src)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_once()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = sum(times) / len(times)
    ranks = batch.rank[:count].cpu().numpy()
    status_ok = int((batch.status[:count] != 0).sum().item()) == 0
    pa = batch.perm_arena.cpu().numpy()
    perms_ok, off = True, 0
    for i in range(count):
        n_i = int(ns[i])
        pr = partners[i]
        placed = np.zeros(n_i, dtype=bool)
        exp, zero = [], []
        for a in range(n_i):
            if placed[a]:
                continue
            b = pr[a]
            if b < 0:
                zero.append(a)
            elif b == a:
                exp.append(a); placed[a] = True
            else:
                exp += [a, int(b)]; placed[a] = placed[b] = True
        perms_ok = perms_ok and np.array_equal(pa[off:off + n_i], np.array(exp + zero))
        off += n_i
    parity = bool(status_ok and np.array_equal(ranks, rs) and perms_ok)

    graph_ms = None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            lr.factor_batched(batch, p, workspace=ws, stream=torch.cuda.current_stream(dev), check=False)
        gt = []
        for _ in range(steps):
            batch.arena.copy_(src)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            gt.append(e0.elapsed_time(e1))
        graph_ms = sum(gt) / len(gt)
        parity = parity and bool(np.array_equal(batch.rank[:count].cpu().numpy(), rs))
        del g
    except Exception as ex:  # capture unsupported in this environment
        graph_ms = {"unavailable": str(ex)[:200]}

    # per-matrix launch loop (the single-matrix entry point), bounded sample
    sub = 256
    batch.arena.copy_(src)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(sub):
        lr.factor(batch.matrix(i), p, check=False)
    torch.cuda.synchronize()
    loop_s = time.perf_counter() - t0
    ops_sub = float(sum(effective_ops(int(ns[i]), int(rs[i])) for i in range(sub)))
    loop_est_ms = loop_s * 1e3 * ops / ops_sub
    del ws, batch, src
    return {"workload": name, "matrices": count, "p": p, "value": ops / (ms * 1e-3) / 1e9, "unit": UNIT,
            "ms_per_batch": ms, "graph_ms_per_batch": graph_ms,
            "effective_ops": ops, "loop_ms_est": loop_est_ms,
            "loop_sample": "ldlt_rpm_factor on matrices 0..%d, %.1f ms, scaled by effective ops" % (sub - 1, loop_s * 1e3),
            "speedup_vs_loop": loop_est_ms / ms,
            "update_form": "mma.sync bf16 2-limb (p < 2^16)",
            "schedule": {"kb_ncut_kbsmall": list(tuned["best"]),
                         "tuned_ms": {str(list(k)): v for k, v in tuned["ms"].items()}},
            "parity": {"ranks_and_canonical_perms": parity}}


def graph_launches(panels):
    """Kernels one factorisation's graph launches: ingest, loop start and
    finalize, plus five per panel step (panel, L scatter, operand split,
    update, loop step); the while body holds two steps, so an odd panel
    count runs one more step whose kernels return at once."""
    steps = 2 * ((int(round(panels)) + 1) // 2)
    return 3 + 5 * steps


def workload_line(lr, inputs_gpu, name, dev, paths, reps, cpu_seconds, with_cpu):
    """Another workload of inputs.WORKLOADS, timed like the headline step (A
    restored from a device copy inside the CUDA events, inputs resident): per
    arithmetic form its effective Gfops/s, microseconds per pivot of the pivot
    chain and the SYRDK's fraction of the measured bf16 burst peak (limb
    products it issues / its CUDA-event time); the forms must agree bit for
    bit.  Beside it, the CPU oracle on a bounded sample of the same matrix."""
    import numpy as np
    import torch
    import ctypes
    A0, n, r_pl, p, partner = inputs_gpu.workload_matrix(name, device=dev)
    A = torch.empty_like(A0)
    stream = torch.cuda.current_stream(dev)
    L = lr.lib()
    pk, pk_kind = peaks()
    lb, la = tc_digits(p)
    out = {"workload": name, "n": n, "p": p}
    first = None
    for label, path in paths:
        try:
            ws = torch.empty(lr.workspace_bytes(n, p, path), dtype=torch.uint8, device=dev)
        except lr.LdltError as ex:
            out[label] = {"unavailable": str(ex)}
            continue
        for _ in range(2):
            A.copy_(A0)
            lr.factor(A, p, path=path, workspace=ws, check=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            A.copy_(A0)
            res = lr.factor(A, p, path=path, workspace=ws, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        # phases from one profiled pass (host loop, events per phase)
        L.ldlt_rpm_profile_reset()
        L.ldlt_rpm_profile_enable(1)
        A.copy_(A0)
        lr.factor(A, p, path=path, workspace=ws, check=False)
        torch.cuda.synchronize()
        L.ldlt_rpm_profile_enable(0)
        prof = (ctypes.c_double * 32)()
        L.ldlt_rpm_profile_read(prof)
        A.copy_(A0)
        res = lr.factor(A, p, path=path, workspace=ws, check=False)
        rk = int(res["rank"].item())
        ops = effective_ops(n, rk)
        syrdk_ms = prof[2]
        macs = prof[3]
        line = {"value": ops / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms, "rank": rk,
                "status": int(res["status"].item()), "reps": reps,
                "pivot_chain_ms": prof[0],
                "us_per_pivot": prof[0] * 1e3 / max(rk, 1),
                "syrdk_ms": syrdk_ms}
        if path == lr.PATH_TC and syrdk_ms > 0:
            tf = 2.0 * la * lb * macs / (syrdk_ms * 1e-3) / 1e12
            line["syrdk"] = {"achieved_tflops": tf, "peak": pk.get("bf16_tflops", 1900.0),
                             "frac": tf / pk.get("bf16_tflops", 1900.0),
                             "peak_source": "%s bf16 burst" % pk_kind,
                             "limb_products_per_mac": la * lb}
        elif syrdk_ms > 0:
            line["syrdk"] = {"gmac_per_s": macs / (syrdk_ms * 1e-3) / 1e9}
        rpm = lr.rpm_from_factor(res).cpu().numpy()
        if partner is not None:
            line["rpm_equals_planted"] = bool(np.array_equal(rpm, partner))
        snap = (torch.tril(A).clone(), res["perm"].clone(), res["e"].clone())
        if first is None:
            first = snap
        else:
            line["bit_exact_vs_%s" % paths[0][0]] = bool(torch.equal(snap[0], first[0]) and
                                                        torch.equal(snap[1], first[1]) and
                                                        torch.equal(snap[2], first[2]))
        out[label] = line
        del ws
    if with_cpu:
        A_host = np.tril(A0.cpu().numpy()).astype(np.uint32)
        cb = cpu_oracle_sample(A_host, p, cpu_seconds)
        out["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "spread")}
        del A_host
    del A, A0, first
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1802_10453_gb300 as lr
    from paper_1802_10453_gb300 import inputs, inputs_gpu

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    kind, n, r_planted, p, all_pairs = inputs.WORKLOADS[args.workload]
    A0, n, r_planted, p, partner = inputs_gpu.workload_matrix(args.workload, device=dev)
    A = torch.empty_like(A0)
    stream = torch.cuda.current_stream(dev)
    ws = torch.empty(lr.workspace_bytes(n, p, lr.PATH_TC), dtype=torch.uint8, device=dev)
    L = lr.lib()

    def step(path, wsb):
        A.copy_(A0)
        return lr.factor(A, p, path=path, workspace=wsb, check=False)

    for _ in range(args.warmup):
        res = step(lr.PATH_TC, ws)
    torch.cuda.synchronize()
    if int(res["status"].item()) != 0:
        raise SystemExit("device status %d" % int(res["status"].item()))
    rank_found = int(res["rank"].item())

    # timed region: the production path (one CUDA graph per factorisation,
    # nothing read back), inputs resident in HBM
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        res = step(lr.PATH_TC, ws)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    # phase breakdown: the same kernels from the profiling host loop (CUDA
    # events around each phase of each panel), a separate untimed pass
    psteps = max(1, min(args.steps, 3))
    import ctypes
    L.ldlt_rpm_profile_reset()
    L.ldlt_rpm_profile_enable(1)
    for _ in range(psteps):
        pres = step(lr.PATH_TC, ws)
    torch.cuda.synchronize()
    L.ldlt_rpm_profile_enable(0)
    prof = (ctypes.c_double * 32)()
    L.ldlt_rpm_profile_read(prof)
    prof = [v / psteps for v in prof]
    hbmp = (ctypes.c_double * 16)()
    L.ldlt_rpm_profile_read_hbm(hbmp)
    hbmp = [v / psteps for v in hbmp]
    if int(pres["status"].item()) != 0 or int(pres["rank"].item()) != rank_found:
        raise SystemExit("profiled pass disagrees with the timed one")
    from paper_1802_10453_gb300.replicas import max_over_ranks, whole_job_rate
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world, device=dev)
    ms_step = ms_total / args.steps
    ops = effective_ops(n, rank_found)
    value = whole_job_rate(ops, world, ms_step * 1e-3) / 1e9

    # parity of the timed output: R_A must be the planted supp(R)
    rpm = lr.rpm_from_factor(res).cpu().numpy()
    parity = bool(partner is not None and np.array_equal(rpm, partner) and int(res["status"].item()) == 0)

    # roofline of the dominant kernel (level-3 update on tensor cores)
    pk, pk_kind = peaks()
    limbs_b, limbs_a = tc_digits(p)
    syrdk_ms = prof[2]
    macs = prof[3]
    launches = prof[4]
    flops_issued_alg = 2.0 * limbs_a * limbs_b * macs
    achieved = flops_issued_alg / (syrdk_ms * 1e-3) / 1e12 if syrdk_ms > 0 else None
    # each launch runs for a fraction of a millisecond at full clock, so the
    # burst peak is the fair denominator; the sustained one is reported beside it
    peak = pk.get("bf16_tflops", 1900.0)
    peak_sus = pk.get("bf16_tflops_sustained", 1700.0)
    traffic_ratio = profile_traffic(os.path.join(ROOT, "paper_1802_10453_gb300", "csrc", "syrdk_tc.cu"))
    syrdk_alg_bytes = hbmp[12] / hbmp[13] if hbmp[13] else None  # per launch
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": (traffic_ratio * syrdk_alg_bytes
                            if (traffic_ratio is not None and syrdk_alg_bytes) else None),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the first three "
                                  "update launches of this workload (profiles/syrdk_tc_traffic_n16384.md) "
                                  "over their algorithmic bytes, times the algorithmic bytes per launch",
                "kernel": "syrdk_tc_kernel (bf16 limb tcgen05 SYRDK)",
                "peak_source": ("measured bf16 burst (MEASURED_PEAKS.json)" if pk_kind == "measured"
                                else "fallback bf16 burst 1.9 PFLOP/s"),
                "peak_sustained": peak_sus,
                "frac_of_sustained": (achieved / peak_sus) if achieved else None,
                "avg_launch_ms": syrdk_ms / launches if launches else None,
                "launches_per_step": launches,
                "alg_flops_per_step": flops_issued_alg,
                "alg_bytes_per_launch": syrdk_alg_bytes,
                "traffic_over_alg_bytes": traffic_ratio,
                "timing": "CUDA events around each launch in a profiled pass of %d step(s)" % psteps}

    # the HBM-streaming kernels: algorithmic bytes (counted by the library from
    # the launch sizes) over their CUDA-event time, against the measured copy peak
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    hbm_kernels = {}
    for i, name in enumerate(["ingest_kernel", "finalize_kernel", "lw_scatter_kernel", "split_tc_kernel"]):
        ms_k, nl, alg = hbmp[i], hbmp[4 + i], hbmp[8 + i]
        if ms_k > 0 and nl > 0:
            gbs = alg / (ms_k * 1e-3) / 1e9
            hbm_kernels[name] = {"launches": nl, "ms": ms_k, "alg_bytes": alg, "achieved_gbs": gbs,
                                 "frac": gbs / hbm_peak}
    hbm_kernels["peak_gbs"] = hbm_peak
    hbm_kernels["peak_source"] = ("measured copy (MEASURED_PEAKS.json)" if pk_kind == "measured"
                                  else "fallback 6.8 TB/s")
    hbm_kernels["timing"] = "CUDA events around each launch in the profiled pass (per step)"

    phases = {"pivot_chain_ms": prof[0], "operand_prep_ms": prof[1],
              "syrdk_ms": syrdk_ms, "panels": prof[6], "far_scans": prof[7],
              "source": "profiled pass (host loop, events per phase); the timed steps run the graph",
              "leader_ms": {k: prof[8 + i] / (clocks.get("sm_mhz") or 2070.0) / 1e3
                            for i, k in enumerate(["z_vector", "cand_column", "tail_1x1", "tail_scan",
                                                   "tail_2x2", "rollback", "waits_skips", "row_start"])},
              "chain_diag": {k: prof[16 + i] for i, k in enumerate(
                  ["rows", "pend_full_waits", "pend_full_cycles", "ring_wait_cycles", "rollbacks",
                   "helper1_idle_cycles", "helper1_busy_cycles", "helper1_events", "pub_batches",
                   "events", "t0_wait_b1", "t0_wait_b2", "t511_wait_b1", "t511_wait_b2", "t0_schur",
                   "t511_schur"])}}
    # the cycle counters exist only in a build with LDLT_CHAIN_PROFILE; drop the empty ones
    phases["leader_ms"] = {k: v for k, v in phases["leader_ms"].items() if v} or None
    phases["chain_diag"] = {k: v for k, v in phases["chain_diag"].items() if v}
    # the pivot chain is latency-bound: its figure is time per decision
    phases["us_per_pivot"] = phases["pivot_chain_ms"] * 1e3 / max(rank_found, 1)
    phases["us_per_row_iteration"] = phases["pivot_chain_ms"] * 1e3 / max(phases["chain_diag"]["rows"], 1.0)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hA = torch.empty((n, n), dtype=torch.int32, pin_memory=True)
        hA.copy_(A0.cpu())
        hL = torch.empty((n, n), dtype=torch.int32, pin_memory=True)
        hperm = torch.empty(n, dtype=torch.int32, pin_memory=True)
        he = torch.empty(n, dtype=torch.int32, pin_memory=True)
        hr = torch.empty(1, dtype=torch.int64, pin_memory=True)
        e_steps = max(1, min(args.steps, 3))
        for it in range(1 + e_steps):
            if it == 1:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            A.copy_(hA, non_blocking=True)
            rr = lr.factor(A, p, path=lr.PATH_TC, workspace=ws, check=False)
            hL.copy_(A, non_blocking=True)
            hperm.copy_(rr["perm"], non_blocking=True)
            he.copy_(rr["e"], non_blocking=True)
            hr.copy_(rr["rank"], non_blocking=True)
            torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / e_steps
        e2e = {"value": ops * world / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": n * n * 4,
               "d2h_bytes_per_step": n * n * 4 + 8 * n + 8, "ms_per_step": dt * 1e3}
        del hA, hL

    # the FP64 form on the same matrix, same device (comparison line)
    fp64 = None
    if not args.no_fp64 and rank == 0:
        try:
            A_tc = A.clone()
            ws64 = torch.empty(lr.workspace_bytes(n, p, lr.PATH_FP64), dtype=torch.uint8, device=dev)
            step(lr.PATH_FP64, ws64)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r64 = step(lr.PATH_FP64, ws64)
            e1.record(stream)
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1)
            rpm64 = lr.rpm_from_factor(r64).cpu().numpy()
            same = bool(torch.equal(torch.tril(A), torch.tril(A_tc)) and np.array_equal(rpm64, rpm)
                        and torch.equal(r64["perm"], res["perm"]) and torch.equal(r64["e"], res["e"]))
            fp64 = {"value": ops / (ms64 * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms64,
                    "bit_exact_vs_tc_form": same}
            del ws64, A_tc
        except lr.LdltError as ex:
            fp64 = {"unavailable": str(ex)}

    # consumer: A X = B with the factor of the timed step (n = 16384)
    solve_line = None
    if rank == 0:
        sv = {}
        for nrhs in (1, 64):
            Bd = torch.randint(0, p, (n, nrhs), dtype=torch.int32, device=dev)
            wsv = torch.empty(4 * n * nrhs, dtype=torch.uint8, device=dev)
            lr.solve(A, res, Bd, workspace=wsv, check=False)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                lr.solve(A, res, Bd, workspace=wsv, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_sv = e0.elapsed_time(e1) / 3
            # L is read once forward and once backward: 2 * 4 * n(n-1)/2 bytes
            gbs = 4.0 * n * (n - 1) / (ms_sv * 1e-3) / 1e9
            sv[str(nrhs)] = {"ms": ms_sv, "L_read_GBps": gbs}
        solve_line = {"n": n, "by_nrhs": sv, "form": "blocked forward/backward substitution, 64-row blocks",
                      "note": "random B (consistency not required for timing)"}

    # given-P mode: the same matrix refactored with the timed step's order and blocks
    given_line = None
    if rank == 0:
        gperm, gstarts, grank = res["perm"].clone(), res["e"].clone(), int(res["rank"].item())
        wsg = torch.empty(lr.given_workspace_bytes(n, p, lr.PATH_TC), dtype=torch.uint8, device=dev)
        ms_g = []
        for it in range(4):
            A.copy_(A0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gres = lr.factor_given(A, p, gperm, gstarts, grank, stream=stream, workspace=wsg, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            if it:
                ms_g.append(e0.elapsed_time(e1))
        ms_gv = statistics.median(ms_g)
        given_line = {"ms": ms_gv, "value": ops / (ms_gv * 1e-3) / 1e9, "unit": UNIT,
                      "status": int(gres["status"].item()),
                      "form": "P^T A P gathered in the ingest pass, same GPU path, structure checked"}
        # the order of the recursive Algorithms 2/3, read off R_A on the host,
        # then the given-P mode in that order
        t0 = time.perf_counter()
        rpm_h = lr.rpm_from_factor(res).cpu().tolist()
        rperm, rstarts, rrank = lr.recursive_order(rpm_h)
        host_ms = (time.perf_counter() - t0) * 1e3
        ms_r = []
        for it in range(3):
            A.copy_(A0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rres = lr.factor_given(A, p, rperm, rstarts, rrank, stream=stream, workspace=wsg, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            if it:
                ms_r.append(e0.elapsed_time(e1))
        given_line["recursive_order"] = {"ms": statistics.median(ms_r), "host_order_ms": host_ms,
                                         "status": int(rres["status"].item()),
                                         "rpm_equals_planted": bool(
                                             (lr.rpm_from_factor(rres).cpu().numpy() == partner).all())
                                         if partner is not None else None}
        del wsg

    # Algorithm 1 (TRSS): X^T U + U^T X = C at n = 4096 over the paper's 23-bit prime
    trss_line = None
    if rank == 0:
        nt, pt = 4096, 8388593
        gen = torch.Generator(device=dev)
        gen.manual_seed(1802)
        Ut = torch.randint(0, pt, (nt, nt), dtype=torch.int32, device=dev, generator=gen).triu_()
        Ut.diagonal().copy_(torch.randint(1, pt, (nt,), dtype=torch.int32, device=dev, generator=gen))
        C0 = torch.randint(0, pt, (nt, nt), dtype=torch.int32, device=dev, generator=gen)
        Ct = torch.empty_like(C0)
        wst = torch.empty(lr.trss_workspace_bytes(nt, pt), dtype=torch.uint8, device=dev)
        forms = {}
        for tensor in (True, False):
            ms_t = []
            for it in range(4):
                Ct.copy_(C0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st_t = lr.trss(Ut, Ct, pt, stream=stream, check=False, tensor=tensor, workspace=wst)
                e1.record(stream)
                torch.cuda.synchronize()
                if it:
                    ms_t.append(e0.elapsed_time(e1))
            forms[tensor] = (statistics.median(ms_t), int(st_t.item()), torch.triu(Ct).clone())
        ms_tr = forms[True][0]
        macs = nt ** 3 / 3.0  # the SYR2K updates dominate: sum over blocks of b (n - k)^2
        trss_line = {"n": nt, "p": pt, "ms": ms_tr, "gmac_per_s": macs / (ms_tr * 1e-3) / 1e9,
                     "status": forms[True][1],
                     "form": "blocked right-looking (64-row blocks), one launch per block for the "
                             "diagonal TRSS (X = M U with M from V^T C V, V = U_kk^-1 precomputed), the "
                             "panel TRMM+TRSM (a warp per column) and the update's limb operands, then "
                             "the trailing SYR2K on tcgen05 (bf16 limbs, exact) for orders >= 256, "
                             "CUDA cores below",
                     "cuda_core_form": {"ms": forms[False][0], "status": forms[False][1]},
                     "bit_exact_vs_cuda_core_form": bool(torch.equal(forms[True][2], forms[False][2]))}
        del wst, forms

    batched = None
    if rank == 0 and not args.no_batched:
        batched = batched_bench(lr, inputs, inputs_gpu, dev, max(3, min(args.steps, 10)))

    configs = None
    if rank == 0 and not args.no_configs:
        configs = {
            "uniform_n4096_p8388593": workload_line(
                lr, inputs_gpu, "uniform_n4096_p8388593", dev, [("tc", lr.PATH_TC), ("fp64", lr.PATH_FP64)],
                5, 4.0, world == 1 and not args.no_cpu),
            "planted_n32768_r16384_p2147483647_pairs": workload_line(
                lr, inputs_gpu, "planted_n32768_r16384_p2147483647_pairs", dev, [("tc", lr.PATH_TC)],
                2, 6.0, world == 1 and not args.no_cpu)}

    cpu = None
    cpu1 = None
    if rank == 0 and world == 1 and not args.no_cpu:
        A_host = np.tril(A0.cpu().numpy()).astype(np.uint32)
        cb = cpu_oracle_sample(A_host, p, args.cpu_seconds)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "spread")}
        cpu1 = cpu_one_core()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 (8-bit balanced limbs, fp32 accumulate) over u32 residues",
            "data": "synthetic (seeded A = T R T^T, GPU generator)",
            "config": {"workload": args.workload, "n": n, "rank": rank_found, "p": p,
                       "limbs": {"a_side": limbs_a, "b_side": limbs_b}, "path": "tcgen05 bf16-limb",
                       "l2": "inputs larger than L2 (1 GiB matrix); A restored from a device copy each step (inside the timed region)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "parity": {"rpm_equals_planted": parity},
            "phases": phases,
            "roofline": roofline,
            "hbm_kernels": hbm_kernels,
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": graph_launches(prof[6]) * args.steps,
            "fp64_form": fp64,
            "batched": batched,
            "configs": configs,
            "solve": solve_line,
            "trss": trss_line,
            "given_p": given_line,
            "cpu_baseline": cpu,
            "cpu_one_core": cpu1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
