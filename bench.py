"""Benchmark of the mixed precision Gram-matrix thin SVD on GB300.

One step = one full pass of Algorithm 1 (Gram on the tensor cores, combine,
FP64 Jacobi, sort/cast, U) on one resident synthetic instance of the
4,194,304 x 64 FP32 workload (the configuration the headline metric is
quoted on).  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--no-cpu-baseline] [--no-plain] [--sharded | --replicas]

With torchrun (N > 1) the FP32 workloads run row-sharded (Sec. 4.2.1): every
rank holds its own m rows of an (N m) x n matrix, the Gram is formed with one
all-reduce MAX of the column exponents and one all-reduce SUM of the exact
integer limbs (NCCL), and every rank runs the n x n stage and its rows of U:
weak scaling.  --replicas runs independent instances instead; --sharded takes
the sharded path at N = 1 too (under torchrun with a one-rank NCCL group, so
the collectives run).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A GB/s per thin SVD, mixed vs all-FP64 on GB300, sigma rel err≤1e-5; %HBM peak"
DEFAULT_WORKLOAD = "ozaki_4194304x64_fp32"
# gram_tc, gram_combine, chol_piv, kappa (beside the Jacobi), onesided_jacobi, finish, compute_u_tc,
# finalize_info
KERNELS_PER_STEP = 8
# Arithmetic peaks measured on GB300 with the library's probe kernels (python -m
# paper_2603_11953_gb300.peaks; profiles/peaks_gb300.md); bench.py measures them again at run
# time and falls back to these only when the probe cannot run.
RECORDED_FP64_GFLOPS = 1251.7
RECORDED_FP32_TFLOPS = 78.1
# TF32 dense tensor rate per BF16 rate (nominal 1.1 / 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each stage's kernels, from
# the ncu --set full summaries in profiles/ (captured at m = 1,048,576 rows); stages whose traffic
# grows with m are scaled by m / 1,048,576.  None where no capture covers the stage.
NCU_TRAFFIC = {
    "ozaki_4194304x64_fp32": {"gram": (271.798528e6, True),          # gram_tc_kernel (+ combine 10 MB)
                              "eig": (0.10368e6, False),             # onesided_jacobi_kernel<1>
                              "compute_u": (482.920192e6, True)},    # compute_u_tc_kernel<1>
    "stress_16777216x32_fp64": {"gram": None,
                                "eig": (0.119296e6, False),          # eig_dd_kernel
                                "compute_u": (491.981568e6, True)},  # compute_u_kernel<double>
}
NCU_ROWS = 1048576


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return dict(hbm=float(p["hbm_gbs"]), bf16=float(p["bf16_tflops"]),
                    bf16_sus=float(p.get("bf16_tflops_sustained", p["bf16_tflops"])),
                    sm_max_mhz=float(p.get("sm_max_mhz", 2070.0)), src="measured")
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, sm_max_mhz=2070.0, src="fallback")


def arith_peaks(skip=False):
    """FP64 and FP32 FMA peaks of this GPU, measured now with the library's probe kernels."""
    if not skip:
        try:
            from paper_2603_11953_gb300 import peaks as P
            f64, t64 = P.probe("fp64_fma", 2000)
            f32, t32 = P.probe("fp32_fma", 20000)
            return {"fp64_gflops": f64 / (t64 * 1e-3) / 1e9, "fp32_tflops": f32 / (t32 * 1e-3) / 1e12,
                    "src": "measured now (probe kernels)"}
        except Exception as exc:  # noqa: BLE001 - reported in the line
            return {"fp64_gflops": RECORDED_FP64_GFLOPS, "fp32_tflops": RECORDED_FP32_TFLOPS,
                    "src": f"recorded (probe failed: {exc.__class__.__name__})"}
    return {"fp64_gflops": RECORDED_FP64_GFLOPS, "fp32_tflops": RECORDED_FP32_TFLOPS, "src": "recorded"}


def sample_accuracy(T, A, A_cpu, rows, m, n, working, higher, local, stream):
    """sigma of the mixed form and of the all-FP64 plain form on the first `rows` rows of A (the
    same rows the CPU baseline uses), against the oracle's double-double Algorithm 1 on them."""
    import numpy as np
    import torch
    import oracle
    from paper_2603_11953_gb300 import workloads
    ref = oracle.svd(workloads.to_numpy_colmajor(A_cpu, rows), higher=2)
    s_ref = ref["sigma_h"] + ref["sigma_h_lo"]
    out = {"sample": f"first {rows} rows", "reference": "oracle: exact Gram + double-double Jacobi",
           "oracle_status": int(ref["status"])}
    dev = A.device
    for name, kw, hi in (("mixed", {}, higher), ("fp64_plain", {"gram_variant": 1}, T.TSVD_FP64)):
        h, _ = T.tsvd_create(local, stream.cuda_stream, T.tsvd_opts(**kw))
        sig = torch.zeros(n, dtype=A.dtype, device=dev)
        V = torch.zeros(n, n, dtype=A.dtype, device=dev)
        info = torch.zeros(6, dtype=torch.int32, device=dev)
        T.tsvd_solve(h, A, rows, n, A.shape[0], working, hi, sig, V, n, None, 0, info)
        torch.cuda.synchronize(dev)
        T.tsvd_destroy(h)
        s = sig.double().cpu().numpy()
        out[f"sigma_max_rel_err_{name}"] = float(np.max(np.abs(s - s_ref) / s_ref))
        out[f"status_{name}"] = T.tsvd_status_string(int(info[0].item()))
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        if shutil.which("nvidia-smi") is None:
            return self
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits", "-lms", "100"],
                                     stdout=self.tmp, stderr=subprocess.DEVNULL)
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.tmp is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus, force=False):
    """RANK/LOCAL_RANK/WORLD_SIZE from the launcher; a process group for several ranks, or for one
    rank under a launcher when `force` (the row-sharded path then runs its collectives)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 or (force and "MASTER_ADDR" in os.environ):
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(A_cpu, m, n, rows, reps=1):
    """The oracle as it stands (single thread) on the first `rows` rows: FP64 n x n stage for
    FP32 inputs, double-double for FP64 inputs."""
    import numpy as np
    import oracle
    from paper_2603_11953_gb300 import workloads
    An = workloads.to_numpy_colmajor(A_cpu, rows)
    fp64 = An.dtype == np.float64
    t0 = time.perf_counter()
    for _ in range(reps):
        r = oracle.svd(An, higher=2 if fp64 else 1)
        oracle.rows_times(An, r["W_w"], np.arange(rows), 53 if fp64 else 24)
    dt = (time.perf_counter() - t0) / reps
    gbs = rows * n * An.itemsize / dt / 1e9
    return gbs, dt


def run_reference_batch(args):
    """--impl reference on the batched workload: the oracle over its first instances (the same
    instances, by seed, as the first ones of the 4096-instance batch) until about --ref-rows rows."""
    import numpy as np
    import oracle
    from paper_2603_11953_gb300 import workloads
    buf, metas = workloads.make_batch(count=8, device="cpu")
    picked, rows = [], 0
    for md in metas:
        if picked and rows >= args.ref_rows:
            break
        A = buf[md["offset"]:md["offset"] + md["lda"] * md["n"]].view(md["n"], md["lda"]).T[:md["m"]]
        picked.append(np.asfortranarray(A.numpy()))
        rows += md["m"]

    def one():
        t0 = time.perf_counter()
        for A in picked:
            r = oracle.svd(A, higher=1)
            oracle.rows_times(A, r["W_w"], np.arange(A.shape[0]), 24)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        one()
    tot = sum(one() for _ in range(args.steps))
    nbytes = sum(A.shape[0] * A.shape[1] * 4 for A in picked)
    gbs = args.steps * nbytes / tot / 1e9
    sample = f"the first {len(picked)} instances ({rows} rows) of {BATCH_WORKLOAD}: exact Gram + FP64 Jacobi + exact U"
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "instances_sample": len(picked), "rows_sample": rows},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    """--impl reference: the CPU oracle on a bounded sample of the workload."""
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    import torch
    from paper_2603_11953_gb300 import workloads
    if args.workload == BATCH_WORKLOAD:
        return run_reference_batch(args)
    spec = workloads.CONFIGS[args.workload]
    rows = args.ref_rows
    A, _ = workloads.make_config(spec, device="cpu", m=rows)
    for _ in range(args.warmup):
        cpu_baseline(A, rows, spec.n, min(rows, 2048))
    times = []
    for _ in range(args.steps):
        _, dt = cpu_baseline(A, rows, spec.n, rows)
        times.append(dt)
    tot = sum(times)
    gbs = args.steps * rows * spec.n * A.element_size() / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp32" if spec.dtype == torch.float32 else "fp64", "data": "synthetic",
            "config": {"workload": spec.name, "m_sample": rows, "n": spec.n, "m_full": spec.m},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {rows} rows of {spec.name}: exact Gram + "
                                       f"{'FP64' if spec.dtype == torch.float32 else 'double-double'} "
                                       "Jacobi + exact U rows"},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


BATCH_WORKLOAD = "batch_4096_ragged_fp32"


def run_batch(args):
    """The ragged batched workload: 4096 instances (m log-uniform in [1024, 65536], n from
    {8, 16, 24, 32, 48, 64}, lda = m rounded up to 4, 256-byte aligned bases in one buffer); one step
    is one tsvd_batch_solve over all of them (sigma, V and U)."""
    import numpy as np
    import torch
    import paper_2603_11953_gb300 as T
    from paper_2603_11953_gb300 import workloads

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    buf, metas = workloads.make_batch(count=args.batch_count, device=dev)
    count = len(metas)
    ms = [md["m"] for md in metas]
    ns = [md["n"] for md in metas]
    ldas = [md["lda"] for md in metas]
    base = buf.data_ptr()
    Ap = [base + 4 * md["offset"] for md in metas]
    Ubuf = torch.empty_like(buf)
    Up = [Ubuf.data_ptr() + 4 * md["offset"] for md in metas]
    sbuf = torch.zeros(sum(ns), device=dev)
    vbuf = torch.zeros(sum(n * n for n in ns), device=dev)
    so, vo = np.cumsum([0] + ns[:-1]), np.cumsum([0] + [n * n for n in ns[:-1]])
    Sp = [sbuf.data_ptr() + 4 * int(o) for o in so]
    Vp = [vbuf.data_ptr() + 4 * int(o) for o in vo]
    info = torch.zeros(6 * count, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    h, _ = T.tsvd_create(local, stream.cuda_stream, T.tsvd_opts(timing=max(3, min(args.steps, 1024))))

    def step():
        T.tsvd_batch_solve(h, count, Ap, ms, ns, ldas, T.TSVD_FP32, T.TSVD_FP64, Sp, Vp, ns, Up, ldas, info)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    status = T.tsvd_sync_status(h)
    barrier(world)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier(world)
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    stage_ms = T.tsvd_stage_ms_mean(h, min(args.steps, 1024))
    ms_step = ms_total / args.steps
    bytes_A = sum(m * n * 4 for m, n in zip(ms, ns))
    value = world * args.steps * bytes_A / (ms_total * 1e-3) / 1e9
    pk = peaks()
    inf = info.view(count, 6).cpu().numpy()
    sweeps = inf[:, 1]
    jac_flops = float(sum(n ** 3 / 3.0 + sw * (n * (n - 1) // 2) * 8 * n for n, sw in zip(ns, sweeps)))
    arp = arith_peaks(args.no_probe)
    gram_ms, eig_ms, u_ms = stage_ms[0], stage_ms[1], stage_ms[2]
    cands = {
        "gram": (gram_ms, {"bound": "hbm", "achieved": bytes_A / (gram_ms * 1e-3) / 1e9, "peak": pk["hbm"],
                           "unit": "GB/s"}),
        "jacobi": (eig_ms, {"bound": "alu", "achieved": jac_flops / (eig_ms * 1e-3) / 1e9,
                            "peak": arp["fp64_gflops"], "unit": "GFLOP/s"}),
        "compute_u": (u_ms, {"bound": "hbm", "achieved": 2.0 * bytes_A / (u_ms * 1e-3) / 1e9, "peak": pk["hbm"],
                             "unit": "GB/s"}),
    }
    dom = max(cands, key=lambda k: cands[k][0])
    rl = dict(cands[dom][1])
    rl.update(kernel=dom, frac=rl["achieved"] / rl["peak"], traffic=None, peak_source=pk["src"])
    # tensor-core Gram for instances TMA can load (16-byte aligned, lda % 4 == 0), else one
    # CUDA-core launch per padded width; then combine, eig + finish, U, statuses (2)
    cuda_core = {16 if n <= 16 else 32 if n <= 32 else 48 if n <= 48 else 64
                 for md, n in zip(metas, ns) if (4 * md["offset"]) % 16 or md["lda"] % 4}
    launches = 1 + len(cuda_core) + 1 + 2 + 1 + 2
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        done_bytes, k = 0, 0
        while k < count and time.perf_counter() - t0 < 10.0:
            md = metas[k]
            A_np = buf[md["offset"]:md["offset"] + md["lda"] * md["n"]].view(md["n"], md["lda"]).T[:md["m"]]
            A_np = np.asfortranarray(A_np.cpu().numpy())
            r = oracle.svd(A_np, higher=1)
            oracle.rows_times(A_np, r["W_w"], np.arange(md["m"]), 24)
            done_bytes += md["m"] * md["n"] * 4
            k += 1
        dt = time.perf_counter() - t0
        cpu = {"value": done_bytes / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"the first {k} instances of {BATCH_WORKLOAD}: exact Gram + FP64 Jacobi + exact U ({dt:.1f} s)"}
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "instances": count, "rows": int(sum(ms)),
                       "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (A is %.2f GB > 129 MB)" % (bytes_A / 1e9),
                       "status": T.tsvd_status_string(status)},
            "roofline": rl,
            "stages": {"gram_ms": gram_ms, "eig_ms": eig_ms, "u_ms": u_ms, "total_ms": stage_ms[3],
                       "sweeps_max": int(sweeps.max()), "sweeps_mean": float(sweeps.mean())},
            "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches * args.steps, "clocks": clk.summary()}
    T.tsvd_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=32768)
    ap.add_argument("--ref-rows", type=int, default=16384)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--sharded", action="store_true",
                    help="row-sharded solve (each rank's rows; one all-reduce of the exact Gram limbs); "
                         "the default with several ranks")
    ap.add_argument("--replicas", action="store_true", help="several ranks: independent replicas instead")
    ap.add_argument("--rows", type=int, default=0,
                    help="smaller m of the same workload (profiling captures); 0 = the workload's m")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == BATCH_WORKLOAD:
        return run_batch(args)

    import torch
    import paper_2603_11953_gb300 as T
    from paper_2603_11953_gb300 import workloads

    world, rank, local = dist_setup(args.gpus, force=args.sharded)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = workloads.CONFIGS[args.workload]
    m, n = (args.rows if args.rows > 0 else spec.m), spec.n
    A, meta = workloads.make_config(spec, device=dev, seed_offset=rank, m=m)
    esize = A.element_size()
    working = T.TSVD_FP32 if spec.dtype == torch.float32 else T.TSVD_FP64
    higher = T.TSVD_FP64 if working == T.TSVD_FP32 else T.TSVD_DD
    wdt = spec.dtype
    stream = torch.cuda.current_stream(dev)
    # per-stage events of every timed call (averaged over the timed region below)
    h, _ = T.tsvd_create(local, stream.cuda_stream, T.tsvd_opts(timing=max(3, min(args.steps, 1024))))
    sigma = torch.zeros(n, dtype=wdt, device=dev)
    V = torch.zeros(n, n, dtype=wdt, device=dev)
    U = torch.zeros(n, m, dtype=wdt, device=dev)
    info = torch.zeros(6, dtype=torch.int32, device=dev)

    # Row-sharded (Sec. 4.2.1): every rank holds its own m rows (seeded by rank) of a (world m) x n
    # matrix; the Gram is formed from one all-reduce MAX of the column exponents and one all-reduce
    # SUM of the exact integer limbs, every rank runs the n x n stage and its own rows of U.
    use_shard = (args.sharded or (world > 1 and not args.replicas)) and working == T.TSVD_FP32 and n <= 64
    gram_ev = []
    if use_shard:
        from paper_2603_11953_gb300 import sharded
        ops = sharded.LibraryOps(h, check=False)

        def step():
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            G = sharded.sharded_gram(A, m, n, m, ops)
            g1.record(stream)
            ops.solve(G, A, m, n, m, sigma, V, U, m, info)
            gram_ev.append((g0, g1))
    else:
        def step():
            T.tsvd_solve(h, A, m, n, m, working, higher, sigma, V, n, U, m, info)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    status = int(info[0].item())

    barrier(world)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier(world)
    ms_total = ev0.elapsed_time(ev1)
    # per-stage device times averaged over the timed steps (events the library recorded on
    # its stream around each stage of each call)
    stage_ms = T.tsvd_stage_ms_mean(h, min(args.steps, 1024))
    if use_shard:
        # the Gram stage (exponents, partial, both all-reduces, finish) from this loop's events
        gms = sum(a.elapsed_time(b) for a, b in gram_ev[-args.steps:]) / args.steps
        stage_ms = [gms, stage_ms[1], stage_ms[2], gms + stage_ms[3]]
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_step = ms_total / args.steps
    bytes_A = m * n * esize
    value = world * args.steps * bytes_A / (ms_total * 1e-3) / 1e9
    clocks = clk.summary()

    # end to end through the public API with host buffers (pinned): every step copies its A from
    # host memory, solves, and copies U, sigma and V back.  Steps alternate between two handles on
    # two streams (each with its own device buffers), so one step's copy back overlaps the next
    # step's upload and compute, as a caller streaming many matrices would run it.
    e2e = None
    if not args.no_e2e:
        A_host = torch.empty((n, m), dtype=wdt, pin_memory=True)
        A_host.copy_(A.T.reshape(n, m), non_blocking=False)
        NCS = 2  # copy streams per lane (4 streams and 8 chunks measured slower)
        lanes = []
        for _ in range(2):
            st_ = torch.cuda.Stream(dev)
            hh, _ = T.tsvd_create(local, st_.cuda_stream, T.tsvd_opts())
            lanes.append(dict(s=st_, h=hh, ops=sharded.LibraryOps(hh, check=False) if use_shard else None,
                              c=[torch.cuda.Stream(dev) for _ in range(NCS)],
                              A=torch.empty((n, m), dtype=wdt, device=dev),
                              U=torch.empty((n, m), dtype=wdt, device=dev), sig=torch.empty(n, dtype=wdt, device=dev),
                              V=torch.empty((n, n), dtype=wdt, device=dev),
                              info=torch.zeros(6, dtype=torch.int32, device=dev),
                              Uh=torch.empty((n, m), dtype=wdt, pin_memory=True),
                              sh=torch.empty(n, dtype=wdt, pin_memory=True),
                              Vh=torch.empty((n, n), dtype=wdt, pin_memory=True)))
        K = max(6, args.steps // 2)
        NCH = 4  # column chunks per copy, spread over the copy streams (more copy engines busy)
        bounds = [n * i // NCH for i in range(NCH + 1)]

        def e2e_step(k):
            L = lanes[k % 2]
            for i in range(NCH):
                with torch.cuda.stream(L["c"][i % NCS]):
                    L["A"][bounds[i]:bounds[i + 1]].copy_(A_host[bounds[i]:bounds[i + 1]], non_blocking=True)
            for c in L["c"]:
                L["s"].wait_stream(c)
            with torch.cuda.stream(L["s"]):
                if use_shard:
                    sharded.sharded_solve(L["A"].T, m, n, m, L["sig"], L["V"], L["ops"], L["U"], m, L["info"])
                else:
                    T.tsvd_solve(L["h"], L["A"], m, n, m, working, higher, L["sig"], L["V"], n, L["U"], m,
                                 L["info"])
            for c in L["c"]:
                c.wait_stream(L["s"])
            for i in range(NCH):
                with torch.cuda.stream(L["c"][i % NCS]):
                    L["Uh"][bounds[i]:bounds[i + 1]].copy_(L["U"][bounds[i]:bounds[i + 1]], non_blocking=True)
            with torch.cuda.stream(L["c"][0]):
                L["sh"].copy_(L["sig"], non_blocking=True)
                L["Vh"].copy_(L["V"], non_blocking=True)

        for k in range(2):
            e2e_step(k)
        torch.cuda.synchronize(dev)
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for L in lanes:
            L["s"].wait_event(e0)
            for c in L["c"]:
                c.wait_event(e0)
        for k in range(K):
            e2e_step(k)
        for L in lanes:
            stream.wait_stream(L["s"])
            for c in L["c"]:
                stream.wait_stream(c)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        ms_e2e = max_over_ranks(e0.elapsed_time(e1), world, dev) / K
        e2e_status = max(int(L["info"][0].item()) for L in lanes)
        e2e = {"value": world * bytes_A / (ms_e2e * 1e-3) / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": bytes_A, "d2h_bytes_per_step": bytes_A + n * esize + n * n * esize,
               "ms_per_step": ms_e2e, "steps": K, "streams": 2, "copy_chunks": NCH, "copy_streams": NCS,
               "status": T.tsvd_status_string(e2e_status)}
        for L in lanes:
            T.tsvd_destroy(L["h"])
        del A_host, lanes

    info_main = info.cpu()  # status, sweeps, off-norm, kappa(B) of the last timed step
    # the all-FP64 plain form of the same method (FP64 DFMA Gram, same n x n stage and U),
    # timed on the same resident A
    plain = None
    sig_mixed = sigma.double().cpu().numpy()
    if not args.no_plain and n <= 64:
        hp, _ = T.tsvd_create(local, stream.cuda_stream, T.tsvd_opts(timing=3, gram_variant=1))
        sig_p = torch.zeros_like(sigma)
        T.tsvd_solve(hp, A, m, n, m, working, T.TSVD_FP64, sig_p, V, n, U, m, info)
        torch.cuda.synchronize(dev)
        kp = 3
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(kp):
            T.tsvd_solve(hp, A, m, n, m, working, T.TSVD_FP64, sig_p, V, n, U, m, info)
        p1.record(stream)
        torch.cuda.synchronize(dev)
        pst = T.tsvd_stage_ms_mean(hp, kp)
        ms_plain = p0.elapsed_time(p1) / kp
        sp = sig_p.double().cpu().numpy()
        plain = {"value": bytes_A / (ms_plain * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms_plain,
                 "gram_ms": pst[0], "eig_ms": pst[1], "u_ms": pst[2], "speedup_mixed_vs_plain": ms_plain / ms_step,
                 "sigma_max_rel_diff_vs_mixed": float((abs(sp - sig_mixed) / sig_mixed).max()),
                 "status": T.tsvd_status_string(int(info[0].item()))}
        T.tsvd_destroy(hp)

    # the other eigen stage (two-sided Jacobi on M_h) and the other U (CUDA-core FP32 FMA),
    # each with everything else at its default, on the same resident A
    variants = {}
    if not args.no_variants and n <= 64 and working == T.TSVD_FP32:
        for name, kw in (("eig_two_sided", dict(eig_variant=1)), ("u_cuda_core_fp32", dict(u_variant=1)),
                         ("eig_alg2_fp32_svd_of_R", dict(eig_variant=3))):
            hv, _ = T.tsvd_create(local, stream.cuda_stream, T.tsvd_opts(timing=5, **kw))
            for _ in range(7):
                T.tsvd_solve(hv, A, m, n, m, working, higher, sigma, V, n, U, m, info)
            torch.cuda.synchronize(dev)
            vst = T.tsvd_stage_ms_mean(hv, 5)
            variants[name] = {"gram_ms": vst[0], "eig_ms": vst[1], "u_ms": vst[2], "total_ms": vst[3],
                              "status": T.tsvd_status_string(int(info[0].item()))}
            T.tsvd_destroy(hv)
        # the mixed precision Cholesky QR (Sec. 3.1) on the same A: Gram, FP64 Cholesky, Q by FP32
        # substitution (Q into U's buffer); it reads A twice and writes Q once
        hq, _ = T.tsvd_create(local, stream.cuda_stream, T.tsvd_opts())
        Rq = torch.zeros(n * n, dtype=torch.float64, device=dev)
        for _ in range(3):
            T.tsvd_cholqr(hq, A, m, n, m, working, T.TSVD_FP64, U, m, Rq, n, info)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(5):
            T.tsvd_cholqr(hq, A, m, n, m, working, T.TSVD_FP64, U, m, Rq, n, info)
        q1.record(stream)
        torch.cuda.synchronize(dev)
        ms_q = q0.elapsed_time(q1) / 5
        variants["cholqr_mixed"] = {"ms": ms_q, "value_GBps": bytes_A / (ms_q * 1e-3) / 1e9,
                                    "hbm_frac_of_traffic": 3 * bytes_A / (ms_q * 1e-3) / 1e9 / peaks()["hbm"],
                                    "status": T.tsvd_status_string(int(info[0].item()))}
        T.tsvd_destroy(hq)
    pk = peaks()
    arp = arith_peaks(args.no_probe)
    gram_ms, eig_ms, u_ms = stage_ms[0], stage_ms[1], stage_ms[2]
    sweeps = int(info_main[1].item())
    kappa_b = float(info_main.view(torch.float64)[2].item())
    nb = (n + 31) // 32
    if working == T.TSVD_FP64:
        # pieces Gram: one 64-column tensor-core pass per needed 32-column block pair of the m x 4NB
        # piece matrix; double-double n x n stage (about 20 FP64 operations per double-double
        # multiply-add); U = A W in FP64
        nbp = ((n + 31) // 32 * 32) // 32
        npass = sum(1 for b1 in range(4 * nbp) for b2 in range(b1 + 1, 4 * nbp) if b1 // nbp + b2 // nbp <= 3)
        gram_flops = npass * 16 * 2.0 * m * 64 * 64
        eig_flops = 20.0 * (n ** 3 / 3.0 + sweeps * (n * (n - 1) // 2) * 8 * n)
        u_terms = {"fp64": (2.0 * m * n * n / 1e9, arp["fp64_gflops"], "GFLOP/s")}
        launches = 2 + 2 * npass + 5  # colmax, split, npass x (gram_tc + combine), fold, eig_dd, finish, U, finalize
    else:
        passes = 1 if n <= 64 else nb * (nb - 1) // 2
        gram_flops = passes * 16 * 2.0 * m * 64 * 64  # 16 exact digit-pair products per 64-column pass
        if n <= 64:
            # pivoted Cholesky n^3/3, then per sweep every pair's dot product (2n) and rotation (6n)
            eig_flops = n ** 3 / 3.0 + sweeps * (n * (n - 1) // 2) * 8 * n
            # row-sharded: column maxima, exponents, limbs and finish instead of the combine
            launches = KERNELS_PER_STEP + (3 if use_shard else 0)
        else:
            # two-sided: per pair, rows and columns p, q of M (8n) and of V (6n)
            eig_flops = sweeps * (n * (n - 1) // 2) * 14.0 * n
            launches = 2 * passes + 4
        # tensor-core U: three TF32 products per output (A_hi W_hi, A_hi W_lo, A_lo W_hi)
        u_terms = {"tensor_tf32": (3 * 2.0 * m * n * n / 1e12, pk["bf16_sus"] * TF32_PER_BF16, "TFLOP/s")}
    u_terms["hbm"] = (2.0 * bytes_A / 1e9, pk["hbm"], "GB/s")
    gram_terms = {"hbm": (bytes_A / 1e9, pk["hbm"], "GB/s"), "tensor": (gram_flops / 1e12, pk["bf16_sus"], "TFLOP/s")}
    eig_terms = {"fp64": (eig_flops / 1e9, arp["fp64_gflops"], "GFLOP/s")}

    def stage_roofline(ms, terms):
        """Every term as achieved / peak; the binding term is the one with the largest floor."""
        out = {}
        for k, (work, peak, unit) in terms.items():
            ach = work / (ms * 1e-3)
            out[k] = {"achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                      "floor_ms": 1e3 * work / peak}
        bound = max(out, key=lambda k: out[k]["floor_ms"])
        return {"bound": bound, "ms": ms, "terms": out}

    stage_rl = {"gram": stage_roofline(gram_ms, gram_terms), "eig": stage_roofline(eig_ms, eig_terms),
                "compute_u": stage_roofline(u_ms, u_terms)}
    dom = max(stage_rl, key=lambda k: stage_rl[k]["ms"])
    bt = stage_rl[dom]["bound"]
    term = stage_rl[dom]["terms"][bt]
    rl = {"bound": {"hbm": "hbm", "tensor": "tensor", "tensor_tf32": "tensor"}.get(bt, "alu"),
          "achieved": term["achieved"], "peak": term["peak"], "unit": term["unit"], "frac": term["frac"],
          "kernel": dom, "term": bt}
    tr = NCU_TRAFFIC.get(spec.name, {}).get(dom)
    rl["traffic"] = None if tr is None else tr[0] * (m / NCU_ROWS if tr[1] else 1.0)
    rl["peak_source"] = pk["src"] if bt in ("hbm", "tensor", "tensor_tf32") else arp["src"]
    stages = {"gram_ms": gram_ms, "eig_ms": eig_ms, "u_ms": u_ms, "total_ms": stage_ms[3],
              "jacobi_sweeps": sweeps, "kappa_B_estimate": kappa_b, "rooflines": stage_rl,
              "variants": variants or None}

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = min(args.cpu_rows, m)
        A_cpu = A[:rows].cpu()
        gbs, dt = cpu_baseline(A_cpu, rows, n, rows)
        cpu = {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"first {rows} rows of {spec.name}: exact Gram + "
                         f"{'FP64' if working == T.TSVD_FP32 else 'double-double'} Jacobi + exact U rows "
                         f"({dt:.1f} s)"}
        if n <= 64:
            accuracy = sample_accuracy(T, A, A_cpu, rows, m, n, working, higher, local, stream)

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp32" if working == T.TSVD_FP32 else "fp64", "data": "synthetic",
            "config": {"workload": spec.name, "m": m, "n": n, "working": "fp32" if working == 0 else "fp64",
                       "higher": "fp64" if higher == 1 else "dd",
                       "parallelism": f"rowshard{world}" if use_shard else f"replicas{world}",
                       "eig": "pivoted Cholesky + one-sided Jacobi (FP64, 16-CTA cluster)" if n <= 64 and
                              working == T.TSVD_FP32 else "default for this shape",
                       "u": "tcgen05 3-term TF32 split" if working == T.TSVD_FP32 and n <= 64 else "CUDA cores",
                       "l2": "inputs larger than L2 (A is %.2f GB > 129 MB)" % (bytes_A / 1e9),
                       "status": T.tsvd_status_string(int(info_main[0].item()))},
            "roofline": rl, "stages": stages, "fp64_plain": plain, "accuracy": accuracy, "cpu_baseline": cpu,
            "e2e": e2e, "gpu_launches": launches * args.steps, "clocks": clocks, "arith_peaks": arp,
            "hbm_frac_of_A_stream": (bytes_A / (ms_step * 1e-3) / 1e9) / pk["hbm"]}
    T.tsvd_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
