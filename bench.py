"""Benchmark of the Fastfood feature map on GB300 (one JSON line on rank 0).

Workload (per GPU): N = 60000 MNIST-shaped rows (784 values, ~80% zeros,
others U[0,1), padded to d = 1024), E = 16 RBF expansions, sigma = 3,
Philox seed 42. One step = one fused feature pass over the batch:
60000 x 32768 float32 features (7.9 GB) written to HBM. Inputs (188 MB) and
outputs (7.9 GB) are larger than the 129 MB L2, so no flush is needed.

Reported:
  value      features/s of the whole job (all ranks), device-resident inputs
  e2e        the same metric through the C ABI with pinned host buffers, the
             host->device input copy and device->host feature copy inside
             the timed region
  roofline   the feature kernel's algorithmic bytes (784*4 read + 32768*4
             written per row) / its CUDA-event time, against the measured
             HBM copy bandwidth
  train_step config 3 (N=512, E=16, 10 classes): fused forward + adjoint
             backward vs the plain path (materialised features + torch linear
             + torch cross-entropy + adjoint from dphi), both at equal accuracy
  fused_logits softmax-ready logits of the same 60000-row batch without
             writing features
  fwht_sweep   config 2: the standalone transform over 1 GiB batches, d = 2^10..2^20
  uneven_batch config 4: 10000 vectors of mixed d, E and kernel in one persistent
               graph-launched kernel vs one launch per (d, E, kernel) class
  configs01    config 0 (256-row latency check), config 1 (60000 rows, E=8,
               RBF and Matern features and fused logits) and the headline at
               a power-of-2 batch (N = 2^16)
  feature_sweep the batched feature kernels at d = 2^5..2^15
  cpu_baseline the FP64 oracle on a bounded sample of the same workload, one
               spawned process per host core (the single-core figure inside),
               and the plain FP32 C program (cpu_baseline/) on every host core
               over the whole batch, with the host CPU model

--impl reference times the oracle itself (CPU, every host core) on the same
workload, as the reference arm.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

D, E, N, IN_DIM, SIGMA, SEED, C = 1024, 16, 60000, 784, 3.0, 42, 10
F = 2 * E * D
METRIC = "Fastfood features/sec at d=1024,E=16 (MNIST-shaped, 784 padded to 1024)"
WORKLOAD = {"workload": "fastfood_features_rbf", "d": D, "E": E, "in_dim": IN_DIM,
            "batch_per_gpu": N, "sigma": SIGMA, "seed": SEED,
            "l2": "inputs (188 MB) and outputs (7.9 GB) larger than L2; no flush"}
CPU_SAMPLE_ROWS = 1536
# Host-buffer path (e2e): rows per chunk and streams in flight.
E2E_CHUNK_ROWS, E2E_STREAMS, E2E_REPEATS = 2048, 4, 5


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--no-extras", action="store_true", help="skip train_step/fused_logits/e2e/cpu legs")
    p.add_argument("--batch", type=int, default=N,
                   help="rows per GPU (default 60000; smaller values are for profiling captures)")
    p.add_argument("--legs", default="all",
                   help="comma list of extra legs to run (e2e,logits,tc,train,sweep,uneven,configs01,fsweep) or 'all'")
    p.add_argument("--uneven-count", type=int, default=10000,
                   help="vectors in the config-4 leg (smaller values are for profiling captures)")
    return p.parse_args()


def fp32_peak_tflops(dev, mhz=2070.0):
    """SMs x 128 FP32 lanes x 2 (an FMA is two operations) x the maximum SM
    clock (2070 MHz on this GPU, the clock every bench run records)."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("features.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1702_08159_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            j = json.load(f)
        e = j.get(kernel)
        if e and e.get("source_hash") == kernel_source_hash():
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) taken during the timed region.

    Samples are read on a thread with host timestamps; ``mark_start`` and
    ``mark_end`` bracket the timed region and ``summary`` keeps the samples
    inside it (or the nearest one when the region is shorter than the
    sampling interval).
    """

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.samples = []
        self.t0 = self.t1 = None

    def __enter__(self):
        import threading

        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                self.samples.append((time.time(), line))

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        deadline = time.time() + 5.0
        while not self.samples and time.time() < deadline:
            time.sleep(0.01)
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()
        time.sleep(0.03)  # let the sample covering the end arrive

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        parsed = []
        for t, line in self.samples:
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                parsed.append((t, float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not parsed:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t0, t1 = self.t0 or parsed[0][0], self.t1 or parsed[-1][0]
        inside = [p for p in parsed if t0 <= p[0] <= t1]
        if not inside:
            inside = [min(parsed, key=lambda p: abs(p[0] - 0.5 * (t0 + t1)))]
        reasons = sorted({nm for p in inside for nm, v in zip(self.NAMES, p[3])
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(p[1] for p in inside), "sm_max_mhz": inside[0][2],
                "reasons": reasons, "samples_in_region": len(inside),
                "region_ms": 1e3 * (t1 - t0)}


_WORKER_TABLES = None


def _oracle_init(T):
    global _WORKER_TABLES
    _WORKER_TABLES = T


def _oracle_shard(x):
    """Worker of the all-core CPU runs: the oracle's features for one shard of
    rows, with the tables the pool was started with (a checksum comes back,
    not the features)."""
    from oracle import fastfood as ff

    return float(ff.features(x, _WORKER_TABLES).sum())


def oracle_pool(T):
    """One spawned process per host core, each holding the tables."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    return mp.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(T,)), cores


def cpu_baseline_all_cores(rows_per_core=CPU_SAMPLE_ROWS // 2):
    """The same oracle, unchanged, run on every host core at once, each process
    on its own shard of rows; the pool is started and warmed up before the
    timed map."""
    import workloads as wl
    from oracle import fastfood as ff

    T = ff.plan_tables(D, E, ff.RBF, SIGMA, seed=SEED)
    pool, cores = oracle_pool(T)
    x = wl.mnist_like(rows_per_core * cores, IN_DIM, seed=SEED).astype(np.float64)
    shards = [x[i * rows_per_core:(i + 1) * rows_per_core] for i in range(cores)]
    with pool:
        pool.map(_oracle_shard, [s[:2] for s in shards])  # start-up and imports
        t0 = time.perf_counter()
        pool.map(_oracle_shard, shards)
        dt = time.perf_counter() - t0
    return {"value": rows_per_core * cores * F / dt, "unit": "features/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{rows_per_core * cores} rows ({rows_per_core} per process), float64 numpy, {dt:.1f} s"}


def cpu_baseline_fp32(T, reps=3):
    """The plain FP32 CPU program (cpu_baseline/: iterative in-place FP32
    transform and feature map, samples split over POSIX threads) on every
    host core, over the whole 60000-row batch, each feature written to a
    2048-row wrap-around host buffer. Tables: the oracle's generator, rounded
    to float32. Best of `reps` passes; accuracy checked on 4 rows against
    the oracle."""
    import cpu_baseline as cb
    import workloads as wl
    from oracle import fastfood as ff

    tabs = (T["B"].astype(np.float32), T["perm"].astype(np.uint32),
            T["G"].astype(np.float32), T["Cs"].astype(np.float32))
    x = wl.mnist_like(N, IN_DIM, seed=SEED)
    out = np.empty((2048, F), np.float32)
    cores = os.cpu_count() or 1
    cb.features(x[:64], *tabs, threads=cores, out=out)  # load and fault in
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        cb.features(x, *tabs, threads=cores, out=out)
        times.append(time.perf_counter() - t0)
    dt = min(times)
    chk = cb.features(x[:4], *tabs, threads=1)
    T32 = dict(T, G=tabs[2].astype(np.float64), Cs=tabs[3].astype(np.float64))
    err = float(np.abs(chk - ff.features(x[:4].astype(np.float64), T32)).max())
    return {"value": N * F / dt, "unit": "features/s", "cores": cores, "kind": "plain_fp32_c",
            "gbs": N * (IN_DIM + F) * 4 / dt / 1e9, "seconds": dt,
            "sample": f"the whole {N}-row batch (d={D}, E={E}), float32 C, {cores} POSIX threads, "
                      f"best of {reps}", "max_abs_err_vs_oracle_4_rows": err}


def cpu_baseline(rows=CPU_SAMPLE_ROWS):
    """The FP64 oracle (as it stands, single thread) on `rows` rows of the workload."""
    import workloads as wl
    from oracle import fastfood as ff

    T = ff.plan_tables(D, E, ff.RBF, SIGMA, seed=SEED)
    x = wl.mnist_like(rows, IN_DIM, seed=SEED).astype(np.float64)
    t0 = time.perf_counter()
    ff.features(x, T)
    dt = time.perf_counter() - t0
    return {"value": rows * F / dt, "unit": "features/s", "cores": 1, "kind": "oracle",
            "sample": f"{rows} rows of the workload (d={D}, E={E}), float64 numpy, {dt:.1f} s"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as wl
    from oracle import fastfood as ff

    T = ff.plan_tables(D, E, ff.RBF, SIGMA, seed=SEED)
    pool, cores = oracle_pool(T)
    rows = 32 * cores  # per step: 32 rows on each host core
    x = wl.mnist_like(rows, IN_DIM, seed=SEED).astype(np.float64)
    shards = [x[i * 32:(i + 1) * 32] for i in range(cores)]
    with pool:
        for _ in range(max(1, args.warmup)):
            pool.map(_oracle_shard, shards)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_oracle_shard, shards)
        dt = time.perf_counter() - t0
    v = rows * F * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "features/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, reference_step_rows=rows),
            "cpu_baseline": {"value": v, "unit": "features/s", "cores": cores, "kind": "oracle",
                             "sample": f"{rows} rows per step (32 per host core), float64 numpy oracle"},
            "e2e": {"value": v, "unit": "features/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import torch.distributed as dist

    import paper_1702_08159_gb300 as mck
    import workloads as wl
    from paper_1702_08159_gb300 import build, dist as mdist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    build.build()

    nb = args.batch
    plan = mck.Plan(D, E, "rbf", SIGMA, SEED)
    x_host = wl.mnist_like(nb, IN_DIM, seed=SEED + rank)
    x = torch.from_numpy(x_host).to(dev)
    phi = torch.empty((nb, F), device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier(device_ids=[local])

    # The plan's launch shape, picked by the autotuner on this batch (every
    # shape gives the same bits); timed outside the measured region.
    from paper_1702_08159_gb300 import tune

    shape, shape_ms, _ = tune.tune_features(plan, x, out=phi, reps=3)
    for _ in range(args.warmup):
        mck.features(plan, x, out=phi)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        clk.mark_start()
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            mck.features(plan, x, out=phi)
            ev[i][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    barrier()
    ms_local = t_start.elapsed_time(t_end)
    ms = mdist.max_over_ranks(ms_local, device=dev)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    avg_launch_s = statistics.mean(launch_ms) / 1e3
    value = world * nb * F * args.steps / (ms / 1e3)

    bytes_per_row = IN_DIM * 4 + F * 4
    peak, peak_kind = measured_peaks()
    achieved = nb * bytes_per_row / avg_launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                "kernel": "k_feat_warp<10,0>", "bytes_per_launch": nb * bytes_per_row,
                "traffic": ncu_traffic("k_feat_warp<10,0>"),
                "frac_of_nominal_7900_gbs": achieved / 7900.0}
    # Context for the write-dominated kernel: what a plain store stream reaches
    # on this GPU (torch's fill of the same output buffer, no reads), outside
    # the timed region.
    for _ in range(3):
        phi.fill_(0.5)
    torch.cuda.synchronize()
    fill_ms = []
    for _ in range(5):
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_ev.record(stream)
        phi.fill_(0.5)
        b_ev.record(stream)
        torch.cuda.synchronize()
        fill_ms.append(a_ev.elapsed_time(b_ev))
    wgbs = phi.numel() * 4 / (statistics.median(fill_ms) / 1e3) / 1e9
    roofline["write_only_reference"] = {
        "gbs": wgbs, "frac_of_peak": wgbs / peak, "kernel": "torch Tensor.fill_ of the output buffer",
        "bytes": phi.numel() * 4, "feature_kernel_achieved_over_it": achieved / wgbs}

    line = {"metric": METRIC, "value": value, "unit": "features/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (MNIST-shaped stand-in, seeded)",
            "config": dict(WORKLOAD, batch_per_gpu=nb,
                           parallelism=f"dp{world} (samples sharded, no collective)"),
            "hbm_gbs": world * nb * bytes_per_row * args.steps / (ms / 1e3) / 1e9,
            "roofline": roofline, "clocks": clk.summary(), "gpu_launches": args.steps,
            "launch_shape": {"rows_per_item": shape[0], "staged": shape[1],
                             "tuned_ms": {f"{k[0]},{k[1]}": v for k, v in shape_ms.items()}},
            "launch_ms": {"mean": statistics.mean(launch_ms), "min": min(launch_ms),
                          "max": max(launch_ms)}}

    if not args.no_extras:
        legs = set(args.legs.split(",")) if args.legs != "all" else {
            "e2e", "logits", "tc", "train", "sweep", "uneven", "configs01", "fsweep"}
        if world > 1 and args.legs == "all":
            # Under torchrun every rank would repeat the single-GPU
            # characterisation legs; with N GPUs only the end-to-end number
            # (part of the contract at every N) is measured beside the headline.
            legs = {"e2e"}
        if "e2e" in legs:
            line["e2e"] = e2e_leg(mck, plan, x_host, dev, stream, world)
        if "logits" in legs:
            line["fused_logits"] = fused_logits_leg(mck, plan, x, dev, stream, args, phi)
        if "tc" in legs:
            line["features_tensor_core"] = tensor_core_features_leg(mck, plan, x, dev, stream, args,
                                                                    phi)
        if "train" in legs:
            line["train_step"] = train_step_leg(mck, dev, stream, args)
        if "sweep" in legs:
            line["fwht_sweep"] = fwht_sweep_leg(mck, dev, stream, args)
        if "uneven" in legs:
            line["uneven_batch"] = uneven_leg(mck, dev, stream, args)
        if "fsweep" in legs:
            line["feature_sweep"] = feature_sweep_leg(mck, dev, stream, args)
        if "configs01" in legs:
            line["configs01"] = configs01_leg(mck, dev, stream, args)
    del phi
    if rank == 0 and world == 1 and not args.no_extras:
        import cpu_baseline as cb
        from oracle import fastfood as ff

        one = cpu_baseline()
        try:
            line["cpu_baseline"] = cpu_baseline_all_cores()
            line["cpu_baseline"]["single_core"] = one
        except Exception as exc:  # a host without process spawning: one core only
            line["cpu_baseline"] = dict(one, all_cores_error=f"{type(exc).__name__}: {exc}"[:160])
        line["cpu_baseline"]["cpu_model"] = cb.cpu_model()
        try:
            line["cpu_baseline"]["plain_fp32_all_cores"] = cpu_baseline_fp32(
                ff.plan_tables(D, E, ff.RBF, SIGMA, seed=SEED))
        except Exception as exc:
            line["cpu_baseline"]["plain_fp32_all_cores"] = {
                "error": f"{type(exc).__name__}: {exc}"[:160]}
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def e2e_leg(mck, plan, x_host, dev, stream, world):
    """features/s through the public API with pinned host input and output:
    mck.features_host, which moves the batch in chunks over several streams
    (host-to-device copy, kernel, device-to-host copy per chunk)."""
    import torch

    from paper_1702_08159_gb300 import dist as mdist

    steps = 3
    xin = torch.from_numpy(x_host).pin_memory()
    out_host = torch.empty((N, F), dtype=torch.float32, pin_memory=True)
    phi = None
    pipe = mck.HostPipeline(plan, IN_DIM, E2E_CHUNK_ROWS, E2E_STREAMS)

    def step():
        mck.features_host(plan, xin, out=out_host, pipeline=pipe)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    # The host link is shared with whatever else the machine's host is moving
    # (other GPUs' jobs), so the timing is repeated and the median reported,
    # with every repetition beside it.
    reps = []
    for _ in range(E2E_REPEATS):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        reps.append(mdist.max_over_ranks(a.elapsed_time(b), device=dev))
    ms = statistics.median(reps)
    del out_host, phi, pipe
    return {"value": world * N * F * steps / (ms / 1e3), "unit": "features/s",
            "h2d_bytes_per_step": N * IN_DIM * 4, "d2h_bytes_per_step": N * F * 4,
            "steps": steps, "ms_per_step": ms / steps,
            "repetitions_ms_per_step": [r / steps for r in reps],
            "host_link_gbs": N * (IN_DIM + F) * 4 / (ms / steps / 1e3) / 1e9,
            "chunk_rows": E2E_CHUNK_ROWS, "streams": E2E_STREAMS}


def fused_logits_leg(mck, plan, x, dev, stream, args, phi):
    """Logits W phi + b of the headline batch without writing phi, against
    the unfused path on the same data: mck_features into the headline's
    feature buffer, then torch's FP32 addmm (TF32 off, the library's
    precision)."""
    import torch

    import workloads as wl

    W, b = wl.logit_weights(C, F, seed=SEED)
    Wd, bd = torch.from_numpy(W).to(dev), torch.from_numpy(b).to(dev)
    n = x.shape[0]
    out = torch.empty((n, C), device=dev)
    steps = max(3, args.steps // 4)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        e.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(e) / steps

    ms = timed(lambda: mck.fused_logits(plan, x, Wd, bd, out=out))
    out_tc = torch.empty_like(out)
    ms_tc = timed(lambda: mck.fused_logits(plan, x, Wd, bd, out=out_tc, prec="fp16_split"))
    diff_tc = float((out_tc - out).abs().max())
    ms_feat = timed(lambda: mck.features(plan, x, out=phi))
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        unfused = torch.empty_like(out)

        def plain():
            mck.features(plan, x, out=phi)
            torch.addmm(bd, phi, Wd.T, out=unfused)

        ms_unfused = timed(plain)
        ms_gemm = timed(lambda: torch.addmm(bd, phi, Wd.T, out=unfused))
        diff = float((unfused - out).abs().max())
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    # Algorithmic FP32 operations per row: the contraction (2 C 2Ed), the two
    # transforms (2 E d log2 d add/sub) and the G and Cs products (2 E d);
    # sin/cos not counted. Peak: SMs x 128 FP32 lanes x 2 (FMA) x SM clock.
    ops = 2 * C * F + 2 * E * D * int(np.log2(D)) + 2 * E * D
    tflops = n * ops / (ms / 1e3) / 1e12
    peak_t = fp32_peak_tflops(dev)
    hbm, _ = measured_peaks()
    # The best any unfused path could do: the feature kernel as measured, then
    # one read of phi at the measured copy bandwidth (the GEMM's floor).
    ideal_unfused = ms_feat + n * F * 4 / (hbm * 1e9) * 1e3
    return {"rows": n, "samples_per_s": n / (ms / 1e3), "features_per_s": n * F / (ms / 1e3),
            "ms_per_call": ms, "num_classes": C, "gpu_launches_per_call": 1,
            "tensor_core_fp16_split": {
                "ms_per_call": ms_tc, "samples_per_s": n / (ms_tc / 1e3),
                "speedup_vs_fp32_fused": ms / ms_tc, "max_abs_diff_vs_fp32_fused": diff_tc,
                "gpu_launches_per_call": 2,
                "path": "mck_fused_logits_ex(MCK_FP16_SPLIT): FP32 features, W phi on the "
                        "tensor cores (fp16 hi/lo x3, FP32 accumulation)"},
            "unfused": {"ms_per_call": ms_unfused, "ms_gemm_only": ms_gemm,
                        "path": "mck_features + torch FP32 addmm (TF32 off)",
                        "speedup_fused": ms_unfused / ms, "max_abs_diff_vs_fused": diff,
                        "ms_features_only": ms_feat,
                        "ms_ideal_unfused": ideal_unfused,
                        "ideal_unfused": "features as measured + one read of phi at the "
                                         "measured HBM copy bandwidth"},
            "alu": {"ops_per_row": ops, "achieved_tflops": tflops, "peak_tflops": peak_t,
                    "frac": tflops / peak_t, "bound": "alu (FP32)"}}


def tensor_core_features_leg(mck, plan, x, dev, stream, args, phi):
    """The headline batch through mck_features_ex with both transforms on the
    tensor cores (16-bit operands, FP32 accumulation, with and without the
    hi/lo split), against the FP32 butterfly kernel on the same batch. The
    accuracy against the FP64 oracle is held by tests/test_gpu_features_mma.py
    (fp16 hi/lo: the FP32 bar, 1e-5); here the largest difference from the
    FP32 kernel's features is reported beside the time."""
    import torch

    n = x.shape[0]

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        reps = max(5, args.steps // 5)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        e.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(e) / reps

    peak, _ = measured_peaks()
    bytes_ = n * (IN_DIM * 4 + F * 4)
    ms32 = timed(lambda: mck.features(plan, x, out=phi))
    ref = phi[:: max(1, n // 64)].clone()
    out = {"rows": n, "fp32_butterflies": {"ms": ms32, "gbs": bytes_ / (ms32 / 1e3) / 1e9,
                                           "frac_of_measured_hbm": bytes_ / (ms32 / 1e3) / 1e9 / peak}}
    for prec in ("fp16_split", "bf16_split", "fp16", "bf16"):
        ms = timed(lambda: mck.features(plan, x, out=phi, prec=prec))
        diff = float((phi[:: max(1, n // 64)] - ref).abs().max())
        out[prec] = {"ms": ms, "gbs": bytes_ / (ms / 1e3) / 1e9,
                     "frac_of_measured_hbm": bytes_ / (ms / 1e3) / 1e9 / peak,
                     "speed_vs_fp32": ms32 / ms, "max_abs_diff_vs_fp32_sampled_rows": diff}
    return out


def fwht_sweep_leg(mck, dev, stream, args):
    """Config 2: in-place transform of 1 GiB of N(0,1) float32 at d = 2^10..2^20.

    Per d: the mean CUDA-event time of one launch (input restored between
    launches), GB/s at 8 bytes per element (read + write once), the fraction
    of the measured HBM bandwidth, and the max error of sampled rows against
    the FP64 oracle relative to sqrt(d) * rms(x).
    """
    import torch

    import workloads as wl
    from oracle import fastfood as ff

    total = 1 << 28
    host = wl.gaussian(1, total, seed=SEED).reshape(-1)
    x0 = torch.from_numpy(host).to(dev)
    work = torch.empty_like(x0)
    peak, _ = measured_peaks()
    out = []
    for L in range(10, 21):
        d = 1 << L
        n = total // d
        rows = min(n, max(1, (1 << 22) // d))
        work.copy_(x0)
        mck.fwht_(work.view(n, d))
        torch.cuda.synchronize()
        got = work[: rows * d].view(rows, d).cpu().numpy().astype(np.float64)
        xin = host[: rows * d].reshape(rows, d).astype(np.float64)
        ref = ff.fwht(xin)
        rel = float(np.abs(got - ref).max() / (np.sqrt(d) * np.sqrt((xin ** 2).mean())))
        times = []
        for i in range(args.warmup + max(3, args.steps // 4)):
            work.copy_(x0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mck.fwht_(work.view(n, d))
            b.record(stream)
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(a.elapsed_time(b))
        ms = statistics.mean(times)
        gbs = 8.0 * total / (ms / 1e3) / 1e9
        rec = {"d": d, "batch": n, "ms": ms, "gbs": gbs, "frac_of_measured_hbm": gbs / peak,
               "passes": 1 if L <= 17 else 2, "max_err_rel_sqrt_d_rms": rel, "err_rows": rows}
        if L in (16, 17):  # the tunable regime: every candidate's time on this batch
            from paper_1702_08159_gb300 import tune

            work.copy_(x0)
            best, regime_ms, _ = tune.tune_fwht(work.view(n, d), reps=3)
            rec["regimes_ms"] = regime_ms
            rec["tuned_regime"] = best
        out.append(rec)
    # Tensor-core Kronecker-H16 forms (16-bit operands, FP32 accumulation) at
    # every d of the sweep: the tensor cores on each 1024-float block, FP32
    # column passes for the index bits above 10 when d > 1024.
    tc = []
    for L in range(10, 21):
        d = 1 << L
        n = total // d
        rows = min(n, max(1, (1 << 22) // d))
        xin = host[: rows * d].reshape(rows, d).astype(np.float64)
        ref = ff.fwht(xin)
        scale = np.sqrt(d) * np.sqrt((xin ** 2).mean())
        for prec in ("bf16", "fp16", "bf16_split", "fp16_split"):
            work.copy_(x0)
            mck.fwht_(work.view(n, d), prec)
            torch.cuda.synchronize()
            got = work[: rows * d].view(rows, d).cpu().numpy().astype(np.float64)
            rel = float(np.abs(got - ref).max() / scale)
            times = []
            for i in range(args.warmup + 3):
                work.copy_(x0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                mck.fwht_(work.view(n, d), prec)
                b.record(stream)
                torch.cuda.synchronize()
                if i >= args.warmup:
                    times.append(a.elapsed_time(b))
            ms = statistics.mean(times)
            gbs = 8.0 * total / (ms / 1e3) / 1e9
            tc.append({"d": d, "prec": prec, "ms": ms, "gbs": gbs,
                       "frac_of_measured_hbm": gbs / peak, "max_err_rel_sqrt_d_rms": rel,
                       "passes": 1 if L <= 10 else (2 if L <= 15 else 3)})
    del work, x0
    return {"dtype": "f32", "elements_per_d": total, "sizes": out, "tensor_core": tc}


def configs01_leg(mck, dev, stream, args):
    """Config 0 (256 rows, E=1, sigma=1: a latency check) and config 1 (60000
    rows, E=8, sigma=3, RBF and Matern t=40; features and fused 10-class logits)."""
    import torch

    import workloads as wl

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        e.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(e) / reps

    out = {}
    p0 = mck.Plan(D, 1, "rbf", 1.0, SEED)
    x0 = torch.from_numpy(wl.mnist_like(256, IN_DIM, seed=SEED)).to(dev)
    f0 = torch.empty((256, 2 * D), device=dev)
    ms = timed(lambda: mck.features(p0, x0, out=f0), 20)
    out["config0"] = {"rows": 256, "E": 1, "ms": ms, "features_per_s": 256 * 2 * D / (ms / 1e3)}
    p0.close()
    x1 = torch.from_numpy(wl.mnist_like(N, IN_DIM, seed=SEED)).to(dev)
    E1, F1 = 8, 2 * 8 * D
    f1 = torch.empty((N, F1), device=dev)
    W, b = wl.logit_weights(C, F1, seed=SEED)
    Wd, bd = torch.from_numpy(W).to(dev), torch.from_numpy(b).to(dev)
    lo = torch.empty((N, C), device=dev)
    peak, _ = measured_peaks()
    for kern in ("rbf", "matern"):
        pl = mck.Plan(D, E1, kern, 3.0, SEED, matern_t=40)
        ms = timed(lambda: mck.features(pl, x1, out=f1), max(3, args.steps // 5))
        ml = timed(lambda: mck.fused_logits(pl, x1, Wd, bd, out=lo), 3)
        ref = lo.clone()
        mt = timed(lambda: mck.fused_logits(pl, x1, Wd, bd, out=lo, prec="fp16_split"), 3)
        gbs = N * (IN_DIM * 4 + F1 * 4) / (ms / 1e3) / 1e9
        out[f"config1_{kern}"] = {"rows": N, "E": E1, "sigma": 3.0, "ms_features": ms,
                                  "features_per_s": N * F1 / (ms / 1e3), "gbs": gbs,
                                  "frac_of_measured_hbm": gbs / peak,
                                  "ms_fused_logits": ml, "logit_rows_per_s": N / (ml / 1e3),
                                  "ms_fused_logits_tensor_core": mt,
                                  "tensor_core_max_abs_diff": float((lo - ref).abs().max())}
        pl.close()
    del f1, x1
    # the headline at a power-of-2 batch (N = 2^16)
    n2 = 1 << 16
    x2 = torch.from_numpy(wl.mnist_like(n2, IN_DIM, seed=SEED)).to(dev)
    f2 = torch.empty((n2, F), device=dev)
    p2 = mck.Plan(D, E, "rbf", SIGMA, SEED)
    ms = timed(lambda: mck.features(p2, x2, out=f2), max(3, args.steps // 5))
    gbs = n2 * (IN_DIM * 4 + F * 4) / (ms / 1e3) / 1e9
    out["headline_pow2"] = {"rows": n2, "E": E, "ms_features": ms, "features_per_s": n2 * F / (ms / 1e3),
                            "gbs": gbs, "frac_of_measured_hbm": gbs / peak}
    p2.close()
    del f2, x2
    return out


def feature_sweep_leg(mck, dev, stream, args):
    """Batched feature kernels across d: RBF plans with E = 4, N(0,1) rows of
    length d, the batch sized to 1 GiB of features; mean CUDA-event time of a
    launch and GB/s of algorithmic traffic (x read once, features written)."""
    import torch

    import workloads as wl
    from paper_1702_08159_gb300 import tune

    out = []
    for L in range(5, 16):
        d, E = 1 << L, 4
        n = max(1, (1 << 28) // (2 * E * d))
        plan = mck.Plan(d, E, "rbf", 1.0, SEED)
        x = torch.from_numpy(wl.gaussian(n, d, seed=SEED + L)).to(dev)
        phi = torch.empty((n, 2 * E * d), device=dev)

        def timed():
            for _ in range(3):
                mck.features(plan, x, out=phi)
            torch.cuda.synchronize()
            reps = 5
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                mck.features(plan, x, out=phi)
            e.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(e) / reps

        ms_auto = timed()
        shape, shape_ms, _ = tune.tune_features(plan, x, out=phi, reps=3)
        ms = timed()
        gbs = n * (d + 2 * E * d) * 4 / (ms / 1e3) / 1e9
        out.append({"d": d, "E": E, "rows": n, "ms": ms, "gbs": gbs,
                    "frac_of_measured_hbm": gbs / measured_peaks()[0],
                    "ms_automatic_shape": ms_auto, "tuned_shape": list(shape),
                    "tuned_ms": {f"{k[0]},{k[1]}": v for k, v in shape_ms.items()}})
        plan.close()
        del x, phi
    return out


def uneven_leg(mck, dev, stream, args):
    """Config 4: 10000 vectors, d = 2^m (m ~ U{6..14}), E ~ U{1..32}, RBF or Matern
    (t = 40), sigma = 1, N(0,1) entries; plans keyed by (d, kernel) with 32
    expansions. One graph-launched persistent kernel (autotuned grain) vs one
    grouped launch per (d, E, kernel) class."""
    import torch

    import workloads as wl
    from paper_1702_08159_gb300.tune import tune_grain

    b = wl.uneven_batch(args.uneven_count, seed=SEED)
    keys = sorted(set(zip(b["d"].tolist(), b["kernel"].tolist())))
    plans, plan_s = [], {}
    for d, k in keys:
        # plan creation is synchronous (tables on the device, the skewed
        # gather search on the host at d = 1024); the Matern calibration costs
        # t d^2 normals per expansion
        t0 = time.perf_counter()
        plans.append(mck.Plan(d, 32, "rbf" if k == 0 else "matern", 1.0, SEED, matern_t=40))
        plan_s[f"{'rbf' if k == 0 else 'matern'}_d{d}"] = time.perf_counter() - t0
    pidx = np.array([keys.index((d, k)) for d, k in zip(b["d"].tolist(), b["kernel"].tolist())])
    order = np.lexsort((b["E"], b["kernel"], b["d"]))
    items, x_len, phi_len = mck.group_layout(plans, pidx, b["E"], b["d"], order)
    xh = np.zeros(x_len, np.float32)
    for i, v in enumerate(b["x"]):
        o = items["x_offset"][i]
        xh[o: o + len(v)] = v
    x = torch.from_numpy(xh).to(dev)
    phi = torch.empty(phi_len, device=dev)
    feats = int(phi_len)
    g = mck.Group(plans, items, x_len, phi_len)
    best, tune_ms = tune_grain(g, x, phi, reps=3)
    cap = mck.CapturedGroup(g, x, phi)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        e.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(e) / reps

    reps = max(3, args.steps // 5)
    ms_graph = timed(cap.replay, reps)
    ms_direct = timed(lambda: g.features(x, phi), reps)
    # baseline: one grouped launch per (d, E, kernel) class
    cls = {}
    for i in range(len(items)):
        cls.setdefault((int(b["d"][i]), int(b["E"][i]), int(b["kernel"][i])), []).append(i)
    groups = [mck.Group(plans, items[idx], x_len, phi_len) for idx in cls.values()]
    phi_b = torch.empty(phi_len, device=dev)

    def per_class():
        for grp in groups:
            grp.features(x, phi_b)

    ms_per_class = timed(per_class, reps)
    torch.cuda.synchronize()
    same = float((phi - phi_b).abs().max())
    out = {"vectors": len(items), "features": feats, "plans": len(plans),
           "classes": len(cls), "tuned_grain": best, "tune_ms": tune_ms,
           "ms_persistent_graph": ms_graph, "ms_persistent_direct": ms_direct,
           "ms_per_class_launches": ms_per_class,
           "features_per_s_persistent": feats / (ms_graph / 1e3),
           "speedup_vs_per_class": ms_per_class / ms_graph,
           "gb_per_s_written": 4.0 * feats / (ms_graph / 1e3) / 1e9,
           "max_abs_diff_vs_per_class": same, "info": g.info(),
           "plan_create_s_E32": plan_s}
    del phi, phi_b, x, cap, groups, g
    for pl in plans:
        pl.close()
    return out


def train_step_leg(mck, dev, stream, args):
    """Config 3: N=512, d=1024, E=16, 10 classes; fused vs plain fwd+bwd step time."""
    import torch

    import workloads as wl
    from paper_1702_08159_gb300.autograd import FastfoodFeatures, McKernelClassifier

    n = 512
    plan = mck.Plan(D, E, "rbf", 1.0, SEED)
    x = torch.from_numpy(wl.mnist_like(n, IN_DIM, seed=SEED)).to(dev)
    y = torch.from_numpy(wl.labels(n, C, seed=SEED)).to(dev)
    W, b = wl.logit_weights(C, F, seed=SEED)
    model = McKernelClassifier(plan, C, torch.from_numpy(W), torch.from_numpy(b))
    Cs = model.Cs.detach().clone().requires_grad_(True)
    G = model.G.detach().clone().requires_grad_(True)
    Wp = model.W.detach().clone().requires_grad_(True)
    bp = model.b.detach().clone().requires_grad_(True)

    def fused():
        for p in model.parameters():
            p.grad = None
        model.loss(x, y).backward()

    def plain():
        for p in (Cs, G, Wp, bp):
            p.grad = None
        phi = FastfoodFeatures.apply(plan, x, Cs, G)
        loss = torch.nn.functional.cross_entropy(phi @ Wp.T + bp, y.long())
        loss.backward()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        steps = max(5, args.steps)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        e.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(e) / steps

    def graphed(step, params):
        """The same step captured once in a CUDA graph (launch overhead removed)."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                step()  # leaves every parameter with a .grad to accumulate into
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for p in params:
                p.grad.zero_()
            step()
        return g.replay

    def fused_step():
        model.loss(x, y).backward()

    def plain_step():
        phi = FastfoodFeatures.apply(plan, x, Cs, G)
        torch.nn.functional.cross_entropy(phi @ Wp.T + bp, y.long()).backward()

    tf, tp = timed(fused), timed(plain)
    graph = {}
    try:
        graph["ms_fused_graph"] = timed(graphed(fused_step, list(model.parameters())))
        graph["ms_plain_graph"] = timed(graphed(plain_step, [Cs, G, Wp, bp]))
        graph["speedup_vs_plain_graph"] = graph["ms_plain_graph"] / graph["ms_fused_graph"]
    except Exception as exc:  # capture is an optional view of the same step
        graph["graph_error"] = f"{type(exc).__name__}: {exc}"[:200]
    # equal accuracy: the two paths' gradients agree
    fused()
    plain()
    torch.cuda.synchronize()
    dmax = max(float((model.W.grad - Wp.grad).abs().max() / Wp.grad.abs().max()),
               float((model.G.grad - G.grad).abs().max() / G.grad.abs().max()))
    plan.close()
    # ALU view of the fused step: 3 contractions (forward logits, dphi, dW: 2 C
    # 2Ed each) and 6 transforms (2 forward, 2 recomputed, 2 adjoint: E d
    # log2 d each) per row
    ops = 3 * 2 * C * F + 6 * E * D * int(np.log2(D))
    best = graph.get("ms_fused_graph", tf)
    alu = {"ops_per_row": ops, "achieved_tflops": n * ops / (best / 1e3) / 1e12,
           "peak_tflops": fp32_peak_tflops(dev)}
    alu["frac"] = alu["achieved_tflops"] / alu["peak_tflops"]
    return {"batch": n, "ms_fused": tf, "ms_plain": tp, "speedup_vs_plain": tp / tf, **graph,
            "alu_fused": alu,
            "grad_rel_diff_fused_vs_plain": dmax,
            "plain": "mck_features + torch matmul + torch cross_entropy + mck_features_backward"}


if __name__ == "__main__":
    main()
