"""Throughput benchmark of the BlockMGARD GPU path (one JSON line on stdout).

Workload: one 513^3 FP32 Gaussian random field with a k^-5/3 power spectrum
(unit variance, seeded), hybrid hierarchy with 17^3-node In-cache Blocks,
K = 2 in-cache levels and M = 2 global levels, uniform relative L-inf
tolerances 1e-2, 1e-3, 1e-4, 1e-5.  A step compresses the field once at each
of the four tolerances; `value` is input bytes of the step / step time
(compress GB/s over the sweep).  Decompression is timed the same way and
reported beside it, with the compression ratio and the L-inf check of every
tolerance.  The field (540 MB) is larger than the L2 cache, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload batch64    # 64 uneven fields: batched call vs per-field loop
  python bench.py --workload diff257    # differentiable recompose: forward + backward
  python bench.py --workload model      # Eq. 1 fit on this GPU, its knee, Alg. 1 choices
  python bench.py --workload roi385     # ROI error control: CR vs uniform 1e-5, L-inf per region

Under torchrun (N > 1) every rank compresses its own field (seed + rank): the
problems are independent, there is no collective on the data path, scaling
is weak and `value` is the sum over ranks of bytes / the max over ranks of
time.  `--impl reference` times the CPU oracle on a bounded sample of the
same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (513, 513, 513)
TOLS = (1e-2, 1e-3, 1e-4, 1e-5)
PARAMS = dict(block=17, levels=2, global_levels=2)
METRIC = "compress/decompress GB/s on 1 GB300, fraction of HBM peak, CR at L-inf bound"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler is producing lines
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0:
                time.sleep(0.005)
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dev):
    """The largest of a per-rank time over all ranks of the process group (x
    itself without one): whole-job throughput divides the units of every rank
    by the slowest rank's time."""
    import torch

    if torch.distributed.is_available() and torch.distributed.is_initialized() and \
            torch.distributed.get_world_size() > 1:
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t)
    return float(x)


def pipeline_roofline(field_bytes, n_symbols, stream_bytes, g_bytes, ms_per_call, peak):
    """Whole compress call against the HBM peak.  Algorithmic bytes, as the
    method defines them per input element: the field read once (s) and the
    stream written once (s/CR).  Beside them the planned traffic of this
    pipeline: the field read twice (max|u| and the block kernel), the 16-bit
    symbols written once and read twice (histogram, encoder), the
    block-coarse values G written and read once, the stream written once."""
    alg = field_bytes + stream_bytes
    planned = 2 * field_bytes + 3 * 2 * n_symbols + 2 * g_bytes + stream_bytes
    sec = ms_per_call * 1e-3
    return {"alg_bytes_per_call": alg, "ms_per_call": ms_per_call, "achieved": alg / sec / 1e9, "peak": peak,
            "unit": "GB/s", "frac": alg / sec / 1e9 / peak, "planned_bytes_per_call": planned,
            "planned_frac": planned / sec / 1e9 / peak}


def block_flops(B, K):
    """Floating-point operations of the In-cache Block decomposition of one
    block (interpolation, coefficients, the three restriction passes with the
    five-point band and both Thomas recurrences, the coarse correction and
    the quantiser's multiply-add), counted per level of N = B, (B+1)/2, ...
    nodes with C = (N+1)/2 coarse nodes:
      phase A, N^2 lines: 4C (coarse average) + N (differences) + 2(N-C)
               (odd-node interpolation) + 15C (band 10C, Thomas 5C)
      phase B, N C lines: 15C;  phase C, C^2 lines: 15C + C (correction)
      quantiser: 2 per coefficient (N^3 - C^3)."""
    n, total = B, 0
    for _ in range(K):
        c = (n + 1) // 2
        total += n * n * (4 * c + n + 2 * (n - c) + 15 * c) + n * c * 15 * c + c * c * 16 * c + 2 * (n ** 3 - c ** 3)
        n = c
    return total


def fp64_peak_tflops(dev):
    """Measured FP64 rate of this GPU: a cuBLAS DGEMM (4096^3, best of 3)."""
    import torch

    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize(dev)
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * 4096 ** 3 / (best * 1e-3) / 1e12


def whole_job_gbs(ws, bytes_per_rank, ms_max):
    """Weak-scaling aggregate: every rank's bytes over the slowest rank's time."""
    return ws * bytes_per_rank / (ms_max * 1e-3) / 1e9


def run_reference(args):
    """CPU oracle (FP64 C++, one thread) on a bounded sample of the workload."""
    import numpy as np

    import fields
    import oracle

    ws, rank, _ = _dist()
    if rank != 0:
        return
    n = args.ref_edge
    u = fields.power_law_grf((513, 513, 513), seed=2).numpy()[:n, :n, :n].copy()
    oracle.build()
    times = []
    crs = {}
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for tol in TOLS:
            s = oracle.compress(u, tol, rel=True, B=PARAMS["block"], K=PARAMS["levels"], M=PARAMS["global_levels"])
            crs[tol] = u.nbytes / s.size
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    bytes_step = u.nbytes * len(TOLS)
    sec = statistics.median(times)
    value = bytes_step / sec / 1e9
    sample = "%dx%dx%d corner of the 513^3 field (seed 2), %d tolerances per step" % (n, n, n, len(TOLS))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "grf513_f32_b17k2m2_tolsweep", "shape": [513, 513, 513], "sample_shape": [n, n, n],
                   "B": PARAMS["block"], "K": PARAMS["levels"], "M": PARAMS["global_levels"], "tols": list(TOLS),
                   "tol_mode": "relative to max|u|"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cr": {str(k): v for k, v in crs.items()},
    }
    print(json.dumps(line))


BLOCK_KERNEL_SOURCES = ("paper_2609_00205_gb300/csrc/bm_block.cuh", "paper_2609_00205_gb300/csrc/bm_common.cuh")


def kernel_source_digest():
    """sha256 over the sources of the In-cache Block kernel (staleness check of
    the DRAM counters recorded under profiles/)."""
    import hashlib
    h = hashlib.sha256()
    for rel in BLOCK_KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _profiled_traffic():
    """DRAM bytes per launch of the block kernel recorded by ncu (summary in
    profiles/), or None when absent or taken on other kernel sources."""
    prof = os.path.join(ROOT, "profiles", "block_fwd_grf513.md")
    if not os.path.exists(prof):
        return None
    vals = {}
    with open(prof) as f:
        for line in f:
            if ":" in line and line.lstrip("- ").split(":")[0].strip() in ("traffic_bytes_per_launch",
                                                                          "kernel_source_sha256"):
                k, v = line.lstrip("- ").split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256") != kernel_source_digest():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _cpu_model():
    """Host CPU model name (lscpu, else /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_worker(sub, barrier, queue):
    """One host core: the oracle on its own sample at every tolerance (the
    workers start together at a barrier; each reports its own wall time)."""
    import oracle

    oracle.build()
    barrier.wait()
    t0 = time.perf_counter()
    for tol in TOLS:
        oracle.compress(sub, tol, rel=True, B=PARAMS["block"], K=PARAMS["levels"], M=PARAMS["global_levels"])
    queue.put(time.perf_counter() - t0)


def _oracle_all_cores(u_np, edge, procs):
    """The oracle as it stands (single-threaded code) on every host core at
    once: `procs` processes, each compressing its own edge^3 sample of the
    field at the four tolerances; throughput = all bytes / the slowest."""
    import multiprocessing as mp

    import numpy as np

    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    queue = ctx.Queue()
    n = u_np.shape[0]
    offs = [((i * 97) % max(1, n - edge + 1), (i * 61) % max(1, n - edge + 1)) for i in range(procs)]
    ps = [ctx.Process(target=_oracle_worker, args=(np.ascontiguousarray(u_np[a:a + edge, b:b + edge, :edge]),
                                                     barrier, queue)) for a, b in offs]
    for p in ps:
        p.start()
    times = [queue.get(timeout=600) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    return procs * edge ** 3 * u_np.itemsize * len(TOLS) / max(times) / 1e9, max(times)


def _profiled_pipeline():
    """Measured DRAM bytes of every kernel of one compress call (ncu, summary
    under profiles/) over their summed duration, as a fraction of the peak;
    None when absent."""
    prof = os.path.join(ROOT, "profiles", "pipeline_dram_grf385.md")
    if not os.path.exists(prof):
        return None
    vals = {}
    with open(prof) as f:
        for line in f:
            if ":" in line and line.lstrip("- ").split(":")[0].strip() in ("pipeline_dram_bytes", "pipeline_kernel_ms",
                                                                          "pipeline_dram_frac", "kernel_source_sha256"):
                k, v = line.lstrip("- ").split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    try:
        return {"dram_bytes": float(vals["pipeline_dram_bytes"]), "kernel_ms": float(vals["pipeline_kernel_ms"]),
                "frac": float(vals["pipeline_dram_frac"]), "source": "profiles/pipeline_dram_grf385.md",
                "current": vals.get("kernel_source_sha256") == pipeline_source_digest()}
    except (KeyError, ValueError):
        return None


def pipeline_source_digest():
    """sha256 over every CUDA source of the library (staleness check of the
    whole-pipeline DRAM record)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2609_00205_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def cpu_baseline(u_np, edge, dev):
    """The CPU oracle timed on the host: one thread on an edge^3 corner, then
    every host core at once (one process per core, each on its own edge^3
    sample).  The one-thread run also gives the oracle's codes of the corner,
    against which the GPU's codes of the same corner are compared: flips
    within and outside the 1e-6 relative window of a bin edge, per tolerance."""
    import numpy as np
    import torch

    import oracle
    import paper_2609_00205_gb300 as bm

    sub = np.ascontiguousarray(u_np[:edge, :edge, :edge])
    B, K, M = PARAMS["block"], PARAMS["levels"], PARAMS["global_levels"]
    oracle.build()
    t0 = time.perf_counter()
    res = {}
    for tol in TOLS:
        res[tol] = oracle.compress(sub, tol, rel=True, B=B, K=K, M=M, want_codes=True)
    dt = time.perf_counter() - t0
    one = sub.nbytes * len(TOLS) / dt / 1e9
    # flips of the GPU's codes on the same corner
    flips = {}
    coef = oracle.decompose(sub.astype(np.float64), B, K, M)
    t = torch.from_numpy(sub).to(dev)
    for tol in TOLS:
        so, co = res[tol]
        sg = bm.compress(t, tol, mode="rel", **PARAMS)
        if oracle.stream_header(so)["raw"] or oracle.stream_header(sg.cpu().numpy())["raw"]:
            flips[str(tol)] = {"raw": True}
            continue
        cg = bm.stream_codes(sg).cpu().numpy().astype(np.int64)
        hq = oracle.stream_header(so)
        q = np.asarray(so[hq["off_qtab"]:hq["off_qtab"] + 8 * (K + M + 1)]).view(np.float64)
        p = oracle.plan(sub.shape, B, K, M)
        counts, n = [], B
        for _ in range(K):
            c = n // 2 + 1
            counts.append(n ** 3 - c ** 3)
            n = c
        qc = [np.tile(np.concatenate([np.full(c, q[l]) for l, c in enumerate(counts)]), p["nblocks"])]
        for l, c in enumerate(p["global_counts"]):
            qc.append(np.full(c, q[K + l]))
        qc.append(np.full(p["coarsest"], q[K + M]))
        qc = np.concatenate(qc)
        d = np.flatnonzero(cg != co)
        lo = np.minimum(cg[d], co[d])
        dist = np.abs(coef[d] - (lo + 0.5) * qc[d])
        win = (np.abs(cg[d] - co[d]) == 1) & (dist <= 1e-6 * np.maximum(np.abs(coef[d]), qc[d]))
        flips[str(tol)] = {"flips": int(d.size), "within_1e-6": int(win.sum()), "outside_1e-6": int((~win).sum()),
                           "codes": int(cg.size)}
    procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    try:
        allc, allc_s = _oracle_all_cores(u_np, edge, procs)
    except Exception as e:  # a reporting extra: keep the one-thread figure
        allc, allc_s, procs = None, None, 1
        print("all-core oracle leg failed: %s" % e, file=sys.stderr)
    cpu = _cpu_model()
    out = {"value": allc if allc else one, "unit": "GB/s", "cores": procs if allc else 1, "kind": "oracle",
           "cpu_model": cpu,
           "sample": ("%d processes (one per host core), each the oracle on its own %dx%dx%d sample of the same "
                      "field at the %d tolerances (%.1f s); one thread on the %dx%dx%d corner: %.4f GB/s (%.1f s)"
                      % (procs, edge, edge, edge, len(TOLS), allc_s or 0.0, edge, edge, edge, one, dt)),
           "single_thread_value": one,
           "flips_on_sample": flips}
    return out


def _batch64_fields(dev):
    """64 seeded power-law GRFs of uneven shapes and dtypes with their own
    relative tolerances (log-uniform in [1e-5, 1e-2]) and ROI maps (10 % of the
    blocks at a 10x tighter tolerance): 24 planar FP32 fields with sides
    U[100, 2049], 32 3-D FP32 fields with sides U[33, 257], 8 3-D FP64 129^3."""
    import numpy as np
    import torch

    import fields

    rng = np.random.default_rng(64)
    specs = []
    for _ in range(24):
        a, b = rng.integers(100, 2050, size=2)
        specs.append(((int(a), int(b)), torch.float32))
    for _ in range(32):
        specs.append((tuple(int(v) for v in rng.integers(33, 258, size=3)), torch.float32))
    for _ in range(8):
        specs.append(((129, 129, 129), torch.float64))
    out = []
    for i, (shape, dt) in enumerate(specs):
        u = fields.power_law_grf(shape, exponent=float(rng.uniform(-4.0, -1.5)), seed=1000 + i, dtype=dt,
                                 device=dev).contiguous()  # planar fields: a 2-D spectrum
        tol = float(10 ** rng.uniform(-5, -2))
        out.append((u, tol))
    return out


def _roi_maps(fs, block):
    import numpy as np

    rng = np.random.default_rng(65)
    maps = []
    for u, tol in fs:
        nb = int(np.prod([(int(s) + block - 1) // block for s in u.shape]))  # 1-D / 2-D: blocks of the field's dims
        r = np.full(nb, tol)
        r[rng.choice(nb, size=max(1, nb // 10), replace=False)] = tol / 10
        maps.append(r)
    return maps


def run_batch64(args):
    """The batched workload alone, as its own JSON line."""
    import torch

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    print(json.dumps(batch64_measure(dev, args.steps, args.warmup)))


def batch64_measure(dev, steps, warmup):
    """Batched compress of 64 fields vs the per-field loop (same fields,
    tolerances, ROI maps and parameters); the block size and in-cache levels
    are picked by timing each candidate on the batch."""
    import torch

    import paper_2609_00205_gb300 as bm

    bm.load()
    fs = _batch64_fields(dev)
    tols = [t for _, t in fs]
    us = [u for u, _ in fs]
    nbytes = sum(u.numel() * u.element_size() for u in us)
    outs = [torch.empty(bm.compress_bound(u.shape, u.dtype), dtype=torch.uint8, device=dev) for u in us]

    def batch(p, rois):
        return bm.compress_batch(us, tols, rois=rois, outs=outs, **p)

    def loop(p, rois):
        return [bm.compress(u, t, roi=r, out=o, **p) for u, t, r, o in zip(us, tols, rois, outs)]

    def timed(fn, p, rois, k):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record()
        for _ in range(k):
            fn(p, rois)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k, (time.perf_counter() - t0) * 1e3 / k

    # autotuner: block size (edges of 8, 16 and 32 cells are 9, 17 and 33
    # nodes; the paper's 8- and 16-node blocks too) and in-cache levels, one
    # timed batch per candidate
    cands = [dict(block=17, levels=2, global_levels=2), dict(block=9, levels=2, global_levels=2),
             dict(block=17, levels=1, global_levels=2), dict(block=9, levels=1, global_levels=2),
             dict(block=33, levels=2, global_levels=2), dict(block=16, levels=2, global_levels=2),
             dict(block=8, levels=2, global_levels=2)]
    tune = []
    for p in cands:
        rois = _roi_maps(fs, p["block"])
        batch(p, rois)
        tune.append((timed(batch, p, rois, 2)[0], p))
    best = min(tune, key=lambda z: z[0])[1]
    rois = _roi_maps(fs, best["block"])
    for _ in range(warmup):
        batch(best, rois)
        loop(best, rois)
    b_ms, b_wall = timed(batch, best, rois, steps)
    l_ms, l_wall = timed(loop, best, rois, steps)
    res = batch(best, rois)
    ref = loop(best, rois)
    same = all(torch.equal(x, y) for x, y in zip(res, ref))
    cr = nbytes / sum(x.numel() for x in res)
    line = {"metric": "batched compress GB/s, 64 uneven fields (input bytes / time)", "workload": "batch64",
            "value": nbytes / b_ms / 1e6, "unit": "GB/s", "higher_is_better": True,
            "ms_per_batch": b_ms, "wall_ms_per_batch": b_wall, "loop_ms": l_ms, "loop_wall_ms": l_wall,
            "speedup_vs_loop": l_ms / b_ms, "identical_streams": same, "cr": cr, "input_bytes": nbytes,
            "params": best, "tuning_ms": [[round(t, 3), p] for t, p in tune], "steps": steps,
            "warmup": warmup, "data": "synthetic",
            "fields": "24 planar FP32 sides U[100,2049], 32 3-D FP32 sides U[33,257], "
                      "8 3-D FP64 129^3; tolerances log-uniform [1e-5,1e-2], ROI 10% of blocks at 10x tighter",
            "path": "3-D fields with B in {9, 17}: max|u|, quantiser tables and In-cache Block stage in one "
                    "persistent launch per (dtype, B, K) draining a device work queue; other stages and fields "
                    "on the library's stream pool"}
    del fs, us, outs
    torch.cuda.empty_cache()
    return line


def run_diff257(args):
    """The differentiable workload alone, as its own JSON line."""
    import torch

    torch.cuda.set_device(0)
    print(json.dumps(diff257_measure(torch.device("cuda", 0), args.steps, args.warmup)))


def diff257_measure(dev, steps, warmup):
    """Differentiable recomposition on a 257^3 FP32 GRF: loss =
    ||recompose(c) - target||^2 + 0.1 ||grad_x recompose(c)||^2, forward and
    backward timed with CUDA events; the operators are linear, so their
    backward needs no saved level (peak memory is that of the loss)."""
    import torch

    import fields
    import paper_2609_00205_gb300 as bm

    bm.load()
    shape = (257, 257, 257)
    u = fields.power_law_grf(shape, seed=7, dtype=torch.float32, device=dev).contiguous()
    g = torch.Generator(device="cpu").manual_seed(8)
    target = u + 0.05 * torch.randn(shape, generator=g).to(dev)
    c0 = bm.decompose(u, **PARAMS)

    def step():
        c = c0.clone().requires_grad_(True)
        x = bm.recompose_ad(c, shape, **PARAMS)
        loss = ((x - target) ** 2).sum() + 0.1 * sum((torch.diff(x, dim=d) ** 2).sum() for d in range(3))
        loss.backward()
        return c.grad

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    base = torch.cuda.memory_allocated(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    peak = torch.cuda.max_memory_allocated(dev) - base
    # the same loss on a leaf tensor of the field's shape (no decomposition):
    # its autograd graph alone, for comparison with the peak above
    x0 = u.clone()

    def loss_only():
        x = x0.clone().requires_grad_(True)
        loss = ((x - target) ** 2).sum() + 0.1 * sum((torch.diff(x, dim=d) ** 2).sum() for d in range(3))
        loss.backward()
        return x.grad

    loss_only()
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    base2 = torch.cuda.memory_allocated(dev)
    loss_only()
    torch.cuda.synchronize()
    loss_peak = torch.cuda.max_memory_allocated(dev) - base2
    # the operator pair alone: recompose + its adjoint
    gx = torch.randn(shape, generator=g).to(dev)
    a.record()
    for _ in range(steps):
        bm.recompose(c0, shape, **PARAMS)
        bm.recompose_adjoint(gx, **PARAMS)
    b.record()
    torch.cuda.synchronize()
    op_ms = a.elapsed_time(b) / steps
    line = {"metric": "differentiable recompose, forward + backward ms (257^3 FP32)", "workload": "diff257",
            "value": ms, "unit": "ms", "higher_is_better": False, "recompose_plus_adjoint_ms": op_ms,
            "peak_extra_bytes": peak, "loss_only_peak_extra_bytes": loss_peak, "field_bytes": u.numel() * 4,
            "coeff_bytes": c0.numel() * 4, "steps": steps, "warmup": warmup,
            "peak_note": "torch allocations of the step; the library's operators save nothing for backward, and "
                         "the peak is the loss's own autograd tensors (loss_only_peak_extra_bytes, the same loss "
                         "on a leaf tensor) plus the coefficient tensor and its gradient",
            "params": PARAMS, "data": "synthetic",
            "saved_for_backward": "nothing (linear operators: the adjoint needs only the incoming gradient)"}
    return line


def region_errors(d, u, block_mask, block):
    """Max |d - u| over the nodes of ROI blocks and over the other nodes (block
    mask: one bool per block of ``block`` nodes per dimension, row-major)."""
    import numpy as np

    m = np.asarray(block_mask, dtype=bool)
    for ax in range(3):
        m = np.repeat(m, block, axis=ax)
    m = m[: u.shape[0], : u.shape[1], : u.shape[2]]
    e = np.abs(np.asarray(d, dtype=np.float64) - np.asarray(u, dtype=np.float64))
    return (float(e[m].max()) if m.any() else 0.0), (float(e[~m].max()) if (~m).any() else 0.0)


def roi385_measure(dev, steps, warmup):
    """ROI error control on the FP64 385x385x257 field (smooth k^-3 background,
    12 tanh fronts, 6 vortex tubes): ROI = blocks whose max |grad u| exceeds
    the 95th percentile of |grad u|, ROI tolerance 1e-5 and background 1e-2
    (relative to max|u|), B = 9, K = 2, M = 2.  The compression ratio against
    the same field at a uniform 1e-5, the L-inf error of each region against
    its tolerance, compress / decompress GB/s of both streams (CUDA events over
    `steps` calls each), and the FP64 block kernel against the measured FP64
    rate (its arithmetic, not HBM, bounds it on this GPU)."""
    import numpy as np
    import torch

    import fields
    import paper_2609_00205_gb300 as bm

    shape, B = (385, 385, 257), 9
    params = dict(block=B, levels=2, global_levels=2)
    u = fields.roi_field(shape, seed=3, device=dev).contiguous()
    un = u.cpu().numpy()
    mask = fields.gradient_roi(un, B)
    roi = np.where(mask, 1e-5, 1e-2).ravel()
    maxabs = float(np.abs(un).max())
    nbytes = u.numel() * u.element_size()
    out = torch.empty_like(u)
    stream = torch.cuda.current_stream(dev)
    cap = bm.compress_bound(shape, torch.float64)
    obuf = torch.empty(cap, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    res = {}
    for name, tol, r in (("roi", 1e-2, roi), ("uniform_1e-5", 1e-5, None)):
        s = bm.compress(u, tol, mode="rel", roi=r, **params).clone()
        c_ms = timed(lambda: bm.compress(u, tol, mode="rel", roi=r, out=obuf, **params))
        d_ms = timed(lambda: bm.decompress(s, out=out))
        bm.set_timing(True)
        bm.compress(u, tol, mode="rel", roi=r, out=obuf, **params)
        cst = dict(bm.stage_times())
        bm.decompress(s, out=out)
        dst = dict(bm.stage_times())
        bm.set_timing(False)
        d = bm.decompress(s, out=out).cpu().numpy()
        e_roi, e_bg = region_errors(d, un, mask, B)
        t_bg = tol * maxabs if r is not None else 1e-5 * maxabs
        res[name] = {"cr": nbytes / s.numel(), "stream_bytes": int(s.numel()), "compress_ms": c_ms,
                     "decompress_ms": d_ms, "compress_gbs": nbytes / c_ms / 1e6, "decompress_gbs": nbytes / d_ms / 1e6,
                     "max_err_roi": e_roi, "tol_roi": 1e-5 * maxabs, "max_err_background": e_bg,
                     "tol_background": t_bg, "bound_ok": e_roi <= 1e-5 * maxabs and e_bg <= t_bg,
                     "compress_stage_ms": cst, "decompress_stage_ms": dst}
    nblocks = int(mask.size)
    flops = nblocks * block_flops(B, params["levels"])
    k_ms = res["roi"]["compress_stage_ms"].get("incache_decompose", float("nan"))
    fp64 = fp64_peak_tflops(dev)
    return {"workload": "roi385_f64_b9k2m2", "shape": list(shape), "dtype": "f64", "params": params,
            "cr_ratio_roi_vs_uniform": res["roi"]["cr"] / res["uniform_1e-5"]["cr"], "roi_blocks": int(mask.sum()),
            "blocks": nblocks, "steps": steps, "warmup": warmup, "streams": res,
            "roofline": {"bound": "fp64_alu", "kernel": "block_fwd_kernel<double,9,2,0> (incache_decompose)",
                         "flops_per_launch": flops, "ms_per_launch": k_ms,
                         "achieved": flops / (k_ms * 1e-3) / 1e12, "peak": fp64, "unit": "TFLOP/s",
                         "frac": flops / (k_ms * 1e-3) / 1e12 / fp64,
                         "peak_kind": "measured (cuBLAS DGEMM 4096^3 on this GPU); nominal 1.25 TFLOP/s",
                         "hbm_frac": nbytes / (k_ms * 1e-3) / 1e9 / _peaks()[0]}}


def run_roi385(args):
    """The ROI workload alone (one JSON line)."""
    import torch

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    r = roi385_measure(dev, max(20, args.steps), args.warmup)
    line = {"metric": "ROI error control: CR with ROI vs uniform 1e-5, L-inf per region (385x385x257 FP64)",
            "workload": "roi385", "value": r["cr_ratio_roi_vs_uniform"], "unit": "x CR", "higher_is_better": True,
            "data": "synthetic", **r}
    print(json.dumps(line))


def run_model(args):
    """The performance-model workload alone, as its own JSON line."""
    import torch

    torch.cuda.set_device(0)
    print(json.dumps(model_measure()))


def model_measure():
    """Fit the performance model (Eq. 1 for the In-cache Block stage) on this
    GPU for both dtypes, report the knee (90 % of the saturated throughput)
    and Alg. 1's choice for the 513^3 workload under a few time budgets."""
    import paper_2609_00205_gb300 as bm
    import torch

    bm.load()
    out = {"metric": "performance model (Eq. 1) and Alg. 1 selection", "workload": "model", "data": "synthetic"}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        m = bm.perf_model_fit(dt, 17)
        d = m.as_dict()
        d["knee_blocks_90pct"] = bm.perf_model_knee(m, 0.9)
        d["tp_peak_gbs"] = m.block_peak_per_ms * 17 ** 3 * (4 if dt == torch.float32 else 8) / 1e6
        sel = {}
        for budget in (0.8, 1.2, 2.0, 5.0):
            try:
                p, t = bm.select_params(m, SHAPE, budget)
                sel[str(budget)] = {"params": p, "predicted_ms": t}
            except bm.BlockMGARDError as e:
                sel[str(budget)] = {"error": str(e)}
        d["alg1_513"] = sel
        out[name] = d
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--ref-edge", type=int, default=102)
    ap.add_argument("--cpu-edge", type=int, default=221)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-roi", action="store_true", help="skip the FP64 ROI workload in the main line")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-field batched workload in the main line")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the differentiable and performance-model workloads in the main line")
    ap.add_argument("--edge", type=int, default=513, help="field edge (513 = the workload; smaller for profiling)")
    ap.add_argument("--quick", action="store_true", help="compress steps only (profiling runs)")
    ap.add_argument("--workload", default="grf513", choices=["grf513", "batch64", "diff257", "model", "roi385"])
    args = ap.parse_args()
    if args.workload == "batch64" and args.impl == "gpu":
        return run_batch64(args)
    if args.workload == "diff257" and args.impl == "gpu":
        return run_diff257(args)
    if args.workload == "model" and args.impl == "gpu":
        return run_model(args)
    if args.workload == "roi385" and args.impl == "gpu":
        return run_roi385(args)
    global SHAPE
    SHAPE = (args.edge,) * 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import fields
    import paper_2609_00205_gb300 as bm

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bm.load()
    stream = torch.cuda.current_stream(dev)

    u = fields.power_law_grf(SHAPE, seed=2 + rank, dtype=torch.float32, device=dev).contiguous()
    nbytes = u.numel() * 4
    cap = bm.compress_bound(SHAPE, torch.float32)
    bufs = [torch.empty(cap, dtype=torch.uint8, device=dev) for _ in TOLS]
    out_field = torch.empty_like(u)
    maxabs = float(u.abs().max())

    def compress_all(timing=False):
        res = []
        for tol, b in zip(TOLS, bufs):
            s = bm.compress(u, tol, mode="rel", out=b, **PARAMS)
            st = bm.stage_times() if timing else None
            res.append((s, st))
        return res

    # correctness of what is timed: L-inf bound at every tolerance
    checks = {}
    for (s, _), tol in zip(compress_all(), TOLS):
        d = bm.decompress(s, out=out_field)
        err = float((d - u).abs().max())
        checks[tol] = {"cr": nbytes / s.numel(), "max_err_rel": err / maxabs, "bound_ok": err <= tol * maxabs}

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        compress_all()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = bm.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        compress_all()
    ev1.record(stream)
    barrier()
    launches = bm.launch_count() - l0
    clk = clocks.stop()
    comp_ms = ev0.elapsed_time(ev1) / args.steps
    # per-stage times (CUDA events the library records on the call's stream),
    # in separate untimed steps so that the events do not weigh on the number above
    stage_ms = {}
    bm.set_timing(True)
    for _ in range(max(2, args.steps // 4)):
        for (s, st) in compress_all(timing=True):
            for name, ms in st:
                stage_ms.setdefault(name, []).append(ms)
    bm.set_timing(False)
    comp_ms = max_over_ranks(comp_ms, dev)
    value = whole_job_gbs(ws, nbytes * len(TOLS), comp_ms)

    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": comp_ms, "quick": True,
                              "config": {"shape": list(SHAPE)},
                              "stage_ms": {k: statistics.mean(v) for k, v in stage_ms.items()},
                              "gpu_launches": launches, "clocks": clk}))
        return
    # decompression, same protocol
    streams = [s for s, _ in compress_all()]
    for _ in range(args.warmup):
        for s in streams:
            bm.decompress(s, out=out_field)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        for s in streams:
            bm.decompress(s, out=out_field)
    ev1.record(stream)
    barrier()
    decomp_ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev)
    decomp_gbs = whole_job_gbs(ws, nbytes * len(TOLS), decomp_ms)
    dstage = {}
    bm.set_timing(True)
    for _ in range(max(2, args.steps // 4)):
        for s in streams:
            bm.decompress(s, out=out_field)
            for name, ms in bm.stage_times():
                dstage.setdefault(name, []).append(ms)
    bm.set_timing(False)

    # per tolerance throughput (single compress / decompress)
    per_tol = {}
    for tol, b in zip(TOLS, bufs):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            s = bm.compress(u, tol, mode="rel", out=b, **PARAMS)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        c_ms = e0.elapsed_time(e1) / 3
        e0.record(stream)
        for _ in range(3):
            bm.decompress(s, out=out_field)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        d_ms = e0.elapsed_time(e1) / 3
        per_tol[str(tol)] = {"compress_gbs": nbytes / c_ms / 1e6, "decompress_gbs": nbytes / d_ms / 1e6,
                             "cr": checks[tol]["cr"], "max_err_rel": checks[tol]["max_err_rel"],
                             "bound_ok": checks[tol]["bound_ok"]}

    # end to end through the C ABI with host buffers: every step copies the
    # field from pinned host memory, compresses it at every tolerance and reads
    # every stream back to pinned host memory.  Steps are pipelined the way a
    # streaming application would run them: the next step's field is copied in
    # (second device buffer, own stream) and a stream is read back (copy
    # stream) while compressions run.
    host_in = torch.empty(SHAPE, dtype=torch.float32, pin_memory=True)
    host_in.copy_(u.cpu())
    host_out = [[torch.empty(cap, dtype=torch.uint8, pin_memory=True) for _ in TOLS] for _ in range(2)]
    dev_in = [torch.empty_like(u), torch.empty_like(u)]
    bufs2 = [bufs, [torch.empty(cap, dtype=torch.uint8, device=dev) for _ in TOLS]]
    copy_stream = torch.cuda.Stream(dev)
    h2d_stream = torch.cuda.Stream(dev)
    e2e_steps = max(4, args.steps // 2)

    def e2e_run(nsteps):
        """nsteps pipelined steps; returns (event pair, D2H bytes of the last step)."""
        d2h = 0
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h2d_done = [torch.cuda.Event(), torch.cuda.Event()]
        used = [torch.cuda.Event(), torch.cuda.Event()]  # last compression that read dev_in[k]
        d2h_done = [torch.cuda.Event(), torch.cuda.Event()]  # last read-back from bufs2[k]
        with torch.cuda.stream(h2d_stream):
            h2d_stream.wait_event(e0)
            dev_in[0].copy_(host_in, non_blocking=True)
            h2d_done[0].record(h2d_stream)
        for i in range(nsteps):
            k = i % 2
            if i + 1 < nsteps:  # next step's field, once its buffer's last reader is done
                with torch.cuda.stream(h2d_stream):
                    if i >= 1:
                        h2d_stream.wait_event(used[1 - k])
                    dev_in[1 - k].copy_(host_in, non_blocking=True)
                    h2d_done[1 - k].record(h2d_stream)
            stream.wait_event(h2d_done[k])
            if i >= 2:
                stream.wait_event(d2h_done[k])  # this step's output buffers have been read back
            d2h = 0
            for tol, b, ho in zip(TOLS, bufs2[k], host_out[k]):
                s = bm.compress(dev_in[k], tol, mode="rel", out=b, **PARAMS)
                done = torch.cuda.Event()
                done.record(stream)
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(done)
                    ho[: s.numel()].copy_(s, non_blocking=True)
                d2h += s.numel()
            used[k].record(stream)
            d2h_done[k].record(copy_stream)
        stream.wait_stream(copy_stream)  # the timed region ends when every stream is on the host
        e1.record(stream)
        barrier()
        return e0, e1, d2h

    # untimed warm-up over both buffer sets: the first transfers from and to
    # freshly pinned host pages are much slower than the steady state
    e2e_run(max(2, args.warmup))
    ev0, ev1, d2h = e2e_run(e2e_steps)
    e2e_ms = max_over_ranks(ev0.elapsed_time(ev1) / e2e_steps, dev)
    e2e = {"value": whole_job_gbs(ws, nbytes * len(TOLS), e2e_ms), "unit": "GB/s",
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": d2h,
           "pipelining": "step i+1's H2D and step i's D2H overlap the compressions (two buffer sets)"}

    # roofline of the dominant kernel (fused In-cache Block decompose +
    # quantise): algorithmic bytes of the step it performs, per input element
    # the field read once, plus the block-coarse values G it hands to the
    # global levels; the 16-bit symbols it writes for the entropy stage are
    # this pipeline's planned traffic and reported beside it
    peak, peak_kind = _peaks()
    k_ms = statistics.mean(stage_ms.get("incache_decompose", [float("nan")]))
    nb = [-(-n // PARAMS["block"]) for n in SHAPE]
    nblocks = nb[0] * nb[1] * nb[2]
    per_block = 17 ** 3 - 9 ** 3 + 9 ** 3 - 5 ** 3   # coefficients of the two in-cache levels
    g_vals = nblocks * 5 ** 3                          # block-coarse values handed to the global levels
    alg_bytes = nbytes + 4 * g_vals
    planned_bytes = nbytes + 2 * nblocks * per_block + 4 * g_vals
    achieved = alg_bytes / (k_ms * 1e-3) / 1e9
    traffic = _profiled_traffic()
    stage_avg = {k: statistics.mean(v) for k, v in stage_ms.items()}
    mean_stream = statistics.mean(nbytes / checks[t]["cr"] for t in TOLS)
    try:  # whole compress call: field read once + stream written once
        pipe = pipeline_roofline(nbytes, bm.coeff_count(SHAPE, **PARAMS), mean_stream, 4 * g_vals,
                                 comp_ms / len(TOLS), peak)
        pipe["dram_measured"] = _profiled_pipeline()
    except Exception as e:  # a reporting extra: never lose the bench line over it
        pipe = {"error": str(e)}
    # decompress: the inverse block kernel (reads G, writes the field), the
    # decoder (reads the stream) and the whole call (stream + field)
    dstage_avg = {k: statistics.mean(v) for k, v in dstage.items()}
    inv_ms = dstage_avg.get("incache_recompose", float("nan"))
    dec_ms = dstage_avg.get("huffman_decode", float("nan"))
    dcall_ms = decomp_ms / len(TOLS)
    dec_roof = {
        "bound": "hbm", "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
        "block_inv_kernel": {"alg_bytes_per_launch": nbytes + 4 * g_vals, "ms_per_launch": inv_ms,
                             "achieved": (nbytes + 4 * g_vals) / (inv_ms * 1e-3) / 1e9,
                             "frac": (nbytes + 4 * g_vals) / (inv_ms * 1e-3) / 1e9 / peak},
        "decode_kernel": {"alg_bytes_per_launch": mean_stream, "ms_per_launch": dec_ms,
                          "achieved": mean_stream / (dec_ms * 1e-3) / 1e9,
                          "frac": mean_stream / (dec_ms * 1e-3) / 1e9 / peak},
        "call": {"alg_bytes_per_call": nbytes + mean_stream, "ms_per_call": dcall_ms,
                 "achieved": (nbytes + mean_stream) / (dcall_ms * 1e-3) / 1e9,
                 "frac": (nbytes + mean_stream) / (dcall_ms * 1e-3) / 1e9 / peak},
    }
    roi = None
    if not args.no_roi:
        try:
            roi = roi385_measure(dev, max(20, args.steps), args.warmup)
        except Exception as e:  # a reporting extra: never lose the bench line over it
            roi = {"error": str(e)}
    b64 = None
    if not args.no_batch:
        try:
            b64 = batch64_measure(dev, 10, max(2, args.warmup))
        except Exception as e:  # a reporting extra: never lose the bench line over it
            b64 = {"error": str(e)}
    diff = model = None
    if not args.no_extras and not args.quick:
        try:
            diff = diff257_measure(dev, 10, 3)
        except Exception as e:  # a reporting extra: never lose the bench line over it
            diff = {"error": str(e)}
        try:
            model = model_measure()
        except Exception as e:
            model = {"error": str(e)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": comp_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "grf513_f32_b17k2m2_tolsweep", "shape": list(SHAPE), "B": 17, "K": 2, "M": 2,
                       "tols": list(TOLS), "tol_mode": "relative to max|u|", "spectrum": "k^-5/3",
                       "l2": "input 540 MB > 129 MB L2, no flush", "step": "compress at each of the 4 tolerances"},
            "decompress": {"value": decomp_gbs, "unit": "GB/s", "ms_per_step": decomp_ms,
                           "stage_ms": {k: statistics.mean(v) for k, v in dstage.items()}},
            "per_tol": per_tol,
            "roofline": {"bound": "hbm", "kernel": "block_fwd_kernel<float,17,2,0> (incache_decompose)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": traffic, "alg_bytes_per_launch": alg_bytes,
                         "planned_bytes_per_launch": planned_bytes,
                         "planned_frac": planned_bytes / (k_ms * 1e-3) / 1e9 / peak, "ms_per_launch": k_ms},
            "pipeline_roofline": pipe,
            "input_rate_frac": value / ws / peak,
            "decompress_roofline": dec_roof,
            "roi385": roi,
            "batch64": b64,
            "diff257": diff,
            "model": model,
            "stage_ms": stage_avg,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(u.cpu().numpy(), args.cpu_edge, dev)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
