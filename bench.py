#!/usr/bin/env python
"""Benchmark of batched HPS leaf static condensation on one B300 per rank.

Workload: the p = 20 unit-square problem (64 x 64 = 4096 leaves, A_ii of
324 x 324, kappa = 200, b = 1 - 0.5 exp(-|x - (0.5, 0.5)|^2 / 0.02), one body
load of 16 seeded Gaussian bumps), synthetic and resident in HBM.

A step is one hps_condense call over all 4096 leaves (assembly, LU with
partial pivoting, solves, DtN map): one kernel launch.  Two precision paths
run on the same inputs: FP32 LU/solves with FP64 iterative refinement (the
reported `value`) and plain FP64 (reported beside it).  The metric is leaf
condensations per second; TFLOP/s use the algorithmic count per leaf
(2/3 n_i^3 + 2 n_i^2 n_b + 2 n_b^2 (p-2)).

Under torchrun the workload's grid is stacked once per rank in y and split
into the boxes of its merge tree, one box (the single-GPU workload's 4096
leaves) per rank: condensation runs with no collective (weak scaling), and
the reduced solve gathers the box roots' maps on rank 0, merges and solves
the top levels there and scatters the boxes' boundary values back
(paper_2211_14969_b300.distributed); rank 0 prints one JSON line.
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "leaf condensations/s and TFLOP/s, mixed vs FP64 GPU path at rel err ≤1e-10"
UNIT = "leaf condensations/s"

# Refinement setting of every mixed-path measurement (also asserted against
# the oracle by tests/test_gpu_bench_setting.py): stop at an estimated error
# of REFINE_TOL per column, at most REFINE_KMAX corrections, FP64 fallback on.
REFINE_TOL = 1e-12
REFINE_KMAX = 6


# DRAM bytes per full 4096-leaf launch from the ncu capture summarised in
# profiles/condense_kernel_bumps_p20.md (592-leaf case scaled by 4096/592),
# keyed by the hash of the condensation kernel's sources it was taken on;
# reported only while those sources still hash to that value.
TRAFFIC_BY_SOURCE = {"32bed28bed2e680f": {"fp32": 30.89e9, "fp64": 73.00e9}}
CONDENSE_SOURCES = ("condense.cu", "dense_lu.cuh", "tc_gemm.cuh", "hps_internal.cuh")


def source_hash():
    """sha256 (first 16 hex digits) of the condensation kernel's sources, in
    a fixed order."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2211_14969_b300", "csrc")
    files = [os.path.join(csrc, f) for f in CONDENSE_SOURCES]
    h = hashlib.sha256()
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def leaf_flops(p, m=0):
    """Algorithmic flops of one leaf: LU of A_ii, the solves for the n_b
    boundary columns and m loads, and the DtN rows (m = 0 gives the
    per-leaf figure of the S/T operators alone)."""
    q = p - 2
    n, nb = q * q, 4 * q
    return (2.0 / 3.0) * n ** 3 + 2.0 * n * n * (nb + m) + 2.0 * nb * (nb + m) * q


WORKLOADS = {
    "bumps_p20": ("64x64 leaves (4096) of the unit square, p=20 (A_ii 324x324), kappa=200, "
                  "b=1-0.5exp(-|x-c|^2/0.02), m=1 body load of 16 Gaussian bumps (seed 2)"),
    "bumps_p30": "32x32 leaves (1024), p=30 (A_ii 784x784), kappa=200, b and loads as bumps_p20 (seed 3)",
    "annulus_p24": ("annular sector r in [1,2], theta in [0,pi/2] mapped to the unit square, 64x128 leaves "
                    "(8192), p=24, kappa=400, b=1-0.3sin(4r)cos(6theta), m=1 (seed 4)"),
    "uneven": ("128x80 leaves (10240) of the unit square, p drawn from {12,16,20,24,32} with weights "
               "{.3,.25,.2,.15,.1} (seed 5), kappa=300, b as bumps_p20, m=64 body loads"),
    "psi_p20": ("the curved domain {(x1, x2/psi(x1))}, psi(z)=1-sin(z)/4, on 64x64 reference leaves (4096), "
                "p=20, mixed term c12 != 0, b=1, kappa=200, m=1 body load of bumps (seed 6)"),
}


PEAK_SOURCE = {
    "fp32": "148 SMs x 128 FP32 lanes x 2 x max SM clock (unit counts)",
    "fp64": "nominal 1.25 TFLOP/s of the part",
    "bf16": "measured bf16 dense GEMM peak (burst)",
    "tf32": "measured bf16 peak x nominal tf32/bf16 ratio 1.1/2.25",
}


def make_workload(name):
    from paper_2211_14969_b300 import workloads as WL
    return {"bumps_p20": WL.bumps_p20, "bumps_p30": WL.bumps_p30, "annulus_p24": WL.annulus_p24,
            "uneven": WL.uneven, "psi_p20": WL.psi_p20}[name]()


def peaks():
    """Roofline denominators: FP32 and FP64 ALU peaks from unit counts and the
    maximum SM clock (148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz); FP64 is
    the nominal 1.25 TFLOP/s of the part.  HBM and BF16 from the measured
    peaks file (a STREAM-style copy and a BF16 GEMM on this part) when
    present."""
    sm_mhz = 2032.0
    hbm = None
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            mp = json.load(fh)
        sm_mhz = mp.get("sm_max_mhz", sm_mhz)
        hbm = mp.get("hbm_gbs")
    fp32 = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
    bf16 = 1738.9
    if os.path.exists(path):
        bf16 = mp.get("bf16_tflops", bf16)
    # TF32 dense: the measured BF16 peak x the nominal TF32 / BF16 ratio (1.1 / 2.25)
    return {"fp32_tflops": fp32, "fp64_tflops": 1.25, "hbm_gbs": hbm, "bf16_tflops": bf16,
            "tf32_tflops": bf16 * 1.1 / 2.25}


# ---------------------------------------------------------------- distributed

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend=backend)
    return rank, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        mhz, mx, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and parts[1] != self.uuid:
                continue
            try:
                mhz.append(float(parts[2]))
                mx = float(parts[3])
                power.append(float(parts[4]))
            except ValueError:
                continue
            for n, v in zip(names, parts[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------- workload

def make_inputs(w, plan):
    """Coefficients and body loads at the library's node coordinates, packed
    leaf after leaf, as device tensors: the workload's fields are evaluated
    with torch on the device, one vectorised evaluation per leaf order (the
    64 bump loads of the uneven workload are billions of exponentials)."""
    import torch
    lay = plan.layout
    xy = plan.leaf_nodes()
    dev = xy.device
    coef = torch.empty(int(6 * lay.o_p2[-1]), dtype=torch.float64, device=dev)
    f = torch.empty(int(lay.o_p2[-1] * w.m), dtype=torch.float64, device=dev)
    p_all = np.asarray(lay.p)
    for p in np.unique(p_all):
        idx = np.flatnonzero(p_all == p)
        p2 = int(p * p)
        o = torch.from_numpy(lay.o_p2[idx].astype(np.int64)).to(dev)
        gx = (2 * o)[:, None] + torch.arange(p2, device=dev)[None, :]
        x, y = xy[gx], xy[gx + p2]
        c = torch.movedim(w.coefficients(x, y, xp=torch), 0, 1)             # (k, 6, p2)
        coef[(6 * o)[:, None] + torch.arange(6 * p2, device=dev)[None, :]] = c.reshape(len(idx), -1)
        if w.m > 0:
            fl = w.body_load(x, y, xp=torch).reshape(len(idx), -1)          # (k, p2 * m)
            f[(o * w.m)[:, None] + torch.arange(p2 * w.m, device=dev)[None, :]] = fl
    torch.cuda.synchronize()
    return coef, f


def rel_leafwise(a, b, sizes):
    """max over leaves of ||a_l - b_l|| / ||b_l|| for packed per-leaf blocks
    of the given sizes."""
    import torch
    lengths = torch.as_tensor(np.asarray(sizes, dtype=np.int64), device=a.device)
    num = torch.segment_reduce((a - b) ** 2, "sum", lengths=lengths).sqrt()
    den = torch.segment_reduce(b * b, "sum", lengths=lengths).sqrt().clamp_min(1e-300)
    return float((num / den).max())


def time_steps(fn, steps, warmup, ws, stream, on_start=None):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if on_start is not None:
        on_start()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    return max_over_ranks(ms, ws)


_WL_CACHE = {}


def _oracle_chunk(args):
    """Pool worker: condense the given leaves of a named workload with the
    oracle as it stands; returns (leaves done, outputs of the leaves in
    keep)."""
    name, leaves, keep = args
    import oracle.hps_oracle as O
    w = _WL_CACHE.get(name)
    if w is None:
        w = _WL_CACHE[name] = make_workload(name)
    boxes = w.boxes()
    out = {}
    for l in leaves:
        p = int(w.p[l])
        x, y = O.leaf_nodes(p, boxes[l])
        f = w.body_load(x, y).reshape(p * p, -1) if w.m > 0 else None
        r = O.condense_leaf(p, boxes[l], w.coefficients(x, y), w.kappa, f)
        if l in keep:
            out[int(l)] = {k: r[k] for k in ("S", "T", "W", "h") if k in r}
    return len(leaves), out


def _one_blas_thread():
    """Pool initializer: one BLAS thread per worker process."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass


def host_info():
    """CPU model, usable cores and the BLAS library numpy calls."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    blas = None
    try:
        from threadpoolctl import threadpool_info
        libs = [i for i in threadpool_info() if i.get("user_api") == "blas"]
        if libs:
            blas = f"{libs[0].get('internal_api')} {libs[0].get('version')}"
    except Exception:
        pass
    if blas is None:   # numpy's build record
        try:
            b = np.__config__.CONFIG["Build Dependencies"]["blas"]
            blas = f"{b.get('name')} {b.get('version')}"
        except Exception:
            pass
    return {"cpu": model, "nproc": cores, "blas": blas}


class OraclePool:
    """The oracle on every host core: spawned worker processes (not forked:
    the parent holds a CUDA context), one BLAS thread each."""

    def __init__(self, workers=None):
        import concurrent.futures
        import multiprocessing as mp
        self.info = host_info()
        self.workers = workers or self.info["nproc"]
        # spawned workers read these when they import numpy (this process's
        # BLAS, already loaded, keeps its threads); left set so workers the
        # executor starts later inherit them too
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.ex = concurrent.futures.ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"),
                                                         initializer=_one_blas_thread)
        self.warmed = set()

    def warm(self, name):
        """One leaf per worker, untimed: imports, the workload's draws."""
        if name not in self.warmed:
            list(self.ex.map(_oracle_chunk, [(name, [0], ())] * self.workers))
            self.warmed.add(name)

    def run(self, name, leaves, keep=(), budget_s=None, chunk=4):
        """Condense `leaves` across the pool; once budget_s has passed, the
        chunks not yet started are cancelled.  Returns (leaves done,
        seconds, kept outputs)."""
        import concurrent.futures
        self.warm(name)
        keep = set(int(l) for l in keep)
        parts = [leaves[i:i + chunk] for i in range(0, len(leaves), chunk)]
        t0 = time.perf_counter()
        futs = [self.ex.submit(_oracle_chunk, (name, part, keep & set(part))) for part in parts]
        if budget_s is not None:
            for _ in concurrent.futures.as_completed(futs):
                if time.perf_counter() - t0 > budget_s:
                    for g in futs:
                        g.cancel()
                    break
        live = [g for g in futs if not g.cancelled()]
        concurrent.futures.wait(live)
        dt = time.perf_counter() - t0
        done, results = 0, {}
        for g in live:
            n, out = g.result()
            done += n
            results.update(out)
        return done, dt, results

    def close(self):
        self.ex.shutdown(wait=True, cancel_futures=True)


def cpu_baseline(w, name, pool, budget_s, keep=(), repeats=3):
    """The FP64 oracle as it stands over every leaf of the workload on all
    host cores (one process and one BLAS thread per core), best of up to
    `repeats` passes while the passes fit the time budget; if one pass does
    not fit, the leaves done within the budget (a bounded sample, stated)."""
    n = w.n_leaves
    leaves = list(range(n))
    best, spent, results, passes, sample_done = None, 0.0, {}, 0, n
    for rep in range(repeats):
        done, dt, res = pool.run(name, leaves, keep if rep == 0 else (), budget_s=budget_s - spent)
        results.update(res)
        spent += dt
        passes += 1
        rate = done / dt
        if best is None or rate > best:
            best = rate
        if done < n:
            sample_done = done
            break
        if spent + dt > budget_s:
            break
    hi = pool.info
    what = (f"every leaf ({n}), best of {passes} pass(es)" if sample_done == n else
            f"{sample_done} of the {n} leaves within a {budget_s:.0f} s budget (one pass does not fit)")
    rec = {"value": best, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "cpu": hi["cpu"],
           "nproc": hi["nproc"], "blas": hi["blas"],
           "sample": f"{what}; numpy/LAPACK FP64, {pool.workers} processes x 1 BLAS thread"}
    return rec, results


def merge_cpu_baseline(w, n_sub=8):
    """The oracle's merge tree as it stands on the n_sub x n_sub leaves at
    the corner of the grid (leaf maps condensed by the oracle beforehand,
    not timed): algorithmic merge GFLOP/s of that sub-grid."""
    import oracle.hps_oracle as O
    p = int(w.p[0])
    boxes = w.boxes()
    leaves = []
    for ix in range(n_sub):
        for iy in range(n_sub):
            b = boxes[ix * w.ny + iy]
            x, y = O.leaf_nodes(p, b)
            f = w.body_load(x, y).reshape(p * p, -1) if w.m > 0 else None
            leaves.append(O.condense_leaf(p, b, w.coefficients(x, y), w.kappa, f))
    t0 = time.perf_counter()
    O.hps_upward(p, n_sub, n_sub, leaves)
    dt = time.perf_counter() - t0
    gf, _ = merge_flops(p - 2, n_sub, n_sub, max(w.m, 1))
    return {"value": gf / dt / 1e9, "unit": "GFLOP/s (algorithmic, merge)", "kind": "oracle",
            "sample": f"hps_upward of the oracle on the {n_sub}x{n_sub} corner leaves ({gf / 1e9:.2f} Gflop in "
                      f"{dt:.2f} s), numpy/LAPACK FP64"}


def parity_vs_oracle(w, lay, outs, results):
    """Max per-leaf relative error of GPU outputs against the oracle leaves."""
    worst = {}
    m = w.m
    for name, out in outs.items():
        e = 0.0
        for l, ref in results.items():
            ni, nb = int(lay.ni[l]), int(lay.nb[l])
            pairs = [(out["S"][int(lay.o_sb[l]):int(lay.o_sb[l + 1])].reshape(ni, nb), ref["S"]),
                     (out["T"][int(lay.o_bb[l]):int(lay.o_bb[l + 1])].reshape(nb, nb), ref["T"])]
            if m > 0:
                pairs.append((out["h"][int(lay.o_nb[l]) * m:int(lay.o_nb[l + 1]) * m].reshape(nb, m), ref["h"]))
                pairs.append((out["W"][int(lay.o_ni[l]) * m:int(lay.o_ni[l + 1]) * m].reshape(ni, m), ref["W"]))
            for a, b in pairs:
                e = max(e, float(np.linalg.norm(a - b) / np.linalg.norm(b)))
        worst[name] = e
    return worst


# ---------------------------------------------------------------- arms

def config_block(name, w, ws, graph=False):
    out_gb = (sum(int(p - 2) ** 2 * 4 * int(p - 2) + 16 * int(p - 2) ** 2 + int(p - 2) ** 2 * w.m
                  + 4 * int(p - 2) * w.m for p in w.p) * 8) / 1e9
    return {"workload": f"{name}: {WORKLOADS[name]}",
            "n_leaves_per_rank": w.n_leaves, "p": sorted(set(int(v) for v in w.p)), "m": w.m,
            "parallelism": ("leaf-parallel on 1 GPU" if ws == 1 else
                            f"{ws} ranks, one merge-tree box of leaves each (the grid stacked {ws}x in y, "
                            "weak scaling); condensation needs no collective, the reduced solve gathers the "
                            "box roots on rank 0 and scatters their boundary values (NCCL)"),
            "launch": "CUDA graph replay of the persistent kernel" if graph else "one persistent kernel launch",
            "l2": f"no flush: per step the outputs alone are {out_gb:.2f} GB > 126 MB L2"}


def run_reference(args, rank, ws):
    """The reference arm: the FP64 CPU oracle as it stands on every host
    core (one process and one BLAS thread each), on the same workload; each
    step condenses a bounded sample of 4 leaves per core (the next leaves of
    a seeded permutation)."""
    if rank != 0:
        return
    w = make_workload(args.workload)
    pool = OraclePool()
    per_step = 4 * pool.workers
    perm = np.random.default_rng(1234).permutation(w.n_leaves).tolist()
    pos = 0

    def step():
        nonlocal pos
        leaves = [perm[(pos + i) % w.n_leaves] for i in range(per_step)]
        pos += per_step
        return pool.run(args.workload, leaves)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        done += step()[0]
    dt = time.perf_counter() - t0
    pool.close()
    value = done / dt
    flops = float(np.mean([leaf_flops(int(p), w.m) for p in w.p]))
    hi = pool.info
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(args.workload, w, 1),
            "tflops": value * flops / 1e12,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                             "cpu": hi["cpu"], "nproc": hi["nproc"], "blas": hi["blas"],
                             "sample": f"{per_step} leaves per step ({args.steps} steps) of the {w.n_leaves}, "
                                       f"FP64 numpy/LAPACK, {pool.workers} processes x 1 BLAS thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def alloc_outputs(lay, m, paths):
    import torch
    n = lay.n_leaves
    return {name: {"S": torch.empty(int(lay.o_sb[-1]), dtype=torch.float64, device="cuda"),
                   "T": torch.empty(int(lay.o_bb[-1]), dtype=torch.float64, device="cuda"),
                   "h": torch.empty(int(lay.o_nb[-1]) * m, dtype=torch.float64, device="cuda"),
                   "W": torch.empty(int(lay.o_ni[-1]) * m, dtype=torch.float64, device="cuda"),
                   "info": torch.empty(n, dtype=torch.int32, device="cuda")} for name in paths}


def gpu_uuid():
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    except Exception:
        return None


def measure_paths(w, plan, coef, f, outs, paths, steps, warmup, ws, graph=False, traffic=None):
    """Time every precision path on the same resident inputs: `steps`
    hps_condense calls (or CUDA-graph replays) after `warmup`, CUDA events on
    the launch stream, clocks sampled meanwhile.  Returns per-path records."""
    import torch
    stream = torch.cuda.current_stream()
    m = w.m
    graphs = {}
    if graph:
        from paper_2211_14969_b300 import tune
        for name in paths:
            graphs[name] = tune.CondenseGraph(plan, coef, f, m, prec=name, tol=REFINE_TOL, kmax=REFINE_KMAX,
                                              out=outs[name])

    def step(name):
        if name in graphs:
            graphs[name].replay()
        else:
            plan.condense(coef, f, m=m, prec=name, tol=REFINE_TOL, kmax=REFINE_KMAX, out=outs[name])

    flops = float(sum(leaf_flops(int(p), m) for p in w.p))
    pk = peaks()
    res = {}
    n = w.n_leaves
    for name in paths:
        with ClockSampler(gpu_uuid()) as cs:
            ms = time_steps(lambda: step(name), steps, warmup, ws, stream,
                            on_start=None if graphs else (lambda: plan.set_timing(True)))
        per_step = ms / steps
        if graphs:
            kernel_ms = per_step          # a replay is the counter reset plus the one kernel
        else:
            kt = plan.phase_times()        # kernel-only events of the timed calls
            plan.set_timing(False)
            kernel_ms = kt[0] / kt[1]
        info = outs[name]["info"].cpu().numpy()
        fallback_leaves = plan.fallback_count() if name != "fp64" else 0
        peak = pk[name + "_tflops"]
        achieved = flops / (kernel_ms * 1e-3) / 1e12
        res[name] = {"ms_per_step": per_step, "value": ws * n / (per_step * 1e-3),
                     "tflops": ws * flops / (per_step * 1e-3) / 1e12, "kernel_ms": kernel_ms,
                     "info_nonzero": int((info != 0).sum()),
                     "fp64_fallback_leaves": int(fallback_leaves),
                     "roofline": {"bound": "tensor" if name in ("tf32", "bf16") else "alu", "achieved": achieved,
                                  "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                                  "traffic": (traffic or {}).get(name), "peak_source": PEAK_SOURCE[name]},
                     "clocks": cs.summary(), "gpu_launches": steps}
    return res, flops


def sample_leaves(w, k, seed=0):
    """k seeded random leaves plus the first and last of the work queue."""
    queue = np.argsort(-np.asarray(w.p), kind="stable")
    rng = np.random.default_rng(seed)
    return sorted(set(rng.choice(w.n_leaves, size=min(k, w.n_leaves), replace=False).tolist())
                  | {int(queue[0]), int(queue[-1])})


def per_order_launches(w, plan, coef, f, res, steps):
    """The uneven workload: one plan and launch per order, back to back on
    the same stream, against the fused single launch."""
    import torch
    from paper_2211_14969_b300 import hps
    lay = plan.layout
    m = w.m
    stream = torch.cuda.current_stream()
    per_order, subs = {}, []
    for p in sorted(set(int(v) for v in w.p)):
        idx = np.flatnonzero(np.asarray(w.p) == p)
        sp = hps.Plan(w.p[idx], w.boxes()[idx], w.kappa)
        sl = sp.layout
        gx = np.concatenate([np.arange(6 * int(lay.o_p2[l]), 6 * int(lay.o_p2[l + 1])) for l in idx])
        gf = np.concatenate([np.arange(int(lay.o_p2[l]) * m, int(lay.o_p2[l + 1]) * m) for l in idx])
        c_sub, f_sub = coef[torch.from_numpy(gx).cuda()], f[torch.from_numpy(gf).cuda()]
        subs.append((sp, c_sub, f_sub, alloc_outputs(sl, m, ("x",))["x"]))
    for name in ("fp64", "fp32"):
        def per_order_step():
            for sp, c_sub, f_sub, o in subs:
                sp.condense(c_sub, f_sub, m=m, prec=name, tol=REFINE_TOL, kmax=REFINE_KMAX, out=o)
        ms_po = time_steps(per_order_step, steps, 3, 1, stream) / steps
        per_order[name] = {"ms_per_step": ms_po, "value": w.n_leaves / (ms_po * 1e-3), "launches": len(subs),
                           "fused_ms_per_step": res[name]["ms_per_step"],
                           "fused_speedup": ms_po / res[name]["ms_per_step"]}
    for sp, *_ in subs:
        sp.close()
    return per_order


def workload_block(name, ws, pool, steps=3, warmup=3, cpu_seconds=10.0):
    """One more BASELINE workload measured in the default run: its paths on
    the same inputs, each mixed path's error against the FP64 path over all
    leaves, both against the oracle on sampled leaves, the oracle on all
    host cores within a time budget, and (uneven) CUDA-graph replay of the
    fused launch against one launch per order."""
    import torch
    from paper_2211_14969_b300 import hps
    w = make_workload(name)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    lay = plan.layout
    m = w.m
    coef, f = make_inputs(w, plan)
    paths = ("fp32", "fp64", "tf32", "bf16") if name == "bumps_p30" else ("fp32", "fp64")
    outs = alloc_outputs(lay, m, paths)
    graph = name == "uneven"
    res, flops = measure_paths(w, plan, coef, f, outs, paths, steps, warmup, ws, graph=graph)
    sizes = {"S": lay.sb, "T": lay.bb, "h": lay.nb * m, "W": lay.ni * m}
    o64 = outs["fp64"]
    block = {"config": config_block(name, w, ws, graph), "algorithmic_flops_per_step": flops,
             "refinement": {"tol": REFINE_TOL, "kmax": REFINE_KMAX, "fp64_fallback": True}}
    for pth in paths:
        r = res[pth]
        rec = {k: r[k] for k in ("value", "ms_per_step", "tflops", "kernel_ms", "roofline", "clocks",
                                 "gpu_launches", "info_nonzero", "fp64_fallback_leaves")}
        rec["unit"] = UNIT
        if pth != "fp64":
            rec["max_leaf_relerr_vs_fp64"] = {k: rel_leafwise(outs[pth][k], o64[k], sizes[k]) for k in sizes}
        block[f"{pth}_path"] = rec
    keep = sample_leaves(w, 6, seed=11)
    if pool is not None:
        cpu, results = cpu_baseline(w, name, pool, cpu_seconds, keep=keep, repeats=1)
        missing = [l for l in keep if l not in results]
        if missing:
            results.update(pool.run(name, missing, keep=missing)[2])
        outs_np = {k: {kk: vv.cpu().numpy() for kk, vv in v.items()} for k, v in outs.items()}
        block["parity_vs_oracle_sampled"] = parity_vs_oracle(w, lay, outs_np, results)
        block["parity_leaves"] = keep
        block["cpu_baseline"] = cpu
    if name == "uneven":
        block["per_order_launches"] = per_order_launches(w, plan, coef, f, res, steps)
    plan.close()
    del outs, coef, f
    torch.cuda.empty_cache()
    return block


def rank_view(w, ws, rank):
    """Weak scaling over ws ranks: the workload's nx x ny leaf grid stacked
    ws times in y (nx x ny*ws leaves of the same size on [0,1] x [0,ws],
    the fields evaluated there), partitioned into the boxes of its merge
    tree; rank r owns box r, the nx x ny leaves with y in [r, r+1] (rank
    0's box is the single-GPU workload itself).  Returns the rank's leaves
    as a workload (local order) and the partition."""
    from paper_2211_14969_b300 import distributed as D
    from paper_2211_14969_b300 import workloads as WL
    part = D.Partition(w.nx, w.ny * ws, ws)
    if (part.wx0, part.wy0) != (w.nx, w.ny):
        raise SystemExit("multi-rank runs need a workload grid with nx <= ny")
    lv = part.leaves(rank)
    hx, hy = 1.0 / w.nx, 1.0 / w.ny
    ix, iy = lv // (w.ny * ws), lv % (w.ny * ws)
    boxes = np.stack([ix * hx, iy * hy, np.full(len(lv), hx), np.full(len(lv), hy)], axis=1)
    v = WL.scaled(w, w.nx, w.ny)
    v.p = np.full(len(lv), int(w.p[0]), dtype=np.int32)
    v.boxes = lambda b=boxes: b
    return v, part


def split_reduced_solve(w, part, plan, out, rank, ws, steps, warmup):
    """The merge tree split over the ranks (paper_2211_14969_b300.distributed):
    each rank merges its box to the box root and forms the root's [T | h];
    rank 0 gathers them over NCCL, merges the grid of boxes and solves it
    for the boxes' boundary values from outer Dirichlet data; those are
    scattered back and every rank solves its box.  FP64 leaf maps."""
    import torch
    from paper_2211_14969_b300 import distributed as D
    m = w.m
    q = int(w.p[0]) - 2
    be = D.LibraryBackend(int(w.p[0]), w.kappa, part, rank, w.boxes(), plan=plan, out=out)
    exch = D.TorchExchange(rank, ws, device="cuda")
    g = torch.from_numpy(np.random.default_rng(7).standard_normal((part.root_nodes(q), m))).cuda()
    sol = {}

    def step():
        D.split_merge(be, exch, part, rank, q, m)
        sol["u"] = D.split_solve(be, exch, part, rank, q, g if rank == 0 else None, m)

    stream = torch.cuda.current_stream()
    ms = time_steps(step, steps, warmup, ws, stream)
    nb = part.box_nodes(q)
    return {"ms": ms / steps, "world": ws, "box_leaves": [part.wx0, part.wy0], "box_grid": [part.bx, part.by],
            "exchange": f"gather of {ws} root [T | h] blocks ({nb} x {nb + m} FP64 each) on rank 0, scatter of "
                        f"{ws} boundary blocks ({nb} x {m})",
            "exchange_bytes": int(ws * nb * (nb + 2 * m) * 8)}


def run_gpu(args, rank, ws):
    import torch
    from paper_2211_14969_b300 import hps
    from paper_2211_14969_b300 import workloads as WL

    w = make_workload(args.workload)
    part = None
    if ws > 1:
        w, part = rank_view(w, ws, rank)
    if args.leaves:
        full_boxes = w.boxes()[: args.leaves]
        w = WL.scaled(w, w.nx, w.ny)
        w.nx, w.ny = 1, args.leaves        # the first N leaves of the tiling
        w.boxes = lambda: full_boxes
        w.p = w.p[: args.leaves]
    n = w.n_leaves
    m = w.m
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    lay = plan.layout
    coef, f = make_inputs(w, plan)
    stream = torch.cuda.current_stream()
    all_paths = ("fp64", "fp32", "tf32", "bf16")
    paths = all_paths if args.prec == "both" else (args.prec,)
    outs = alloc_outputs(lay, m, paths)
    full_p20 = args.workload == "bumps_p20" and not args.leaves
    traffic = TRAFFIC_BY_SOURCE.get(source_hash(), {}) if full_p20 else {}
    # the oracle pool starts before the timed GPU work and is reused by every block
    pool = OraclePool() if (rank == 0 and ws == 1 and not args.no_cpu_baseline and args.prec == "both"
                            and not args.leaves) else None
    res, flops = measure_paths(w, plan, coef, f, outs, paths, args.steps, args.warmup, ws, graph=args.graph,
                               traffic=traffic)
    if args.prec != "both" or args.leaves:
        if rank == 0:
            print(json.dumps({"profiling_case": True, "leaves": n, **{k: {kk: vv for kk, vv in v.items()
                                                                          if kk != "clocks"} for k, v in res.items()}}))
        plan.close()
        return None
    o64, o32 = outs["fp64"], outs["fp32"]
    sizes = {"S": lay.sb, "T": lay.bb, "h": lay.nb * m, "W": lay.ni * m}
    err = {k: rel_leafwise(o32[k], o64[k], sizes[k]) for k in ("S", "T", "h", "W")}
    tc_paths = {}
    for name in ("tf32", "bf16"):
        r = res[name]
        tc_paths[name + "_path"] = {
            "value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"], "tflops": r["tflops"],
            "dtype": f"{name} x3 split (hi*hi + hi*lo + lo*hi) on tcgen05, f32 accumulate, + f64 refinement",
            "roofline": r["roofline"], "clocks": r["clocks"], "gpu_launches": args.steps,
            "fp64_fallback_leaves": r["fp64_fallback_leaves"], "info_nonzero": r["info_nonzero"],
            "max_leaf_relerr_vs_fp64": {k: rel_leafwise(outs[name][k], o64[k], sizes[k]) for k in ("S", "T", "h", "W")}}

    # end to end through the C ABI with host buffers (hps_condense_host):
    # H2D of the inputs, condensation, D2H of every output, each step, in
    # chunks whose copies overlap the launches; and the same with one chunk
    # (copies, then the launch, then the copies back)
    e2e = None
    if (rank == 0 or ws > 1) and "fp32" in outs:
        coef_p = coef.cpu().pin_memory()
        f_p = f.cpu().pin_memory()
        host_out = {k: torch.empty(v.numel(), dtype=v.dtype).pin_memory() for k, v in o32.items()}
        steps_e2e = max(2, args.steps // 2)
        h2d = coef_p.numel() * 8 + f_p.numel() * 8
        d2h = sum(v.numel() * v.element_size() for v in host_out.values())
        rates = {}
        for chunks in (8, 1):
            ms_e2e = time_steps(lambda: plan.condense_host(coef_p, f_p, m=m, prec="fp32", tol=REFINE_TOL,
                                                           kmax=REFINE_KMAX, out=host_out, chunks=chunks),
                                steps_e2e, 1, ws, stream)
            rates[chunks] = ws * n / (ms_e2e / steps_e2e * 1e-3)
        same = all(torch.equal(host_out[k], o32[k].cpu()) for k in host_out)
        e2e = {"value": rates[8], "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "api": "hps_condense_host, pinned host buffers, 8 chunks (copies overlap the launches)",
               "value_one_chunk": rates[1], "equals_device_call": bool(same)}

    # the impedance-to-impedance leaf maps on the same leaves (FP64; the
    # complex leaf system in real form, 2(n_i + n_b) unknowns)
    iti = None
    if rank == 0 and ws == 1 and not args.no_extra:
        iti = iti_timing(w, plan, coef, f, max(3, args.steps // 3), 3, ws)

    per_order = None
    if args.workload == "uneven" and rank == 0:
        per_order = per_order_launches(w, plan, coef, f, res, max(2, args.steps // 2))

    # the reduced solve on the same grid, from the FP64 leaf maps: every
    # merge level (hps_merge) and the downward pass with leaf recovery
    # (hps_solve) for random Dirichlet data
    reduced = None
    if part is not None and "fp64" in outs:
        reduced = {"split_over_ranks": split_reduced_solve(w, part, plan, outs["fp64"], rank, ws,
                                                           max(3, args.steps // 3), 3)}
    elif (len(set(int(v) for v in w.p)) == 1 and "fp64" in outs
            and w.nx * w.ny == n and (w.nx & (w.nx - 1)) == 0 and (w.ny & (w.ny - 1)) == 0):
        o = outs["fp64"]
        q = int(w.p[0]) - 2
        g = torch.from_numpy(np.random.default_rng(7).standard_normal(2 * (w.nx + w.ny) * q * m)).cuda()
        u = torch.empty(int(lay.o_p2[-1]) * m, dtype=torch.float64, device="cuda")
        rs = max(3, args.steps // 3)
        with ClockSampler(gpu_uuid()) as cs:
            t_merge = time_steps(lambda: plan.merge(w.nx, w.ny, o["T"], o["h"], m), rs, 3, ws, stream)
        merge_launches = plan.last_launch_count()
        t_solve = time_steps(lambda: plan.solve(g, o["S"], o["W"], m, out=u), rs, 3, ws, stream)
        mflops, _ = merge_flops(q, w.nx, w.ny, m)
        tf = mflops / (t_merge / rs * 1e-3) / 1e12
        reduced = {"merge_ms": t_merge / rs, "solve_ms": t_solve / rs, "merge_gflop": mflops / 1e9,
                   "merge_tflops": tf,
                   "roofline": {"bound": "alu", "achieved": tf, "peak": 1.25, "unit": "TFLOP/s", "frac": tf / 1.25,
                                "traffic": None, "peak_source": "nominal 1.25 TFLOP/s FP64 of the part; FP64 flops per second, the large products of which run FP64-accurate on the BF16 tensor cores (exact integer slices), so frac can exceed 1"},
                   "gpu_launches_merge": merge_launches, "flux_mismatch": flux_mismatch(w, lay, o, u, m),
                   "clocks": cs.summary()}
        # SlabLU (Section 2, Eq. (dell1)) on the same leaf maps and data
        if w.nx >= 16:
            sl, u_slab = slab_timing(w, plan, o, g, 16, rs, 3, ws)
            sl["u_relerr_vs_merge_tree"] = float((u_slab - u).norm() / u.norm())
            reduced["slablu"] = sl

    line = None
    if rank == 0:
        cpu = None
        parity = None
        if pool is not None:
            keep = sample_leaves(w, 72, seed=5)
            cpu, results = cpu_baseline(w, args.workload, pool, args.cpu_seconds, keep=keep)
            missing = [l for l in keep if l not in results]
            if missing:
                results.update(pool.run(args.workload, missing, keep=missing)[2])
            outs_np = {k: {kk: vv.cpu().numpy() for kk, vv in v.items()} for k, v in outs.items()}
            parity = parity_vs_oracle(w, lay, outs_np, results)
        r32, r64 = res["fp32"], res["fp64"]
        line = {"metric": METRIC, "value": r32["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r32["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic (seeded Gaussian bumps, analytic coefficient fields), resident in HBM",
                "algorithmic_flops_per_step": flops,
                "config": config_block(args.workload, w, ws, bool(args.graph)),
                "tflops": r32["tflops"],
                "precision_path": (f"fp32 LU/solves + fp64 residual refinement (stop when the estimated error "
                                   f"eta_k^2/eta_(k-1) <= {REFINE_TOL:g} in every column, kmax {REFINE_KMAX})"),
                "roofline": r32["roofline"],
                "clocks": r32["clocks"],
                "e2e": e2e,
                "gpu_launches": args.steps,
                "fp64_path": {"value": r64["value"], "unit": UNIT, "ms_per_step": r64["ms_per_step"],
                              "tflops": r64["tflops"], "dtype": "f64", "roofline": r64["roofline"],
                              "clocks": r64["clocks"], "gpu_launches": args.steps},
                "mixed_vs_fp64_max_leaf_relerr": err,
                **tc_paths,
                "info_nonzero": {"fp32": r32["info_nonzero"], "fp64": r64["info_nonzero"]},
                "mixed_leaves_recondensed_in_fp64": r32["fp64_fallback_leaves"],
                "cpu_baseline": cpu,
                "parity_vs_oracle_sampled": parity,
                "parity_leaves": len(keep) if pool is not None else 0}
        if reduced is not None:
            if pool is not None:
                reduced["cpu_baseline"] = merge_cpu_baseline(w)
                reduced["cpu_baseline"]["cores"] = 1
            line["reduced_solve_fp64"] = reduced
        if per_order is not None:
            line["per_order_launches"] = per_order
        if iti is not None:
            line["iti_fp64_path"] = iti
    plan.close()
    del outs
    torch.cuda.empty_cache()
    # the other BASELINE workloads, each with its own paths, errors, roofline
    # and clocks (one GPU: the default run and rank 0 of a single-rank job)
    if rank == 0 and ws == 1 and not args.no_extra and args.workload == "bumps_p20":
        line["workloads"] = {nm: workload_block(nm, ws, pool) for nm in ("bumps_p30", "annulus_p24", "uneven")}
    if pool is not None:
        pool.close()
    if line is not None:
        print(json.dumps(line), flush=True)
    return line


def run_leaf_solve(args, rank, ws):
    """The two leaf solves after the reduced solve, on the same edge values:
    u_i = S u_b + W from stored solution operators, against re-forming and
    re-factoring every leaf (the paper's choice, which keeps no S); plus the
    condensation with and without storing S, the cost the stored solve
    carries.  One JSON line."""
    import torch
    from paper_2211_14969_b300 import hps
    w = make_workload(args.workload)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    lay = plan.layout
    coef, f1 = make_inputs(w, plan)
    stream = torch.cuda.current_stream()
    sizes_u = [int(p) ** 2 for p in lay.p]
    s_bytes = int(lay.o_sb[-1]) * 8
    res = {}
    for m in (1, 64):
        rng = np.random.default_rng(100 + m)
        f = f1 if m == w.m else torch.from_numpy(rng.standard_normal(int(lay.o_p2[-1] * m))).cuda()
        ub = torch.from_numpy(rng.standard_normal(int(lay.o_nb[-1] * m))).cuda()
        cond = plan.condense(coef, f, m=m, prec="fp64")
        u_rec = torch.empty(int(lay.o_p2[-1] * m), dtype=torch.float64, device="cuda")
        t_rec = time_steps(lambda: plan.leaf_recover(cond["S"], cond["W"], ub, m, out=u_rec),
                           args.steps, args.warmup, ws, stream)
        row = {"stored_S": {"value": w.n_leaves * args.steps / (t_rec / 1e3), "ms_per_step": t_rec / args.steps}}
        for prec, name in (("fp64", "refactor_fp64"), ("fp32", "refactor_mixed")):
            o = {"u": torch.empty_like(u_rec), "info": torch.empty(lay.n_leaves, dtype=torch.int32, device="cuda")}
            t = time_steps(lambda: plan.leaf_resolve(coef, ub, f, m=m, prec=prec, tol=REFINE_TOL, kmax=REFINE_KMAX, out=o),
                           args.steps, args.warmup, ws, stream)
            err = rel_leafwise(o["u"], u_rec, [s * m for s in sizes_u])
            row[name] = {"value": w.n_leaves * args.steps / (t / 1e3), "ms_per_step": t / args.steps,
                         "max_leaf_relerr_vs_stored_S": err, "info_nonzero": int((o["info"] != 0).sum()),
                         "fp64_fallback_leaves": plan.fallback_count() if prec == "fp32" else 0}
        for prec in ("fp64", "fp32"):
            for store in (True, False):
                t = time_steps(lambda: plan.condense(coef, f, m=m, prec=prec, tol=REFINE_TOL, kmax=REFINE_KMAX, store_S=store),
                               args.steps, args.warmup, ws, stream)
                row[f"condense_{prec}_{'with' if store else 'without'}_S_ms"] = t / args.steps
        res[f"m={m}"] = row
    if rank == 0:
        print(json.dumps({"metric": "leaf solves/s after the reduced solve: stored S vs re-formed and re-factored leaves",
                          "unit": "leaf solves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": True, "data": "synthetic (random edge values and, for m = 64, loads)",
                          "config": config_block(args.workload, w, ws), "S_bytes_stored": s_bytes,
                          "results": res}), flush=True)


def merge_flops(q, nx, ny, m):
    """Algorithmic flops of hps_merge over an nx x ny grid (q edge nodes per
    leaf side): per merge the LU of Z (2/3 n3^3), the solve for the parent's
    n_p + m right-hand columns (2 n3^2 (n_p + m)) and, below the root, the
    parent's [T | h] update (2 n_p n3 (n_p + m)); merges alternate x then y."""
    wx = wy = 1
    total = 0.0
    levels = []
    while wx < nx or wy < ny:
        along_x = wx < nx and (wx <= wy or wy == ny)
        n3 = (wy if along_x else wx) * q
        npar = 2 * ((2 * wx + wy) if along_x else (wx + 2 * wy)) * q
        if along_x:
            wx *= 2
        else:
            wy *= 2
        nm = (nx // wx) * (ny // wy)
        root = wx == nx and wy == ny
        f = nm * (2.0 / 3.0 * n3 ** 3 + 2.0 * n3 ** 2 * (npar + m) + (0.0 if root else 2.0 * npar * n3 * (npar + m)))
        levels.append({"merges": nm, "n3": n3, "n_parent": npar, "gflop": f / 1e9})
        total += f
    return total, levels


def iti_leaf_flops(p, m):
    """Algorithmic flops of one ItI leaf map as computed: the LU of the real
    form of the complex leaf system (2N unknowns, N = n_i + n_b) and its
    solve for n_b + m right-hand columns."""
    q = p - 2
    n2 = 2 * (q * q + 4 * q)
    return (2.0 / 3.0) * n2 ** 3 + 2.0 * n2 ** 2 * (4 * q + m)


def iti_timing(w, plan, coef, f, steps, warmup, ws):
    """hps_iti_condense over all the workload's leaves, eta = kappa."""
    import torch
    stream = torch.cuda.current_stream()
    with ClockSampler(gpu_uuid()) as cs:
        ms = time_steps(lambda: plan.iti_condense(coef, f, m=w.m, eta=w.kappa, store_Y=True), steps, warmup, ws,
                        stream)
    out = plan.iti_condense(coef, f, m=w.m, eta=w.kappa)
    torch.cuda.synchronize()
    flops = float(sum(iti_leaf_flops(int(p), w.m) for p in w.p))
    tf = flops / (ms / steps * 1e-3) / 1e12
    return {"value": w.n_leaves / (ms / steps * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "tflops": tf,
            "dtype": "f64 (complex leaf system in real form)", "eta": w.kappa,
            "roofline": {"bound": "alu", "achieved": tf, "peak": 1.25, "unit": "TFLOP/s", "frac": tf / 1.25,
                         "traffic": None, "peak_source": "nominal 1.25 TFLOP/s FP64 of the part"},
            "info_nonzero": int((out["info"] != 0).sum()), "gpu_launches": steps, "clocks": cs.summary()}


def slab_flops(q, nx, ny, s, m):
    """Algorithmic flops of hps_slab_factor: the merges inside the slabs (per
    merge as merge_flops, every level forming its parent's [T | h], the
    slabs' own maps included) and the block LU over the S - 1 interfaces of
    n = ny q nodes (per interface the LU of Delta (2/3 n^3), the solve for
    its 2n + m right-hand columns (2 n^2 (2n + m)) and, after the first,
    Delta_k = D_k + L_k S_{k-1} with its body-load column (2 n^2 (n + m)))."""
    wx = wy = 1
    total = 0.0
    while wx < s or wy < ny:
        along_x = wx < s and (wx <= wy or wy == ny)
        n3 = (wy if along_x else wx) * q
        npar = 2 * ((2 * wx + wy) if along_x else (wx + 2 * wy)) * q
        if along_x:
            wx *= 2
        else:
            wy *= 2
        nm = (nx // wx) * (ny // wy)
        total += nm * (2.0 / 3.0 * n3 ** 3 + 2.0 * n3 ** 2 * (npar + m) + 2.0 * npar * n3 * (npar + m))
    n = ny * q
    S = nx // s
    for k in range(S - 1):
        total += 2.0 / 3.0 * n ** 3 + 2.0 * n ** 2 * (2 * n + m) + (2.0 * n ** 2 * (n + m) if k else 0.0)
    return total


def slab_timing(w, plan, out, g, s, steps, warmup, ws):
    """hps_slab_factor and hps_slab_solve (SlabLU, slabs of s leaf columns)
    on the plan's grid from the FP64 leaf maps, timed like the merge tree;
    the solution's flux continuity across every interior edge."""
    import torch
    stream = torch.cuda.current_stream()
    m = w.m
    q = int(w.p[0]) - 2
    with ClockSampler(gpu_uuid()) as cs:
        t_f = time_steps(lambda: plan.slab_factor(w.nx, w.ny, s, out["T"], out["h"], m), steps, warmup, ws, stream)
    launches = plan.last_launch_count()
    u = torch.empty(int(plan.layout.o_p2[-1]) * m, dtype=torch.float64, device="cuda")
    t_s = time_steps(lambda: plan.slab_solve(g, out["S"], out["W"], m, out=u), steps, warmup, ws, stream)
    fl = slab_flops(q, w.nx, w.ny, s, m)
    tf = fl / (t_f / steps * 1e-3) / 1e12
    return {"slab_leaf_columns": s, "interfaces": w.nx // s - 1, "interface_nodes": w.ny * q,
            "factor_ms": t_f / steps, "solve_ms": t_s / steps, "factor_gflop": fl / 1e9, "factor_tflops": tf,
            "roofline": {"bound": "alu", "achieved": tf, "peak": 1.25, "unit": "TFLOP/s", "frac": tf / 1.25,
                         "traffic": None, "peak_source": "nominal 1.25 TFLOP/s FP64 of the part; FP64 flops per second, the large products of which run FP64-accurate on the BF16 tensor cores (exact integer slices), so frac can exceed 1"},
            "gpu_launches_factor": launches, "flux_mismatch": flux_mismatch(w, plan.layout, out, u, m),
            "clocks": cs.summary()}, u


def flux_mismatch(w, lay, out, u, m):
    """Flux continuity of a solved grid: per leaf the outward flux T u_b + h
    at its edge nodes [W, E, S, N]; across every interior edge the two
    leaves' fluxes must cancel.  Returns max |sum| / max |flux|."""
    import torch
    p = int(lay.p[0])
    q, nl = p - 2, lay.n_leaves
    j = torch.arange(1, p - 1, device=u.device)
    edge = torch.cat([j, (p - 1) * p + j, j * p, j * p + p - 1])
    U = u.view(nl, p * p, m)[:, edge, :]
    flux = torch.bmm(out["T"].view(nl, 4 * q, 4 * q), U) + out["h"].view(nl, 4 * q, m)
    F = flux.view(w.nx, w.ny, 4, q, m)
    ew = F[:-1, :, 1] + F[1:, :, 0]          # E of (ix, iy) against W of (ix + 1, iy)
    sn = F[:, :-1, 3] + F[:, 1:, 2]          # N of (ix, iy) against S of (ix, iy + 1)
    worst = max(float(ew.abs().max()) if ew.numel() else 0.0, float(sn.abs().max()) if sn.numel() else 0.0)
    return worst / float(flux.abs().max())


def run_merge_solve(args, rank, ws):
    """The reduced solve after condensation on the same grid: hps_merge
    (all levels of Schur complements) and hps_solve (downward pass and leaf
    recovery), with the large levels near the root solved over many CTAs
    against one CTA per merge on every level.  One JSON line."""
    import torch
    from paper_2211_14969_b300 import hps
    w = make_workload(args.workload)
    if len(set(int(p) for p in w.p)) != 1:
        raise SystemExit("--merge-solve needs a uniform-order workload")
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    lay = plan.layout
    coef, f = make_inputs(w, plan)
    stream = torch.cuda.current_stream()
    m = w.m
    out = plan.condense(coef, f, m=m, prec="fp64")
    q = int(lay.p[0]) - 2
    n_outer = 2 * (w.nx + w.ny) * q
    g = torch.from_numpy(np.random.default_rng(7).standard_normal(n_outer * m)).cuda()
    flops, levels = merge_flops(q, w.nx, w.ny, m)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    except Exception:
        pass
    res = {}
    u_ref = None
    for name, below, tensor, steps, warmup in (("split", -1, True, args.steps, args.warmup),
                                               ("split_parent_maps_fp64_pipe", -1, False, args.steps, args.warmup),
                                               ("one_cta_per_merge", 0, True, max(1, min(args.steps, 2)), 1)):
        plan.set_merge_split(below)
        plan.set_merge_tensor(tensor)
        with ClockSampler(uuid) as ck:
            t_merge = time_steps(lambda: plan.merge(w.nx, w.ny, out["T"], out["h"], m), steps, warmup, ws, stream)
        launches = plan.last_launch_count()
        u = torch.empty(int(lay.o_p2[-1]) * m, dtype=torch.float64, device="cuda")
        t_solve = time_steps(lambda: plan.solve(g, out["S"], out["W"], m, out=u), steps, warmup, ws, stream)
        row = {"merge_ms": t_merge / steps, "solve_ms": t_solve / steps,
               "merge_tflops": flops / (t_merge / steps / 1e3) / 1e12, "merge_launches": launches,
               "flux_mismatch": flux_mismatch(w, lay, out, u, m), "clocks": ck.summary()}
        if u_ref is None:
            u_ref = u.clone()
        else:
            row["u_relerr_vs_split"] = float((u - u_ref).norm() / u_ref.norm())
        res[name] = row
    plan.set_merge_split(-1)
    plan.set_merge_tensor(True)
    slabs = {}
    for sw in (4, 8, 16):
        if sw <= w.nx:
            sl, u_slab = slab_timing(w, plan, out, g, sw, args.steps, args.warmup, ws)
            sl["u_relerr_vs_merge_tree"] = float((u_slab - u_ref).norm() / u_ref.norm())
            slabs[f"s={sw}"] = sl
    res["slablu"] = slabs
    if rank == 0:
        pk = 1.25
        sp = res["split"]
        print(json.dumps({"metric": "reduced solve after condensation: hps_merge + hps_solve time",
                          "unit": "ms", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": False, "dtype": "f64",
                          "data": "synthetic (the workload's FP64 leaf maps; random Dirichlet data)",
                          "config": config_block(args.workload, w, ws),
                          "value": sp["merge_ms"] + sp["solve_ms"],
                          "merge_gflop": flops / 1e9,
                          "roofline": {"bound": "alu", "achieved": sp["merge_tflops"], "peak": pk, "unit": "TFLOP/s",
                                       "frac": sp["merge_tflops"] / pk, "traffic": None,
                                       "peak_source": "nominal 1.25 TFLOP/s FP64 of the part; FP64 flops per second, the large products of which run FP64-accurate on the BF16 tensor cores (exact integer slices), so frac can exceed 1"},
                          "levels": levels, "results": res}), flush=True)


def run_merge_kernels(args):
    """Per-kernel device times of hps_merge (CUDA activity trace, no
    replay), the parents' maps and right-hand-side updates on the tensor
    cores and on the FP64 pipe; with --no-trace only the merges run."""
    import torch
    from paper_2211_14969_b300 import hps
    from paper_2211_14969_b300 import workloads as WL
    n = args.merge_kernels
    w = WL.bumps_p20() if n == 64 else WL.bumps(p=20, nx=n, ny=n, kappa=200.0, seed=1, m=1)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f = make_inputs(w, plan)
    out = plan.condense(coef, f, m=1, prec="fp64")
    plan.set_merge_split(args.merge_split)
    res = {}
    for tensor in (True, False):
        plan.set_merge_tensor(tensor)
        for _ in range(max(1, args.warmup)):
            plan.merge(w.nx, w.ny, out["T"], out["h"], 1)
        torch.cuda.synchronize()
        if args.no_trace:
            continue
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            plan.merge(w.nx, w.ny, out["T"], out["h"], 1)
            torch.cuda.synchronize()
        agg = {}
        for e in prof.events():
            if e.device_type != torch.autograd.DeviceType.CUDA:
                continue
            k = e.name.replace("void ", "").replace("hps::", "").replace("(anonymous namespace)::", "").split("(")[0]
            a = agg.setdefault(k, [0, 0.0])
            a[0] += 1
            a[1] += e.device_time_total / 1e3
        total = sum(v[1] for v in agg.values())
        res["tensor_cores" if tensor else "fp64_pipe"] = {
            "kernel_ms_total": total,
            "kernels": {k: {"launches": v[0], "ms": v[1], "share": v[1] / total}
                        for k, v in sorted(agg.items(), key=lambda kv: -kv[1][1])}}
    plan.close()
    if not args.no_trace:
        print(json.dumps({"mode": "merge kernel breakdown", "grid": [w.nx, w.ny], "p": 20,
                          "merge_split": args.merge_split, "results": res}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=60.0,
                    help="time budget of the oracle leg over every leaf of the headline workload")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the bumps_p30 / annulus_p24 / uneven blocks of the default run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="both", choices=["both", "fp32", "fp64", "tf32", "bf16"],
                    help="profiling: run one path only")
    ap.add_argument("--leaves", type=int, default=0,
                    help="profiling: condense only the first N leaves (no e2e, no CPU leg)")
    ap.add_argument("--workload", default="bumps_p20", choices=sorted(WORKLOADS),
                    help="bumps_p20 (default, the headline workload) or another seeded workload")
    ap.add_argument("--graph", action="store_true", help="time CUDA-graph replays of the launch")
    ap.add_argument("--merge-solve", action="store_true",
                    help="time hps_merge + hps_solve on the workload's grid (split vs one CTA per merge) and "
                         "SlabLU (hps_slab_factor + hps_slab_solve) for slab widths 4, 8, 16")
    ap.add_argument("--leaf-solve", action="store_true",
                    help="time the leaf solve after the reduced solve: stored S vs re-factored leaves")
    ap.add_argument("--merge-kernels", type=int, default=0, metavar="N",
                    help="profiling mode: hps_merge on an N x N grid of p = 20 leaves (64: bumps_p20), one kernel "
                         "breakdown per parent-map path from the CUDA activity trace")
    ap.add_argument("--merge-split", type=int, default=-1,
                    help="with --merge-kernels: hps_set_merge_split (0: one CTA per merge, a single stream)")
    ap.add_argument("--no-trace", action="store_true", help="with --merge-kernels: run the merges only (for ncu)")
    args = ap.parse_args(argv)
    rank, ws = dist_setup()
    if args.merge_kernels:
        run_merge_kernels(args)
    elif args.leaf_solve:
        run_leaf_solve(args, rank, ws)
    elif args.merge_solve:
        run_merge_solve(args, rank, ws)
    elif args.impl == "reference":
        run_reference(args, rank, ws)
    else:
        run_gpu(args, rank, ws)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
