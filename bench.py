#!/usr/bin/env python3
"""Benchmark: F4-shaped matrices reduced per second on one GB300, modular GOPS
against the roofline of the dominant kernel, batched against plain.

One step = one whole Faugere-Lachartre reduction (pivot analysis and split,
C*A^-1, Schur update, reduced echelon form of D', output assembly; the
echelon form of the new order) of the 150,000 x 200,000 workload: 120,000
designated pivots, 0.5% density (~149M nonzeros), rows in multiline pairs
sharing ~90% of their pattern, A banded (2,048 pivot columns) in diagonal
blocks of 4,096 with 5% cross-block entries.  Inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbla|reference]

Prints one JSON line (rank 0).  Under torchrun every rank reduces its own
matrix (replicas; no data-path collective) and the time is the maximum over
ranks.  On one GPU the line also carries:
  * "fl_40000x60000": the 40,000 x 60,000 workload on the sparse and the
    dense path, with the oracle's full work counts (modular GOPS) and a
    bit-exact check of the result against the oracle's stored digest, and
    its dense Schur update on each exact product (tcgen05 bf16 digits,
    mma.sync u8, mma.sync f64) against that pipe's own measured peak;
  * "batched": 256 F4 matrices of uneven sizes (rows log-uniform in
    500-20,000, p in {65521, 32003}) one call per matrix against the batch
    entry point, whose reductions overlap on the device;
  * "serving": Poisson request streams at 50-500 req/s served with continuous
    batching, p50/p99 latency and matrices/s.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
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

METRIC = "F4 matrices reduced/sec and modular GOPS vs roofline, batched vs plain, bit-exact"
UNIT = "matrices/s"
WORKLOAD = "fl_150000x200000"
GOLDEN = os.path.join(ROOT, "tests", "golden")


def args_parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbla", choices=["gbla", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink rows, columns and pivots (small cases for profiling)")
    ap.add_argument("--want-reduced", type=int, default=0)
    ap.add_argument("--path", type=int, default=0, help="0 auto, 1 dense, 2 sparse")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the 40k x 60k, batched and serving blocks")
    ap.add_argument("--batch", type=int, default=256, help="matrices in the batched-vs-plain measurement")
    ap.add_argument("--serve-rates", default="50,100,200,500", help="Poisson arrival rates (req/s)")
    ap.add_argument("--serve-pool", type=int, default=12, help="matrices in the serving pool")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="arrival window per rate (at most 100 requests)")
    return ap.parse_args(argv)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_workload(name, scale, rank):
    """One rank's matrix: the named workload (scaled), with a seed of its own,
    so that the ranks reduce independent matrices (weak scaling)."""
    from paper_1602_06097_gb300 import synth
    spec = synth.workload(name) if scale == 1.0 else synth.scaled(name, scale)
    return dataclasses.replace(spec, seed=spec.seed + 1000 * rank)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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


# ------------------------------------------------------ committed records
def profiled_traffic(name="dram_traffic_fl_150000x200000.md",
                     src=os.path.join("paper_1602_06097_gb300", "csrc", "modgemm.cu"), launches=None):
    """DRAM bytes per launch of the dense product from the committed ncu
    summary, if the kernel's source region (named in the summary) still
    hashes as it did when the counters were taken and, given the launches
    per reduction measured now, the summary counted as many (else None)."""
    import re
    try:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        code = open(os.path.join(ROOT, src)).read()
    except OSError:
        return None
    m1 = re.search(r"traffic_bytes_per_launch:\s*(\d+)", txt)
    m2 = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", txt)
    m3 = re.search(r'kernel_region: \S+ "([^"]+)" \.\. "([^"]+)"', txt)
    if not (m1 and m2 and m3):
        return None
    a, b = code.find(m3.group(1)), code.find(m3.group(2))
    if a < 0 or b <= a or hashlib.sha256(code[a:b].encode()).hexdigest() != m2.group(1):
        return None
    m4 = re.search(r"launches_per_reduction:\s*(\d+)", txt)
    if launches is not None and (not m4 or int(m4.group(1)) != int(round(launches))):
        return None
    return int(m1.group(1))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def oracle_record(kind, name):
    """The oracle's stored record of a workload (written by
    tests/golden/make_oracle_digest.py), or None."""
    path = os.path.join(GOLDEN, f"oracle_{kind}{name}.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return None


def sha256_csr(row_ptr, col, val):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(row_ptr, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(col, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(val, dtype="<u2").tobytes())
    return h.hexdigest()


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


# --------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(rp, c, v, m, n, p, budget_s=15.0):
    """Time the oracle's row reduction of Alg. 2 (every non-pivot row reduced
    by the normalised pivot rows) on a sample of the non-pivot rows, doubling
    the sample until it takes budget_s / 3 or more.  The rows are reduced
    independently, so the whole matrix's row reduction takes
    t_sample * m_cd / s; the Gauss-Jordan pass on the Schur complement, which
    the oracle cannot finish at this size in bounded time, is not included:
    1 / t is an upper bound on the oracle's matrices per second."""
    import oracle
    piv = oracle.pivots(m, n, rp, c)
    is_piv = np.zeros(m, bool)
    is_piv[piv[piv >= 0]] = True
    cd = np.nonzero(~is_piv & (np.diff(rp) > 0))[0]
    m_cd = len(cd)
    rng = np.random.default_rng(1602)
    order = rng.permutation(m_cd)
    s = 16
    while True:
        s = min(s, m_cd)
        keep = np.sort(np.concatenate([np.nonzero(is_piv)[0], cd[order[:s]]]))
        lens = np.diff(rp)[keep]
        srp = np.zeros(len(keep) + 1, np.int64)
        np.cumsum(lens, out=srp[1:])
        idx = np.repeat(rp[keep], lens) + (np.arange(srp[-1]) - np.repeat(srp[:-1], lens))
        t0 = time.perf_counter()
        oracle.row_counts(len(keep), n, p, srp, c[idx], v[idx])
        wall = time.perf_counter() - t0
        if wall >= budget_s / 3 or s >= m_cd:
            break
        s *= 2
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t_full = wall * m_cd / s
    return {"t_full_s": t_full, "sample_wall_s": wall, "rows": s, "m_cd": m_cd, "threads": threads}


def cpu_sample_text(cb):
    return (f"oracle row reduction of Alg. 2 for {cb['rows']} of the {cb['m_cd']} non-pivot rows "
            f"(random sample, every pivot row) in {cb['sample_wall_s']:.1f} s on {cb['threads']} threads "
            f"({cpu_model()}), scaled by m_cd/rows to {cb['t_full_s']:.0f} s per matrix; the Gauss-Jordan "
            f"pass on the Schur complement is not timed, so the value is an upper bound on the oracle's rate")


def run_reference(a, world, rank):
    """The oracle on the host cores (rank 0 only), each step a bounded sample
    of the same workload scaled to matrices per second."""
    if rank != 0:
        return
    from paper_1602_06097_gb300 import synth
    spec = synth.workload(a.workload) if a.scale == 1.0 else synth.scaled(a.workload, a.scale)
    rp, c, v = synth.fl_matrix(spec)
    budget = max(2.0, 120.0 / max(1, a.steps + a.warmup))
    vals, last = [], None
    for i in range(a.warmup + a.steps):
        last = cpu_oracle_sample(rp, c, v, spec.m, spec.n, spec.p, budget)
        if i >= a.warmup:
            vals.append(1.0 / last["t_full_s"])
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": config_of(spec, a),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["threads"], "kind": "oracle",
                             "sample": cpu_sample_text(last)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(spec, a):
    return {"workload": a.workload + ("" if a.scale == 1.0 else f"@scale{a.scale}"), "rows": spec.m,
            "cols": spec.n, "designated_pivots": spec.npiv, "p": spec.p, "density": spec.density,
            "run_len": list(spec.run_len), "band": spec.band, "block": spec.block if spec.band else None,
            "groups": list(spec.group) if spec.group else None, "want_reduced": a.want_reduced,
            "path": ["auto", "dense", "sparse"][a.path],
            "l2": "inputs larger than L2 (the CSR input alone exceeds 129 MB)", "input": "resident in HBM"}


# ------------------------------------------------------------ extra blocks
def reduce_steps(gbla, d, shape, p, stream, steps, path=0):
    import torch
    stats = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        r = gbla.reduce_device(*d, shape, p, stream=stream, path=path)
        stats.append(r.stats)
        r.free()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps, stats


def mean_of(stats, key):
    return float(np.mean([s[key] for s in stats]))


def ms_step_est(stats):
    return mean_of(stats, "ms_total")


def block_40000x60000(gbla, synth, peak, stream):
    """The 40,000 x 60,000 workload on both paths with the oracle's full work
    counts, and its result against the oracle's stored digest."""
    import torch
    name = "fl_40000x60000"
    spec = synth.workload(name)
    rp, c, v = synth.fl_matrix(spec)
    d = (torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(), torch.from_numpy(v.view(np.int16)).cuda())
    rec = oracle_record("", name)
    out = {"rows": spec.m, "cols": spec.n}
    for path, label in ((2, "sparse"), (1, "dense")):
        reduce_steps(gbla, d, (spec.m, spec.n), spec.p, stream, 2, path)
        ms, stats = reduce_steps(gbla, d, (spec.m, spec.n), spec.p, stream, 5, path)
        blk = {"ms_per_matrix": ms, "matrices_per_s": 1e3 / ms,
               "phase_ms": {k: mean_of(stats, k) for k in ("ms_split", "ms_trsm", "ms_schur", "ms_echelon",
                                                           "ms_output")}}
        if rec:
            ops = rec["ops"]
            blk["modular_gops"] = (ops[0] + ops[1] + ops[2] + ops[3]) / (ms / 1e3) / 1e9
            schur_ms = blk["phase_ms"]["ms_schur"]
            blk["schur_tflops_algorithmic"] = 8.0 * ops[1] / (schur_ms / 1e3) / 1e12
            blk["schur_frac_algorithmic"] = blk["schur_tflops_algorithmic"] / peak
        if label == "sparse":
            ex = mean_of(stats, "schur_exec_mod_ops")
            blk["schur_tflops_executed"] = 8.0 * ex / (blk["phase_ms"]["ms_schur"] / 1e3) / 1e12
        out[label] = blk
    r = gbla.reduce_device(*d, (spec.m, spec.n), spec.p, stream=stream)
    rank, orp, oc, ov = r.to_host()
    r.free()
    digest = sha256_csr(orp, oc, ov)
    out["bit_exact_vs_oracle"] = bool(rec and digest == rec["result_sha256"] and
                                      sha256_csr(rp, c, v) == rec["input_sha256"])
    if rec:
        out["oracle_counts"] = {"ops_b": rec["ops"][0], "ops_c": rec["ops"][1], "ops_d": rec["ops"][2],
                                "ops_e": rec["ops"][3]}
        out["oracle_whole_matrix"] = {"seconds": rec["oracle_seconds"]["total"], "threads": rec["threads"],
                                      "cpu": rec["cpu"], "kind": "measured, whole matrix (recorded run)"}
    out["speedup_sparse_over_dense"] = out["dense"]["ms_per_matrix"] / out["sparse"]["ms_per_matrix"]
    out["schur_variants"] = schur_variants(gbla, d, (spec.m, spec.n), spec.p, stream, peak, rec)
    out["reduced_form_orders"] = reduced_form_orders(gbla, d, (spec.m, spec.n), spec.p, stream)
    return out


def reduced_form_orders(gbla, d, shape, p, stream):
    """RREF of the workload in the new order (Sec. 4.3: C A^-1, Schur update,
    echelon of D', then A^-1 B and its fix-up) against the original order
    (Sec. 4.1: A^-1 B first, Schur update with C, echelon, fix-up), one
    event-timed reduction each after a warm-up, and the two results compared
    on the device."""
    import torch
    out, res = {}, {}
    for order, label in ((0, "new_order"), (1, "trsm_first")):
        gbla.reduce_device(*d, shape, p, want_reduced=True, order=order, stream=stream).free()
        r = gbla.reduce_device(*d, shape, p, want_reduced=True, order=order, stream=stream)
        st = r.stats
        res[label] = r
        out[label] = {"ms": st["ms_total"], "path": ["", "dense", "sparse"][int(st["path"])],
                      "phase_ms": {k: st[k] for k in ("ms_split", "ms_trsm", "ms_schur", "ms_echelon", "ms_backsub",
                                                      "ms_output")}}
    a, b = res["new_order"], res["trsm_first"]
    out["equal"] = bool(a.rank == b.rank and a.nnz == b.nnz and
                        all(torch.equal(x, y) for x, y in zip(a.tensors(), b.tensors())))
    a.free()
    b.free()
    return out


def schur_variants(gbla, d, shape, p, stream, bf16_peak, rec):
    """The dense path's Schur update D <- D - X*B on each exact product
    (tcgen05 bf16 digits; mma.sync u8 bytes; mma.sync f64 balanced residues),
    one reduction each, the Schur phase event-timed.  Each is set against its
    own pipe's peak: bf16 the measured cuBLAS figure, u8 and f64 the library's
    issue-rate microbenchmark run here.  Work = the product's multiply-adds
    (zero staircase excluded) x the instruction ops each needs: 4 bf16 digit
    products (8 flops), 4 byte products (8 ops), 1 fp64 fma (2 flops)."""
    peaks = {"fp64": gbla.pipe_peak(gbla.GEMM_FP64, stream), "u8": gbla.pipe_peak(gbla.GEMM_U8, stream)}
    out = {"peaks": {"tcgen05_bf16_tflops": bf16_peak, "mma_sync_u8_tops_measured": peaks["u8"],
                     "mma_sync_fp64_tflops_measured": peaks["fp64"]}}
    for variant, label, per_op, pk in ((gbla.GEMM_TCGEN05, "tcgen05_bf16", 8.0, bf16_peak),
                                       (gbla.GEMM_U8, "mma_sync_u8", 8.0, peaks["u8"]),
                                       (gbla.GEMM_FP64, "mma_sync_fp64", 2.0, peaks["fp64"])):
        r = gbla.reduce_device(*d, shape, p, stream=stream, path=1, variant=variant)
        st = r.stats
        rank, orp, oc, ov = r.to_host()
        r.free()
        ms, ops = st["ms_schur"], st["schur_mod_ops"]
        ach = per_op * ops / (ms / 1e3) / 1e12 if ms > 0 else None
        out[label] = {"schur_ms": ms, "reduction_ms": st["ms_total"], "schur_mod_ops": ops, "ops_per_mod_op": per_op,
                      "achieved": ach, "peak": pk, "frac_of_own_peak": ach / pk if ach else None,
                      "bit_exact_vs_oracle": bool(rec and sha256_csr(orp, oc, ov) == rec["result_sha256"])}
    return out


def format2_block(gbla, synth, spec, rp, c, v, d, stream, hbm_peak):
    """The workload written as a Format 2 file (Sec. 3.2: column runs,
    coefficients stored once per polynomial) and decoded on the device from a
    page-locked host buffer.  Decode time = the decoder's event-timed device
    work after the file's sections are on the device; its algorithmic bytes =
    the file's sections read once + the CSR written (8 (m+1) + 6 nnz).  The
    decoded CSR must equal the generated one, and the decoded matrix,
    reduced in place, must give the direct reduction's rank and result."""
    import torch
    t0 = time.perf_counter()
    buf = synth.encode_format2(spec.m, spec.n, spec.p, rp, c, v)
    enc_s = time.perf_counter() - t0
    pinned = torch.frombuffer(bytearray(buf), dtype=torch.uint8).pin_memory().numpy()
    gbla.decode_format2(pinned, stream=stream, timed=True).free()
    dev_ms, e2e_ms = [], []
    for i in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dm = gbla.decode_format2(pinned, stream=stream, timed=True)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        dev_ms.append(dm.decode_ms)
        if i < 2:
            dm.free()
    csr_bytes = 8 * (spec.m + 1) + 6 * len(c)
    file_bytes = len(buf)
    ms = statistics.median(dev_ms)
    out = {"file_bytes": file_bytes, "csr_bytes": csr_bytes, "file_over_csr": file_bytes / csr_bytes,
           "encode_s_host": enc_s, "decode_ms": ms,
           "roofline": {"bound": "hbm", "unit": "GB/s", "algorithmic_bytes": file_bytes + csr_bytes,
                        "achieved": (file_bytes + csr_bytes) / (ms / 1e3) / 1e9, "peak": hbm_peak,
                        "frac": (file_bytes + csr_bytes) / (ms / 1e3) / 1e9 / hbm_peak},
           "e2e_ms_from_pinned_host": statistics.median(e2e_ms)}
    try:
        trp, tc, tv = dm.tensors()
        out["decoded_equals_input"] = bool(torch.equal(trp, d[0]) and torch.equal(tc, d[1]) and torch.equal(tv, d[2]))
        r1 = gbla.reduce_device(trp, tc, tv, (dm.m, dm.n), dm.p, stream=stream)
        r2 = gbla.reduce_device(*d, (spec.m, spec.n), spec.p, stream=stream)
        try:
            out["reduced_in_place_equals_direct"] = bool(
                r1.rank == r2.rank and r1.nnz == r2.nnz and all(torch.equal(x, y) for x, y in
                                                                 zip(r1.tensors(), r2.tensors())))
        finally:
            r1.free()
            r2.free()
    finally:
        dm.free()
    return out


def sparse_d_block(gbla, synth, stream):
    """The echelon step's forward passes on a workload whose Schur complement
    stays sparse: column panels against the sparse SGE (Alg. 3, Sec. 5.1)
    and the automatic choice, one warm-up and three event-timed reductions
    each; the results are compared on the device."""
    import torch
    name = "fl_sparse_d_40000x120000"
    spec = synth.workload(name)
    rp, c, v = synth.fl_matrix(spec)
    d = (torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(), torch.from_numpy(v.view(np.int16)).cuda())
    out = {"workload": name, "rows": spec.m, "cols": spec.n, "nnz": int(len(c))}
    keep = {}
    for ech, label in ((1, "panels"), (2, "sge"), (0, "auto")):
        gbla.reduce_device(*d, (spec.m, spec.n), spec.p, echelon=ech, stream=stream).free()
        runs = []
        for i in range(3):
            r = gbla.reduce_device(*d, (spec.m, spec.n), spec.p, echelon=ech, stream=stream)
            runs.append(r.stats)
            if i == 2:
                keep[label] = r
            else:
                r.free()
        out[label] = {"ms_per_matrix": statistics.median(x["ms_total"] for x in runs),
                      "ms_echelon": statistics.median(x["ms_echelon"] for x in runs),
                      "forward_pass": ["", "panels", "sge"][int(runs[-1]["echelon_method"])],
                      "d_density": runs[-1]["d_density"]}
    ref = keep["panels"]
    out["results_equal"] = all(
        r.rank == ref.rank and r.nnz == ref.nnz and all(torch.equal(x, y) for x, y in zip(r.tensors(), ref.tensors()))
        for r in keep.values())
    for r in keep.values():
        r.free()
    out["sge_speedup_on_echelon"] = out["panels"]["ms_echelon"] / out["sge"]["ms_echelon"]
    return out


def wide_limbs_block(gbla, stream, peak):
    """The exact modular product for 32-bit coefficients (four bf16 digits per
    residue, seven fp32 accumulators) on an 8,192^3 product with p = 2^31 - 1,
    against the 16-bit product (two digits) on the same shape with p = 65521:
    each call event-timed including its digit-plane conversions, after a
    warm-up.  Work: 16 (32-bit) or 4 (16-bit) digit products per modular
    multiply-add, 2 flops each."""
    import torch
    n = 8192
    out = {"shape": [n, n, n]}
    for label, p, dt, fn, prods in (("u32_p2147483647", 2147483647, torch.int32, gbla.modmatmul32, 16),
                                    ("u16_p65521", 65521, torch.int16, gbla.modmatmul, 4)):
        hi = min(p, 2 ** 31 - 1)
        A = torch.randint(0, hi, (n, n), dtype=torch.int64, device="cuda")
        B = torch.randint(0, hi, (n, n), dtype=torch.int64, device="cuda")
        if dt == torch.int16:
            A, B = (A.to(torch.int32).to(torch.int16)), (B.to(torch.int32).to(torch.int16))
        else:
            A, B = A.to(torch.int32), B.to(torch.int32)
        C = torch.zeros((n, n), dtype=dt, device="cuda")
        fn(A, B, C, p, stream=stream)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(3):
            ev0.record(stream)
            fn(A, B, C, p, stream=stream)
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        t = min(ms) / 1e3
        out[label] = {"ms": t * 1e3, "modular_tops": n ** 3 / t / 1e12,
                      "bf16_tflops": 2 * prods * n ** 3 / t / 1e12, "frac_of_bf16_peak": 2 * prods * n ** 3 / t / 1e12 / peak}
        del A, B, C
    torch.cuda.empty_cache()
    return out


BATCH_SEED = 20160223   # batched mix (256 matrices)
SERVE_SEED = 20160224   # serving pool


def batched_vs_plain(gbla, synth, count):
    """A batch of F4-shaped matrices of uneven sizes (rows log-uniform in
    500-20,000, columns 1.3-1.6 x rows, 60-80% pivots, 1-5% density, p in
    {65521, 32003}) reduced one call per matrix, then through the batch entry
    point (8 workers whose reductions overlap on the device).  Device-resident:
    inputs in HBM, results left on the device (the plain calls on one
    stream).  Host: page-locked host inputs and host results, copies inside
    both."""
    import torch
    specs = synth.mixed_batch(count, BATCH_SEED)
    t0 = time.perf_counter()
    mats = [synth.fl_matrix(sp) + ((sp.m, sp.n), sp.p) for sp in specs]
    gen_s = time.perf_counter() - t0
    dev = [(torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(), torch.from_numpy(v.view(np.int16)).cuda(),
            shape, p) for rp, c, v, shape, p in mats]
    stream = torch.cuda.current_stream()
    out = {"matrices": count, "rows": [int(min(sp.m for sp in specs)), int(max(sp.m for sp in specs))],
           "primes": sorted({int(sp.p) for sp in specs}), "input_nnz": int(sum(len(mt[1]) for mt in mats)),
           "generate_s": gen_s, "workers": 8}
    # device-resident
    for r in gbla.reduce_batch_device(dev[:16], workers=8):
        r.free()
    for d in dev[:4]:
        gbla.reduce_device(*d, stream=stream).free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = []
    for d in dev:
        r = gbla.reduce_device(*d, stream=stream)
        plain.append(r)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    batched = gbla.reduce_batch_device(dev, workers=8)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    # the same batch with the autotuner: one pass runs the trials of every
    # shape bucket, the timed pass after it runs each bucket's fastest choice
    for r in gbla.reduce_batch_device(dev, workers=8, autotune=True):
        r.free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tuned = gbla.reduce_batch_device(dev, workers=8, autotune=True)
    torch.cuda.synchronize()
    t_tuned = time.perf_counter() - t0
    same = same_tuned = True
    for a, b, c_ in zip(plain, batched, tuned):
        ta, tb, tt = a.tensors(), b.tensors(), c_.tensors()
        same = same and a.rank == b.rank and all(torch.equal(x, y) for x, y in zip(ta, tb))
        same_tuned = same_tuned and a.rank == c_.rank and all(torch.equal(x, y) for x, y in zip(ta, tt))
    for r in plain + batched + tuned:
        r.free()
    out["device"] = {"plain_matrices_per_s": count / t_plain, "batched_matrices_per_s": count / t_batch,
                     "speedup": t_plain / t_batch, "batched_equals_plain": bool(same),
                     "autotuned_matrices_per_s": count / t_tuned, "autotuned_speedup": t_plain / t_tuned,
                     "autotuned_equals_plain": bool(same_tuned),
                     "includes": "inputs resident in HBM, results left on the device"}
    # host inputs (page-locked) and host results
    pinned = [(torch.from_numpy(rp).pin_memory().numpy(), torch.from_numpy(c).pin_memory().numpy(),
               torch.from_numpy(v.view(np.int16)).pin_memory().numpy().view(np.uint16), shape, p)
              for rp, c, v, shape, p in mats]
    gbla.reduce_batch(pinned, workers=8)   # warms the page-locked result cache for a whole batch
    t0 = time.perf_counter()
    plain_h = [gbla.reduce(*m) for m in pinned]
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    batched_h = gbla.reduce_batch(pinned, workers=8)
    t_batch = time.perf_counter() - t0
    same = all(a[0] == b[0] and all(np.array_equal(x, y) for x, y in zip(a[1:], b[1:]))
               for a, b in zip(plain_h, batched_h))
    out["host"] = {"plain_matrices_per_s": count / t_plain, "batched_matrices_per_s": count / t_batch,
                   "speedup": t_plain / t_batch, "batched_equals_plain": bool(same),
                   "includes": "page-locked host inputs and host results (H2D/D2H inside both)"}
    out["speedup"] = out["device"]["speedup"]
    return out


def fingerprint(res):
    """A cheap key of a result: rank, row pointers and every 61st column and
    value (the tests compare served results in full)."""
    r, rp, c, v = res
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(rp, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(c[::61], dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(v[::61], dtype="<u2").tobytes())
    return int(r), h.hexdigest()


def serving(gbla, synth, rates, pool, seconds, max_requests=100):
    """Poisson request streams drawn from a pool of seeded F4 matrices (rows
    log-uniform in 1,000-50,000, p in {32003, 65521}), served by the request
    server (8 workers, admission by device-memory footprint, requests overlap
    on the device); latency from submit to result ready (server-side); a
    waiter thread collects results as they complete, and every served result
    must match the same request reduced alone."""
    specs = synth.mixed_batch(pool, SERVE_SEED, rows=(1000, 50000), primes=(32003, 65521))
    mats = [synth.fl_matrix(sp) + ((sp.m, sp.n), sp.p) for sp in specs]
    solo = [fingerprint(gbla.reduce(*m)) for m in mats]
    out = []
    for rate in rates:
        rng = np.random.default_rng(SERVE_SEED + int(rate))
        nreq = int(max(20, min(max_requests, rate * seconds)))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
        pick = rng.integers(0, len(mats), size=nreq)
        lat, ok, failed = [], [True], []
        with gbla.Server(workers=8) as srv:
            tickets = []
            cv = threading.Condition()

            def waiter():
                for i in range(nreq):
                    with cv:
                        cv.wait_for(lambda: len(tickets) > i)
                        t = tickets[i]
                    code, res, ms = srv.wait(t, 300.0)
                    if code != 0:
                        failed.append(code)
                        continue
                    ok[0] = ok[0] and fingerprint(res) == solo[pick[i]]
                    lat.append(ms)

            th = threading.Thread(target=waiter)
            th.start()
            t0 = time.perf_counter()
            for i in range(nreq):
                dt = t0 + arrivals[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                t = srv.submit(*mats[pick[i]])
                with cv:
                    tickets.append(t)
                    cv.notify()
            th.join()
            wall = time.perf_counter() - t0
        if failed:
            raise RuntimeError(f"served requests failed with codes {sorted(set(failed))}")
        lat = np.asarray(lat)
        out.append({"rate_req_per_s": rate, "requests": nreq, "matrices_per_s": nreq / wall,
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "mean_ms": float(lat.mean()), "results_equal_solo": bool(ok[0])})
    return {"pool": pool, "pool_rows": [int(min(sp.m for sp in specs)), int(max(sp.m for sp in specs))],
            "pool_nnz": int(sum(len(mt[1]) for mt in mats)), "workers": 8, "rates": out}


# --------------------------------------------------------------- GPU arm
def main():
    a = args_parse()
    world, rank, local = dist_env()
    if a.impl == "reference":
        run_reference(a, world, rank)
        return
    import torch
    from paper_1602_06097_gb300 import gbla, synth
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    gbla.load()
    spec = rank_workload(a.workload, a.scale, rank)
    rp, c, v = synth.fl_matrix(spec)
    m, n, p = spec.m, spec.n, spec.p
    d_rp = torch.from_numpy(rp).cuda()
    d_c = torch.from_numpy(c).cuda()
    d_v = torch.from_numpy(v.view(np.int16)).cuda()
    stream = torch.cuda.current_stream()

    def step():
        res = gbla.reduce_device(d_rp, d_c, d_v, (m, n), p, want_reduced=bool(a.want_reduced), stream=stream,
                                 path=a.path, kernel_times=True)
        st, r, nnz = res.stats, res.rank, res.nnz
        res.free()
        return st, r, nnz

    for _ in range(a.warmup):
        st, r_out, nnz_out = step()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stats = []
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(a.steps):
            stats.append(step()[0])
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    ms_step = ms_total / a.steps
    value = world * a.steps / (ms_total / 1e3)

    st0 = stats[0]
    peaks, kind = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    schur_ms = mean_of(stats, "ms_schur")
    launches = int(sum(s["launches"] for s in stats))
    # Algorithmic work from the oracle's counters (not from the GPU code):
    # ops_b, ops_c of Alg. 2's row reduction on this exact input.
    counts = oracle_record("counts_", a.workload) if (a.scale == 1.0 and rank == 0) else None
    if counts and counts.get("input_sha256") != sha256_csr(rp, c, v):
        counts = None
    ops_c = counts["ops_c"] if counts else None
    exec_ops = mean_of(stats, "schur_exec_mod_ops")
    # Per-kernel live timings (events around every launch of the two
    # tensor-core kernels inside the timed region) and their work.
    tc_ms, g_ms = mean_of(stats, "tc_ms"), mean_of(stats, "gather_ms")
    tc_n, g_n = mean_of(stats, "tc_launches"), mean_of(stats, "gather_launches")
    tc_ops = mean_of(stats, "tc_mod_ops")
    kernels = {
        "modgemm_tc_kernel": {"launches_per_step": tc_n, "ms_per_step": tc_ms,
                              "avg_launch_ms": tc_ms / tc_n if tc_n else None,
                              "mod_ops_per_step": tc_ops,
                              "tflops": 8.0 * tc_ops / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None,
                              "work": "dense products (leaf solves X_J = C_J Z_J, echelon waves, back-"
                                      "substitution): valid rows x columns x K run of every tile, counted on "
                                      "the device; 8 flops per modular multiply-add"},
        "modgemm_gather_kernel": {"launches_per_step": g_n, "ms_per_step": g_ms,
                                  "avg_launch_ms": g_ms / g_n if g_n else None,
                                  "work": "K-compacted sparse products (C*A^-1 updates and the Schur update)"}}
    schur = {"kernel": "modgemm_gather_kernel, the Schur update launch (one per step)", "bound": "tensor",
             "unit": "TFLOP/s", "peak": peak, "launch_ms": schur_ms,
             "algorithmic": "oracle ops_c x 8 flops (4 bf16 digit products per modular multiply-add)",
             "achieved": 8.0 * ops_c / (schur_ms / 1e3) / 1e12 if (ops_c and schur_ms > 0) else None,
             "executed_tflops": 8.0 * exec_ops / (schur_ms / 1e3) / 1e12 if schur_ms > 0 else None}
    schur["frac"] = schur["achieved"] / peak if schur["achieved"] else None
    schur["executed_frac"] = schur["executed_tflops"] / peak if schur["executed_tflops"] else None
    if tc_ms >= g_ms and tc_ms > 0:
        roofline = {"kernel": f"modgemm_tc_kernel (dominant: {tc_ms:.1f} ms of {ms_step_est(stats):.1f} ms per "
                              f"step over {tc_n:.0f} launches; the gathered product {g_ms:.1f} ms)",
                    "bound": "tensor", "unit": "TFLOP/s", "peak": peak, "peak_kind": f"bf16 dense sustained, {kind}",
                    "achieved": kernels["modgemm_tc_kernel"]["tflops"],
                    "frac": kernels["modgemm_tc_kernel"]["tflops"] / peak,
                    "algorithmic": "M x N x K of the dense products over each tile's K run, 8 flops per modular "
                                   "multiply-add (4 bf16 digit products)",
                    "avg_launch_ms": kernels["modgemm_tc_kernel"]["avg_launch_ms"],
                    "traffic": profiled_traffic(launches=tc_n) if (a.workload == WORKLOAD and a.scale == 1.0) else None,
                    "traffic_source": "profiles/dram_traffic_fl_150000x200000.md (ncu, mean over the dense "
                                      "product's launches of one reduction)"}
    else:
        roofline = dict(schur, peak_kind=f"bf16 dense sustained, {kind}", traffic=None)
        roofline["kernel"] = (f"modgemm_gather_kernel (dominant: {g_ms:.1f} ms per step over {g_n:.0f} launches); "
                              "figures of its Schur launch")

    e2e = None
    if not a.no_e2e:
        # end to end through the public API from pinned host buffers
        h_rp = torch.from_numpy(rp).pin_memory().numpy()
        h_c = torch.from_numpy(c).pin_memory().numpy()
        h_v = torch.from_numpy(v.view(np.int16)).pin_memory().numpy().view(np.uint16)
        k_e2e = max(1, min(a.steps, 5))
        for _ in range(2):   # warm the library's page-locked result cache
            gbla.reduce_host(h_rp, h_c, h_v, (m, n), p, want_reduced=bool(a.want_reduced), stream=stream,
                             path=a.path).free()
        torch.cuda.synchronize()
        d2h = 0
        steps_ms = []
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            # inputs copied in and the whole result copied out inside the call;
            # the step reads the rank and the last row's length on the host
            ts = time.perf_counter()
            hr = gbla.reduce_host(h_rp, h_c, h_v, (m, n), p, want_reduced=bool(a.want_reduced), stream=stream,
                                  path=a.path)
            d2h = hr.row_ptr.nbytes + hr.col.nbytes + hr.val.nbytes
            _ = int(hr.row_ptr[-1]) + hr.rank
            st_h = hr.stats
            hr.free()
            steps_ms.append({"wall": round((time.perf_counter() - ts) * 1e3, 2),
                             "split_with_h2d": round(st_h["ms_split"], 2), "output_with_d2h": round(st_h["ms_output"], 2)})
        torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / k_e2e, dist, "cuda")
        e2e = {"value": world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(rp.nbytes + c.nbytes + v.nbytes),
               "d2h_bytes_per_step": int(d2h), "steps": k_e2e, "per_step_ms": steps_ms}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not a.no_cpu_baseline:
        cb = cpu_oracle_sample(rp, c, v, m, n, p)
        cpu = {"value": 1.0 / cb["t_full_s"], "unit": UNIT, "cores": cb["threads"], "kind": "oracle",
               "sample": cpu_sample_text(cb)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u16", "data": "synthetic", "config": config_of(spec, a),
        "modular_gops": ((counts["ops_b"] + counts["ops_c"]) / (ms_step / 1e3) / 1e9) if counts else None,
        "modular_ops": ({"ops_b": counts["ops_b"], "ops_c": counts["ops_c"], "ops_d": None, "ops_e": 0,
                         "source": "oracle.row_counts on this input (tests/golden/oracle_counts_"
                                   f"{a.workload}.json); ops_d (Gauss-Jordan of the Schur complement) is beyond "
                                   "the oracle's bounded time at this size and not included"} if counts else None),
        "rank": int(r_out), "out_nnz": int(nnz_out),
        "shape": {"npiv": st0["npiv"], "m_cd": st0["m_cd"], "n_d": st0["n_d"], "rank_d": st0["rank_d"],
                  "path": ["", "dense", "sparse"][int(st0["path"])], "list_a": st0["list_a"],
                  "list_b": st0["list_b"], "leaf_width": st0["leaf_width"]},
        "phase_ms": {k: mean_of(stats, k) for k in
                     ("ms_split", "ms_trsm", "ms_schur", "ms_echelon", "ms_echelon_back", "ms_backsub", "ms_output",
                      "ms_total")},
        "wall_ms_per_step": wall * 1e3 / a.steps,
        "roofline": roofline, "roofline_schur": schur, "kernels": kernels,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
    }
    if world == 1 and not a.no_extras:
        extras = {}
        hbm = peaks.get("hbm_gbs")
        for key, fn in (("format2", lambda: format2_block(gbla, synth, spec, rp, c, v, (d_rp, d_c, d_v), stream, hbm)),
                        ("fl_40000x60000", lambda: block_40000x60000(gbla, synth, peak, stream)),
                        ("sparse_d", lambda: sparse_d_block(gbla, synth, stream)),
                        ("wide_limbs", lambda: wide_limbs_block(gbla, stream, peak)),
                        ("batched", lambda: batched_vs_plain(gbla, synth, a.batch)),
                        ("serving", lambda: serving(gbla, synth, [float(x) for x in a.serve_rates.split(",")],
                                                    a.serve_pool, a.serve_seconds))):
            try:
                t0 = time.perf_counter()
                extras[key] = fn()
                extras[key]["block_wall_s"] = time.perf_counter() - t0
            except Exception as exc:   # an extra block never hides the main measurement
                extras[key] = {"error": f"{type(exc).__name__}: {exc}"}
        line.update(extras)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
