#!/usr/bin/env python3
"""Benchmark: F4-shaped matrices reduced per second on GB300.

One step = one whole Faugere-Lachartre reduction (pivot analysis and split,
C*A^-1, Schur update, reduced echelon form of D', output assembly) of the
40,000 x 60,000 grouped workload (30,000 designated pivots, 1.5% density,
2-8 runs per row, groups of 2-16 rows sharing ~80% of their pattern; the
non-reduced echelon form), inputs resident in device memory.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbla|reference]

Prints one JSON line (rank 0).  Under torchrun every rank reduces its own
matrix (replicas; no data-path collective) and the time is the maximum over
ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
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
WORKLOAD = "fl_40000x60000"
CPU_SAMPLE_ROWS = 1500


def args_parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbla", choices=["gbla", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink rows, columns and pivots (small cases for profiling)")
    ap.add_argument("--want-reduced", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--extras", action="store_true", help="add the batched-vs-plain and serving measurements")
    ap.add_argument("--batch", type=int, default=32, help="matrices in the batched-vs-plain measurement")
    ap.add_argument("--serve-rate", type=float, default=100.0, help="Poisson arrival rate of the serving run (req/s)")
    ap.add_argument("--serve-requests", type=int, default=160)
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


def profiled_traffic():
    """DRAM bytes per Schur launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    import hashlib
    import re
    try:
        txt = open(os.path.join(ROOT, "profiles", "modgemm_tc_schur_traffic_fl_40000x60000.md")).read()
        src = open(os.path.join(ROOT, "paper_1602_06097_gb300", "csrc", "modgemm.cu"), "rb").read()
    except OSError:
        return None
    m1 = re.search(r"traffic_bytes_per_launch:\s*(\d+)", txt)
    m2 = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", txt)
    if not (m1 and m2) or hashlib.sha256(src).hexdigest() != m2.group(1):
        return None
    return int(m1.group(1))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# --------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(rp, c, v, m, n, p, rows):
    """Time the oracle on a row sample of the workload: every pivot row plus
    the first `rows` non-pivot rows.  The row reduction by the pivot rows costs
    the same per non-pivot row, and the Gauss-Jordan pass on the Schur
    complement grows with the square of its row count, so the whole matrix
    takes t_rows * (m_cd / s) + t_gj * (m_cd / s)^2."""
    import oracle
    piv = oracle.pivots(m, n, rp, c)
    is_piv = np.zeros(m, bool)
    is_piv[piv[piv >= 0]] = True
    nonempty = np.diff(rp) > 0
    cd = np.nonzero(~is_piv & nonempty)[0]
    m_cd = len(cd)
    s = min(rows, m_cd)
    keep = np.sort(np.concatenate([np.nonzero(is_piv)[0], cd[:s]]))
    lens = np.diff(rp)[keep]
    srp = np.zeros(len(keep) + 1, np.int64)
    np.cumsum(lens, out=srp[1:])
    idx = np.repeat(rp[keep], lens) + (np.arange(srp[-1]) - np.repeat(srp[:-1], lens))
    secs = [0.0, 0.0]
    t0 = time.perf_counter()
    oracle.echelon(len(keep), n, p, srp, c[idx], v[idx], phase_seconds=secs)
    wall = time.perf_counter() - t0
    f = m_cd / max(s, 1)
    t_full = secs[0] * f + secs[1] * f * f
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"t_full_s": t_full, "sample_wall_s": wall, "rows": s, "m_cd": m_cd, "phase_s": secs,
            "threads": threads}


def run_reference(a, world, rank):
    """The oracle on the host cores, each step a bounded row sample of the
    same workload scaled to whole matrices per second."""
    if rank != 0:
        return
    from paper_1602_06097_gb300 import synth
    spec = synth.workload(a.workload)
    rp, c, v = synth.fl_matrix(spec)
    vals = []
    last = None
    for i in range(a.warmup + a.steps):
        last = cpu_oracle_sample(rp, c, v, spec.m, spec.n, spec.p, CPU_SAMPLE_ROWS)
        if i >= a.warmup:
            vals.append(1.0 / last["t_full_s"])
    value = float(np.mean(vals))
    sample = (f"oracle echelon on all pivot rows + the first {last['rows']} of {last['m_cd']} non-pivot rows; "
              f"whole-matrix time = t_rows*(m_cd/s) + t_gauss_jordan*(m_cd/s)^2")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": config_of(spec, a),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["threads"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(spec, a):
    return {"workload": a.workload + ("" if a.scale == 1.0 else f"@scale{a.scale}"), "rows": spec.m, "cols": spec.n, "designated_pivots": spec.npiv,
            "p": spec.p, "density": spec.density, "run_len": list(spec.run_len),
            "groups": list(spec.group) if spec.group else None, "want_reduced": a.want_reduced,
            "l2": "inputs larger than L2 (231 MB CSR; >10 GB working set per step)",
            "input": "resident in HBM"}


BATCH_SEED = 20160223   # batched / serving mix


def batched_vs_plain(gbla, synth, count):
    """A batch of F4-shaped matrices of uneven sizes (rows log-uniform in
    500-20,000, columns 1.3-1.6 x rows, 60-80% pivots, 1-5% density, p in
    {65521, 32003}) reduced one call per matrix, then through the batch entry
    point; host inputs and results, copies included in both."""
    specs = synth.mixed_batch(count, BATCH_SEED)
    mats = [synth.fl_matrix(sp) + ((sp.m, sp.n), sp.p) for sp in specs]
    gbla.reduce_batch(mats[:8])                 # warm-up; starts the 8 default batch workers
    for rp, c, v, shape, p in mats[:4]:
        gbla.reduce(rp, c, v, shape, p)
    t0 = time.perf_counter()
    plain = [gbla.reduce(rp, c, v, shape, p)[0] for rp, c, v, shape, p in mats]
    t_plain = time.perf_counter() - t0
    # The first call holds all its results at once and pins new host memory
    # for most of them; a repeated call finds the page-locked result cache
    # warm, as the one-at-a-time calls above do.
    t0 = time.perf_counter()
    first = [r[0] for r in gbla.reduce_batch(mats)]
    t_first = time.perf_counter() - t0
    t0 = time.perf_counter()
    batched = [r[0] for r in gbla.reduce_batch(mats)]
    t_batch = time.perf_counter() - t0
    assert plain == batched == first, "batched ranks differ from one-at-a-time ranks"
    nnz = int(sum(len(mt[1]) for mt in mats))
    return mats, {"matrices": count, "rows": [int(min(sp.m for sp in specs)), int(max(sp.m for sp in specs))],
                  "input_nnz": nnz, "plain_matrices_per_s": count / t_plain, "batched_matrices_per_s": count / t_batch,
                  "batched_first_call_matrices_per_s": count / t_first,
                  "speedup": t_plain / t_batch, "includes": "host inputs and results (H2D/D2H inside)"}


def serving(gbla, mats, rate, nreq):
    """Poisson arrivals (rate req/s) of requests drawn from the batch's
    matrices, served by the request server with continuous batching; latency
    from submit to result ready."""
    rng = np.random.default_rng(BATCH_SEED)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    pick = rng.integers(0, len(mats), size=nreq)
    with gbla.Server(workers=4) as srv:
        tickets = []
        t0 = time.perf_counter()
        for i in range(nreq):
            dt = t0 + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            rp, c, v, shape, p = mats[pick[i]]
            tickets.append(srv.submit(rp, c, v, shape, p))
        lat = []
        for t in tickets:
            code, _, ms = srv.wait(t, 120.0)
            if code != 0:
                raise RuntimeError(f"served request failed with code {code}")
            lat.append(ms)
        wall = time.perf_counter() - t0
    lat = np.asarray(lat)
    return {"rate_req_per_s": rate, "requests": nreq, "matrices_per_s": nreq / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "workers": 4}


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
        res = gbla.reduce_device(d_rp, d_c, d_v, (m, n), p, want_reduced=bool(a.want_reduced), stream=stream)
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

    # dominant kernel: the Schur-update launch of the tensor-core product
    st0 = stats[0]
    m_cd, n_d, npiv = st0["m_cd"], st0["n_d"], st0["npiv"]
    schur_ms = float(np.mean([s["ms_schur"] for s in stats]))
    # algorithmic flops of the Schur launch: its modular multiply-adds over the
    # nonzero staircase of X, times four bf16 digit products of 2 flops each
    flops = 8.0 * float(np.mean([s["schur_mod_ops"] for s in stats]))
    peaks, kind = measured_peaks()
    achieved = flops / (schur_ms / 1e3) / 1e12 if schur_ms > 0 else None
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    mod_ops = float(np.mean([s["mod_ops"] for s in stats]))
    launches = int(sum(s["launches"] for s in stats))

    e2e = None
    if not a.no_e2e:
        # end to end through the public API from pinned host buffers
        h_rp = torch.from_numpy(rp).pin_memory().numpy()
        h_c = torch.from_numpy(c).pin_memory().numpy()
        h_v = torch.from_numpy(v.view(np.int16)).pin_memory().numpy().view(np.uint16)
        k_e2e = max(1, min(a.steps, 3))
        for _ in range(2):   # warm the library's page-locked result cache
            gbla.reduce_host(h_rp, h_c, h_v, (m, n), p, want_reduced=bool(a.want_reduced), stream=stream).free()
        torch.cuda.synchronize()
        d2h = 0
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            # inputs copied in and the whole result copied out inside the call;
            # the step reads the rank and the last row's length on the host
            hr = gbla.reduce_host(h_rp, h_c, h_v, (m, n), p, want_reduced=bool(a.want_reduced), stream=stream)
            d2h = hr.row_ptr.nbytes + hr.col.nbytes + hr.val.nbytes
            _ = int(hr.row_ptr[-1]) + hr.rank
            hr.free()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / k_e2e, dist, "cuda")
        e2e = {"value": world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(rp.nbytes + c.nbytes + v.nbytes),
               "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    extras = {}
    if world == 1 and a.extras:
        mats, extras["batched"] = batched_vs_plain(gbla, synth, a.batch)
        extras["serving"] = serving(gbla, mats, a.serve_rate, a.serve_requests)
    cpu = None
    if world == 1 and not a.no_cpu_baseline:
        cb = cpu_oracle_sample(rp, c, v, m, n, p, CPU_SAMPLE_ROWS)
        cpu = {"value": 1.0 / cb["t_full_s"], "unit": UNIT, "cores": cb["threads"], "kind": "oracle",
               "sample": (f"oracle echelon on all pivot rows + the first {cb['rows']} of {cb['m_cd']} "
                          f"non-pivot rows ({cb['sample_wall_s']:.1f} s); whole-matrix time = "
                          f"t_rows*(m_cd/s) + t_gauss_jordan*(m_cd/s)^2 = {cb['t_full_s']:.0f} s")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u16", "data": "synthetic", "config": config_of(spec, a),
        "modular_gops": mod_ops / (ms_step / 1e3) / 1e9,
        "rank": int(r_out), "out_nnz": int(nnz_out),
        "shape": {"npiv": npiv, "m_cd": m_cd, "n_d": n_d, "rank_d": st0["rank_d"]},
        "phase_ms": {k: float(np.mean([s[k] for s in stats])) for k in
                     ("ms_split", "ms_trsm", "ms_schur", "ms_echelon", "ms_echelon_back", "ms_backsub", "ms_output",
                      "ms_total")},
        "wall_ms_per_step": wall * 1e3 / a.steps,
        "roofline": {"kernel": "modgemm_tc_kernel (Schur update launch)", "bound": "tensor",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": profiled_traffic() if a.workload == WORKLOAD and a.scale == 1.0 else None,
                     "peak_kind": f"bf16 dense sustained, {kind}"},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
