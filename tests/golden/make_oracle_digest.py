"""Write the oracle's result digest for a named workload.

Runs ``oracle.echelon`` (the plain CPU oracle, new order of operations,
Alg. 2 of Sec. 4.3, then Gauss-Jordan of the Schur complement) on the seeded
synthetic workload and stores, in ``oracle_<workload>.json`` beside this
script: the SHA-256 of the generated input (row_ptr int64, col int32,
val uint16, little-endian), the rank, the pivot count, the result's nonzero
count, the SHA-256 of the result arrays in the same encoding, the work
counts [ops_b, ops_c, ops_d, ops_e] in modular multiply-adds, and the
oracle's wall time with the thread count and CPU model of the machine that
ran it.  Only ``oracle/`` and the input generator are called.

    python tests/golden/make_oracle_digest.py fl_40000x60000

With ``--counts-only`` it runs only the oracle's row reduction of Alg. 2
(``oracle.row_counts``) and stores the input digest, the pivot count and the
work counts ops_b and ops_c in ``oracle_counts_<workload>.json``: for a
workload whose Gauss-Jordan pass on the Schur complement the oracle cannot
finish in bounded time.
"""
import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1602_06097_gb300 import synth  # noqa: E402


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
    return platform.processor() or platform.machine()


def counts_only(name):
    spec = synth.workload(name)
    rp, c, v = synth.fl_matrix(spec)
    ops_b, ops_c, npiv, secs = oracle.row_counts(spec.m, spec.n, spec.p, rp, c, v)
    rec = {
        "workload": name,
        "spec": {k: (list(x) if isinstance(x, tuple) else x) for k, x in vars(spec).items()},
        "input_sha256": sha256_csr(rp, c, v),
        "npiv": int(npiv),
        "ops_b": ops_b,
        "ops_c": ops_c,
        "oracle_seconds_row_reduction": secs,
        "threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
        "cpu": cpu_model(),
        "machine": platform.machine(),
    }
    out = os.path.join(HERE, f"oracle_counts_{name}.json")
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


def main(name):
    spec = synth.workload(name)
    rp, c, v = synth.fl_matrix(spec)
    secs, ops = [0.0, 0.0], []
    t0 = time.time()
    rank, orp, oc, ov, npiv = oracle.echelon(spec.m, spec.n, spec.p, rp, c, v, phase_seconds=secs, ops=ops)
    wall = time.time() - t0
    rec = {
        "workload": name,
        "spec": {k: (list(x) if isinstance(x, tuple) else x) for k, x in vars(spec).items()},
        "input_sha256": sha256_csr(rp, c, v),
        "rank": int(rank),
        "npiv": int(npiv),
        "nnz": int(orp[-1]),
        "result_sha256": sha256_csr(orp, oc, ov),
        "ops": [float(x) for x in ops],
        "oracle_seconds": {"total": wall, "row_reduction": secs[0], "gauss_jordan": secs[1]},
        "threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
        "cpu": cpu_model(),
        "machine": platform.machine(),
    }
    out = os.path.join(HERE, f"oracle_{name}.json")
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    name = args[0] if args else "fl_40000x60000"
    counts_only(name) if "--counts-only" in sys.argv else main(name)
