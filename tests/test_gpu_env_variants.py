"""Variants chosen once per process by environment switches, run in child
processes so that the switch is read fresh: the CTA-pair form of the dense
tensor-core product (GBLA_GEMM_PAIR=1: cta_group::2, 256-row tiles) and the
leaf width of the tensor-core back-substitution of the echelon step
(GBLA_BACK_LEAF).  Each child checks the product against exact int64 numpy
at the k-block bound and whole reductions against the oracle, bit for bit.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
import oracle
from paper_1602_06097_gb300 import gbla, synth

def t16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).cuda()

p = 65521
h = (p - 1) // 2
for M, K in ((384, 512), (384, 513), (640, 2112), (300, 1536)):
    rng = np.random.default_rng(M + K)
    choices = np.array([p - 1, h, h + 1, 1, 0, 32640, p - 32640, 128, p - 128])
    A = rng.choice(choices, size=(M, K))
    B = rng.choice(choices, size=(K, 200))
    C = rng.integers(0, p, size=(M, 200))
    tc = t16(C)
    gbla.modmatmul(t16(A), t16(B), tc, p, sign=-1, variant=gbla.GEMM_TCGEN05)
    want = (C - A.astype(np.int64) @ B.astype(np.int64)) % p
    assert np.array_equal(tc.cpu().numpy().view(np.uint16).astype(np.int64), want), (M, K)
specs = [synth.FLSpec(m=2600, n=3700, npiv=1900, density=0.02, run_len=(16, 64), group=(2, 8), seed=903),
         synth.FLSpec(m=3000, n=3300, npiv=1500, density=0.01, run_len=(4, 32), seed=904, p=32003)]
for spec in specs:
    rp, c, v = synth.fl_matrix(spec)
    for path in (gbla.PATH_SPARSE, gbla.PATH_DENSE):
        for reduced in (False, True):
            res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=reduced, path=path)
            ref = (oracle.rref if reduced else oracle.echelon)(spec.m, spec.n, spec.p, rp, c, v)
            assert res[0] == ref[0], (spec.m, path, reduced)
            for x, y in zip(res[1:4], ref[1:4]):
                assert np.array_equal(np.asarray(x, np.int64), np.asarray(y, np.int64)), (spec.m, path, reduced)
if sys.argv[1:] == ["pair"]:
    rp, c, v = synth.fl_matrix(specs[0])
    res = gbla.reduce(rp, c, v, (specs[0].m, specs[0].n), specs[0].p, path=gbla.PATH_DENSE, stats=True)
    assert res[4]["tc_pair_launches"] > 0, res[4]
print("child ok")
"""


def run_child(env_extra, *args):
    env = dict(os.environ)
    env.update(env_extra)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", CHILD, *args], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "child ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def test_cta_pair_product_and_reductions():
    run_child({"GBLA_GEMM_PAIR": "1"}, "pair")


@pytest.mark.parametrize("leaf", ["128", "256", "1024"])
def test_back_substitution_leaf_widths(leaf):
    run_child({"GBLA_BACK_LEAF": leaf})
