"""The autotuner (gbla_options.autotune): the first calls of a shape bucket
try the open choices (path, leaf width, raster group of the gathered
product) one by one, later calls run the fastest; every call's result is the
same exact one, equal to the oracle's.  Choices the caller fixes are kept."""
import numpy as np
import pytest

import oracle
from paper_1602_06097_gb300 import gbla, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def same(a, b):
    assert a[0] == b[0]
    for x, y in zip(a[1:4], b[1:4]):
        assert np.array_equal(np.asarray(x, np.int64), np.asarray(y, np.int64))


def test_trials_then_the_fastest_all_equal_the_oracle():
    spec = synth.FLSpec(m=2900, n=7000, npiv=2300, density=0.013, run_len=(4, 24), seed=1401)
    rp, c, v = synth.fl_matrix(spec)
    ref = oracle.echelon(spec.m, spec.n, spec.p, rp, c, v)
    states, configs = [], set()
    for _ in range(12):
        res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, autotune=True, stats=True)
        same(res, ref)
        st = res[4]
        states.append(st["tune_state"])
        if st["tune_state"] == 1:
            configs.add((st["path"], st["leaf_width"], st["gather_group_m"]))
        if st["tune_state"] == 2 and states.count(2) >= 3:
            break
    assert states[0] == 1, states
    assert 2 in states and states.index(2) > 0 and all(x == 2 for x in states[states.index(2):]), states
    assert len(configs) >= 4   # leaf 512/1024 x two raster groups (+ the dense path)
    # without autotune the same call reports no tuning
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, stats=True)
    assert res[4]["tune_state"] == 0
    same(res, ref)


def test_fixed_choices_are_kept():
    spec = synth.FLSpec(m=3300, n=9000, npiv=2600, density=0.011, run_len=(4, 24), seed=1402, p=32003)
    rp, c, v = synth.fl_matrix(spec)
    ref = oracle.echelon(spec.m, spec.n, spec.p, rp, c, v)
    for _ in range(4):
        res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, autotune=True, path=gbla.PATH_SPARSE, leaf=512,
                          stats=True)
        same(res, ref)
        assert res[4]["path"] == gbla.PATH_SPARSE and res[4]["leaf_width"] == 512


def test_autotuned_batch_equals_the_plain_batch():
    specs = synth.mixed_batch(48, 20161)
    mats = [synth.fl_matrix(s) + ((s.m, s.n), s.p) for s in specs]
    plain = gbla.reduce_batch(mats, workers=8)
    for _ in range(2):
        tuned = gbla.reduce_batch(mats, workers=8, autotune=True)
        for a, b in zip(plain, tuned):
            same(a, b)
