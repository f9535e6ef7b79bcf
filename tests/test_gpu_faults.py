"""Host-side fault injection (no device fault): the allocation after the
next n fails once (gbla_selftest_fail_alloc_after).  Sweeping n from 0 up
drives every allocation failure of a call in turn: each must come back as
GBLA_E_NOMEM with the library's device pool back to where it was (nothing
leaked), and the call that finally succeeds, and every call after, must
still equal the oracle."""
import numpy as np
import pytest

import oracle
from paper_1602_06097_gb300 import gbla, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

NOMEM = 2
SPEC = synth.FLSpec(m=1500, n=2100, npiv=1000, density=0.03, run_len=(8, 40), seed=1201, p=32003)


def same(a, b):
    assert a[0] == b[0]
    for x, y in zip(a[1:4], b[1:4]):
        assert np.array_equal(np.asarray(x, np.int64), np.asarray(y, np.int64))


@pytest.fixture(scope="module")
def mat():
    rp, c, v = synth.fl_matrix(SPEC)
    return rp, c, v


def sweep(run, limit=2000):
    """Returns (allocations the call makes, its result with no fault)."""
    gbla.fail_alloc_after(-1)
    base = gbla.device_bytes_in_use()
    try:
        for n in range(limit):
            gbla.fail_alloc_after(n)
            try:
                out = run()
            except gbla.GblaError as e:
                assert e.code == NOMEM, (n, e)
                assert gbla.device_bytes_in_use() == base, f"pool not released after a fault at allocation {n}"
                continue
            return n, out
        raise AssertionError("the call never completed")
    finally:
        gbla.fail_alloc_after(-1)


@pytest.mark.parametrize("path,reduced,order", [(gbla.PATH_SPARSE, False, 0), (gbla.PATH_SPARSE, True, 0),
                                                (gbla.PATH_DENSE, False, 0), (gbla.PATH_DENSE, True, 0),
                                                (gbla.PATH_DENSE, True, gbla.ORDER_TRSM_FIRST)])
def test_every_allocation_failure_of_a_reduction(mat, path, reduced, order):
    rp, c, v = mat
    n, res = sweep(lambda: gbla.reduce(rp, c, v, (SPEC.m, SPEC.n), SPEC.p, want_reduced=reduced, path=path,
                                       order=order))
    assert n > 10
    ref = (oracle.rref if reduced else oracle.echelon)(SPEC.m, SPEC.n, SPEC.p, rp, c, v)
    same(res, ref)
    same(gbla.reduce(rp, c, v, (SPEC.m, SPEC.n), SPEC.p, want_reduced=reduced, path=path, order=order), ref)


def test_every_allocation_failure_of_a_device_reduction(mat):
    rp, c, v = mat
    d = (torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(), torch.from_numpy(v.view(np.int16)).cuda())

    def run():
        r = gbla.reduce_device(*d, (SPEC.m, SPEC.n), SPEC.p)
        try:
            return r.to_host()
        finally:
            r.free()
    n, res = sweep(run)
    same(res, oracle.echelon(SPEC.m, SPEC.n, SPEC.p, rp, c, v))


def test_every_allocation_failure_of_the_format2_decoder(mat):
    rp, c, v = mat
    buf = synth.encode_format2(SPEC.m, SPEC.n, SPEC.p, rp, c, v)

    def run():
        dm = gbla.decode_format2(buf)
        try:
            return dm.to_host()
        finally:
            dm.free()
    n, (m, drp, dc, dv) = sweep(run)
    assert n > 5 and m == SPEC.m
    assert np.array_equal(drp, rp) and np.array_equal(dc, c) and np.array_equal(dv.view(np.uint16), v)


def test_a_failed_batch_member_leaves_the_others_and_the_pool_intact(mat):
    rp, c, v = mat
    specs = [synth.FLSpec(m=400 + 50 * i, n=600 + 60 * i, npiv=250 + 30 * i, density=0.04, seed=1300 + i)
             for i in range(6)]
    mats = [synth.fl_matrix(s) + ((s.m, s.n), s.p) for s in specs]
    base = gbla.device_bytes_in_use()
    gbla.fail_alloc_after(37)
    with pytest.raises(gbla.GblaError) as e:
        gbla.reduce_batch(mats, workers=3)
    gbla.fail_alloc_after(-1)
    assert e.value.code == NOMEM
    assert gbla.device_bytes_in_use() == base
    for s, mt, r in zip(specs, mats, gbla.reduce_batch(mats, workers=3)):
        same(r, oracle.echelon(s.m, s.n, s.p, *mt[:3]))


def test_a_failed_request_does_not_disturb_the_server(mat):
    rp, c, v = mat
    ref = oracle.echelon(SPEC.m, SPEC.n, SPEC.p, rp, c, v)
    base = gbla.device_bytes_in_use()
    with gbla.Server(workers=1) as srv:
        gbla.fail_alloc_after(20)
        t_bad = srv.submit(rp, c, v, (SPEC.m, SPEC.n), SPEC.p)
        code, res, _ = srv.wait(t_bad, timeout=120.0)
        gbla.fail_alloc_after(-1)
        assert code == NOMEM and res is None
        tickets = [srv.submit(rp, c, v, (SPEC.m, SPEC.n), SPEC.p) for _ in range(3)]
        for t in tickets:
            code, res, _ = srv.wait(t, timeout=120.0)
            assert code == 0
            same(res, ref)
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 4
    assert gbla.device_bytes_in_use() == base


def test_every_allocation_failure_of_a_reduction_with_the_sparse_echelon_pass():
    spec = synth.FLSpec(m=3000, n=9000, npiv=1500, density=0.002, run_len=(1, 4), seed=1501)
    rp, c, v = synth.fl_matrix(spec)
    n, res = sweep(lambda: gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, echelon=gbla.ECHELON_SGE))
    assert n > 10
    same(res, oracle.echelon(spec.m, spec.n, spec.p, rp, c, v))
