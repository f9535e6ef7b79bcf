"""Batch and server: results through the C ABI equal the one-at-a-time
reduction (and the oracle), alone and in the mix."""
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


def mixed_specs(n, seed):
    """F4-shaped matrices of uneven sizes (rows log-uniform, columns 1.3-1.6x
    rows, 60-80% pivots, 1-5% density), p in {65521, 32003}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        m = int(np.exp(rng.uniform(np.log(150), np.log(1800))))
        ncols = int(m * rng.uniform(1.3, 1.6))
        npiv = int(m * rng.uniform(0.6, 0.8))
        out.append(synth.FLSpec(m=m, n=ncols, npiv=npiv, p=int(rng.choice([65521, 32003])),
                                density=float(rng.uniform(0.01, 0.05)), run_len=(4, 32), seed=seed * 1000 + i))
    return out


def test_batch_equals_solo_and_oracle():
    specs = mixed_specs(14, 7)
    mats = [synth.fl_matrix(s) + ((s.m, s.n), s.p) for s in specs]
    batch = gbla.reduce_batch(mats, workers=6)
    for s, mt, res in zip(specs, mats, batch):
        rp, c, v, shape, p = mt
        solo = gbla.reduce(rp, c, v, shape, p)
        same(res, solo)
    for s, mt, res in list(zip(specs, mats, batch))[:4]:
        rp, c, v, shape, p = mt
        same(res, oracle.echelon(s.m, s.n, s.p, rp, c, v)[:4])


def test_batch_reduced_form_and_bad_member():
    specs = mixed_specs(5, 8)
    mats = [synth.fl_matrix(s) + ((s.m, s.n), s.p) for s in specs]
    res = gbla.reduce_batch(mats, want_reduced=True, workers=3)
    for s, mt, r in zip(specs, mats, res):
        rp, c, v, shape, p = mt
        same(r, oracle.rref(s.m, s.n, s.p, rp, c, v))
    bad = list(mats)
    rp, c, v, shape, p = bad[2]
    v2 = v.copy()
    v2[0] = 0                                  # explicit zero: invalid member
    bad[2] = (rp, c, v2, shape, p)
    with pytest.raises(gbla.GblaError):
        gbla.reduce_batch(bad, workers=3)


def test_server_results_equal_solo_in_the_mix():
    specs = mixed_specs(24, 9)
    mats = [synth.fl_matrix(s) + ((s.m, s.n), s.p) for s in specs]
    solo = [gbla.reduce(rp, c, v, shape, p) for rp, c, v, shape, p in mats]
    with gbla.Server(workers=6) as srv:
        tickets = [srv.submit(rp, c, v, shape, p) for rp, c, v, shape, p in mats]
        lat = []
        for t, ref in zip(tickets, solo):
            code, res, ms = srv.wait(t, timeout=120.0)
            assert code == 0
            same(res, ref)
            lat.append(ms)
        st = srv.stats()
    assert st["completed"] == len(mats) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert st["mem_in_use"] == 0 and st["queued"] == 0 and st["running"] == 0


def test_server_budget_admission_and_cancel():
    """A budget below every request's footprint admits one request at a time
    (a request larger than the budget runs alone); queued requests can be
    cancelled; a malformed request fails alone."""
    specs = mixed_specs(6, 10)
    mats = [synth.fl_matrix(s) + ((s.m, s.n), s.p) for s in specs]
    with gbla.Server(mem_budget=1, workers=4) as srv:
        tickets = [srv.submit(rp, c, v, shape, p) for rp, c, v, shape, p in mats]
        assert srv.stats()["running"] <= 1
        assert srv.cancel(tickets[-1]) in (0, 1)   # queued -> cancelled, or already running
        rp, c, v, shape, p = mats[0]
        v2 = v.copy()
        v2[3] = 0
        tbad = srv.submit(rp, c, v2, shape, p)
        for t, mt in zip(tickets[:-1], mats[:-1]):
            code, res, ms = srv.wait(t, timeout=120.0)
            assert code == 0
            same(res, gbla.reduce(*mt))
        code, res, _ = srv.wait(tickets[-1], timeout=120.0)
        assert code in (0, gbla.GBLA_E_CANCELLED)
        code, res, _ = srv.wait(tbad, timeout=120.0)
        assert code == 1 and res is None


def test_batch_workers_persist_across_calls():
    """Batch workers are kept between calls: calls with growing, shrinking and
    default worker counts, and with fewer matrices than workers, all return
    the one-at-a-time results."""
    specs = mixed_specs(9, 11)
    mats = [synth.fl_matrix(s) + ((s.m, s.n), s.p) for s in specs]
    solo = [gbla.reduce(*mt) for mt in mats]
    for workers, count in ((2, 9), (12, 9), (1, 9), (0, 9), (16, 3), (5, 1)):
        res = gbla.reduce_batch(mats[:count], workers=workers)
        assert len(res) == count
        for r, ref in zip(res, solo):
            same(r, ref)
    assert gbla.reduce_batch([], workers=4) == []


def test_server_create_destroy_cycles():
    """Servers created and destroyed in turn (their worker threads release
    their streams and buffers on exit) keep serving exact results."""
    specs = mixed_specs(3, 12)
    mats = [synth.fl_matrix(s) + ((s.m, s.n), s.p) for s in specs]
    solo = [gbla.reduce(*mt) for mt in mats]
    for cycle in range(4):
        with gbla.Server(workers=1 + cycle) as srv:
            tickets = [srv.submit(*mt) for mt in mats]
            for t, ref in zip(tickets, solo):
                code, res, _ = srv.wait(t, timeout=120.0)
                assert code == 0
                same(res, ref)


BATCH_MIX_SEED = 20160223   # the benchmark's 256-matrix batch


def test_batch_mix_of_the_benchmark_members_equal_oracle():
    """The benchmark's 256-matrix batch (rows log-uniform in 500-20,000, p in
    {65521, 32003}) through both batch entry points: every member up to 5,000
    rows equals the oracle bit for bit, every larger one the solo reduction;
    device-resident and host results agree."""
    specs = synth.mixed_batch(256, BATCH_MIX_SEED)
    mats = [synth.fl_matrix(s) + ((s.m, s.n), s.p) for s in specs]
    host = gbla.reduce_batch(mats, workers=8)
    dev_in = [(torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(), torch.from_numpy(v.view(np.int16)).cuda(),
               shape, p) for rp, c, v, shape, p in mats]
    dev = gbla.reduce_batch_device(dev_in, workers=8)
    checked = 0
    for s, mt, h, d in zip(specs, mats, host, dev):
        rp, c, v, shape, p = mt
        rank, orp, oc, ov = d.to_host()
        d.free()
        same(h, (rank, orp, oc, ov))
        if s.m <= 5000:
            same(h, oracle.echelon(s.m, s.n, s.p, rp, c, v)[:4])
            checked += 1
        else:
            same(h, gbla.reduce(rp, c, v, shape, p))
    assert checked >= 100


def test_served_requests_overlap_and_equal_solo_and_oracle():
    """Requests submitted together run concurrently (the server admits
    several at once and their device intervals, from events on the workers'
    streams, intersect) and each result equals the solo reduction and the
    oracle."""
    specs = mixed_specs(24, 11) + synth.mixed_batch(8, 77, rows=(3000, 6000))
    mats = [synth.fl_matrix(s) + ((s.m, s.n), s.p) for s in specs]
    solo = [gbla.reduce(rp, c, v, shape, p) for rp, c, v, shape, p in mats]
    with gbla.Server(workers=8) as srv:
        tickets = [srv.submit(rp, c, v, shape, p) for rp, c, v, shape, p in mats]
        infos = []
        for t, ref in zip(tickets, solo):
            code, res, info = srv.wait_ex(t, timeout=120.0)
            assert code == 0
            same(res, ref)
            infos.append(info)
        st = srv.stats()
    for s, mt, ref in zip(specs, mats, solo):
        rp, c, v, shape, p = mt
        same(ref, oracle.echelon(s.m, s.n, s.p, rp, c, v)[:4])
    assert st["peak_running"] >= 2
    iv = sorted((i["device_start_ms"], i["device_end_ms"]) for i in infos)
    assert all(a >= 0 and b >= a for a, b in iv)
    overlapping = sum(1 for (a0, b0), (a1, b1) in zip(iv, iv[1:]) if a1 < b0)
    assert overlapping >= 1, iv
    busy = sum(b - a for a, b in iv)
    span = max(b for _, b in iv) - iv[0][0]
    assert busy > span, (busy, span)   # more device time in flight than wall time: overlap
    assert max(i["running_at_start"] for i in infos) >= 2
