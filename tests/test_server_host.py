"""Serving runtime and eigenbasis cache on the host (no GPU): the server's
dry-run executor simulates each solve as a sleep, which exercises queueing,
plan building through the cache, memory-budget admission and slot
concurrency; host-only cached plans must equal plans built on their own."""
import ctypes as C
import threading

import numpy as np
import pytest

import oracle as O
from _tpt import load

tpt, L = load()


def _spec(n, stretch, alpha=0.0, beta=1.0, prec=L.TPT_PREC_FP64):
    grids = [O.tanh_grid(n[a], 1.0, stretch[a]) for a in range(3)]
    return dict(n=n, dxf=[g[0] for g in grids], dxc=[g[1] for g in grids], bc=[(1, 1)] * 3,
                xform=(tpt.GEMM, tpt.GEMM), alpha=alpha, beta=beta, precision=prec, rtol=0.0, max_refine=1)


def _need(n):
    # FP64 plan: f + phi + workspace (256 + 4 regions) + alignment slack
    pts = n[0] * n[1] * n[2]
    region = (pts * 8 + 255) // 256 * 256
    return 2 * pts * 8 + 256 + 4 * region + 3 * 256


def _requests(count, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = tuple(int(v) for v in rng.choice([8, 12, 16, 20], size=3))
        stretch = tuple(float(v) for v in rng.choice([1.0, 2.0], size=3))
        out.append((n, stretch))
    return out


def _run(srv, reqs):
    bufs = []
    tickets = []
    for n, stretch in reqs:
        pts = n[0] * n[1] * n[2]
        f = np.zeros(pts)
        phi = np.zeros(pts)
        bufs.append((f, phi))
        tickets.append(srv.submit(f, phi, **_spec(n, stretch)))
    return [srv.wait(t, timeout=60.0) for t in tickets]


def test_dry_run_completes_and_respects_slots_and_budget():
    reqs = _requests(40)
    budget = 3 * max(_need(n) for n, _ in reqs)
    srv = tpt.Server(device=-1, slots=3, setup_threads=2, memory_budget=budget, cache_budget=0,
                     dry_run_ns_per_point=200.0)
    res = _run(srv, reqs)
    st = srv.stats()
    srv.close()
    assert all(r is not None and r["status"] == L.TPT_OK for r in res)
    for r in res:
        assert r["t_submit"] <= r["t_planned"] <= r["t_admit"] <= r["t_done"]
    assert st["submitted"] == st["completed"] == len(reqs) and st["rejected"] == 0
    assert 1 <= st["peak_inflight"] <= 3
    assert st["peak_bytes"] <= budget
    # every x and y direction draws from 4 sizes x 2 stretches: most lookups hit
    assert st["cache_hits"] + st["cache_misses"] == 2 * len(reqs)
    assert st["cache_misses"] <= 8 and st["cache_hits"] >= 2 * len(reqs) - 8


def test_dry_run_admits_in_arrival_order_with_one_setup_thread():
    reqs = _requests(25, seed=4)
    srv = tpt.Server(device=-1, slots=2, setup_threads=1, memory_budget=1 << 40, cache_budget=0,
                     dry_run_ns_per_point=100.0)
    res = _run(srv, reqs)
    srv.close()
    admits = [r["t_admit"] for r in res]
    assert admits == sorted(admits)


def test_memory_budget_serialises_large_requests_and_rejects_oversized():
    n = (20, 20, 20)
    need = _need(n)
    srv = tpt.Server(device=-1, slots=4, setup_threads=2, memory_budget=int(1.5 * need), cache_budget=0,
                     dry_run_ns_per_point=500.0)
    res = _run(srv, [(n, (1.0, 1.0, 1.0))] * 6)
    big = _run(srv, [((40, 40, 40), (1.0, 1.0, 1.0))])[0]      # can never fit the budget
    after = _run(srv, [((8, 8, 8), (1.0, 1.0, 1.0))])[0]        # the server keeps serving
    st = srv.stats()
    srv.close()
    assert all(r["status"] == L.TPT_OK for r in res)
    assert st["peak_inflight"] == 1                             # one at a time fits 1.5 x need
    assert big["status"] == L.TPT_ERR_OOM and after["status"] == L.TPT_OK
    assert st["rejected"] == 1
    # the admitted requests ran one after another
    spans = sorted((r["t_admit"], r["t_done"]) for r in res)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0 - 1e-6


def test_concurrent_submitters_and_wait_timeout():
    srv = tpt.Server(device=-1, slots=2, setup_threads=2, memory_budget=1 << 40, cache_budget=0,
                     dry_run_ns_per_point=50.0)
    results = {}

    def worker(k):
        results[k] = _run(srv, _requests(10, seed=10 + k))

    ths = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert sum(len(v) for v in results.values()) == 40
    assert all(r["status"] == L.TPT_OK for v in results.values() for r in v)
    # a long request reports pending before it finishes
    n = (64, 64, 64)
    f, phi = np.zeros(n[0] ** 3), np.zeros(n[0] ** 3)
    srv2 = tpt.Server(device=-1, slots=1, setup_threads=1, memory_budget=1 << 40, cache_budget=0,
                      dry_run_ns_per_point=2000.0)                 # about 0.5 s
    t = srv2.submit(f, phi, **_spec(n, (1.0, 1.0, 1.0)))
    assert srv2.wait(t, timeout=0.01) is None
    assert srv2.wait(t)["status"] == L.TPT_OK
    with pytest.raises(L.TptError):
        srv2.wait(t)                                                 # forgotten after retrieval
    srv.close()
    srv2.close()


def test_server_argument_checks():
    cfg = L.tpt_server_config(-1, 0, 1, 1 << 20, 0, 0.0)
    h = C.c_void_p()
    assert L.lib.tpt_server_create(C.byref(cfg), C.byref(h)) == L.TPT_ERR_INVALID_ARG
    cfg = L.tpt_server_config(-1, 1, 1, 0, 0, 0.0)
    assert L.lib.tpt_server_create(C.byref(cfg), C.byref(h)) == L.TPT_ERR_INVALID_ARG
    cfg = L.tpt_server_config(-1, 1, 1, 1 << 20, 0, -1.0)
    assert L.lib.tpt_server_create(C.byref(cfg), C.byref(h)) == L.TPT_ERR_INVALID_ARG
    assert L.lib.tpt_server_destroy(None) == L.TPT_ERR_INVALID_ARG


def test_host_cached_plans_equal_standalone_plans():
    cache = tpt.Cache(device=-1, budget_bytes=0)
    for n, stretch in [((12, 16, 10), (2.0, 1.5, 1.0)), ((16, 12, 10), (1.5, 2.0, 1.0)),
                       ((12, 16, 10), (2.0, 1.5, 2.5))]:
        sp = _spec(n, stretch)
        desc, keep = tpt.make_desc(**sp)
        hc, hs = C.c_void_p(), C.c_void_p()
        assert L.lib.tpt_plan_create_cached(C.byref(desc), cache._h, C.byref(hc)) == L.TPT_OK
        assert L.lib.tpt_plan_create(C.byref(desc), -1, C.byref(hs)) == L.TPT_OK
        for d in range(2):
            a, b = np.empty(n[d]), np.empty(n[d])
            assert L.lib.tpt_plan_eigenvalues(hc, d, a.ctypes.data_as(L._dp)) == L.TPT_OK
            assert L.lib.tpt_plan_eigenvalues(hs, d, b.ctypes.data_as(L._dp)) == L.TPT_OK
            assert np.array_equal(a, b)
        L.lib.tpt_plan_destroy(hc)
        L.lib.tpt_plan_destroy(hs)
    st = cache.stats()
    # x of the second plan is y of the first and vice versa: 4 hits out of 6 lookups
    assert st["hits"] == 4 and st["misses"] == 2 and st["device_bytes"] == 0
    cache.close()


def test_warm_fills_the_cache_before_traffic():
    srv = tpt.Server(device=-1, slots=2, setup_threads=1, memory_budget=1 << 40, cache_budget=0,
                     dry_run_ns_per_point=10.0)
    srv.warm(**_spec((12, 16, 10), (2.0, 1.5, 1.0)))
    st0 = srv.stats()
    assert st0["cache_misses"] == 2 and st0["completed"] == 0
    res = _run(srv, [((12, 16, 10), (2.0, 1.5, 1.0)), ((16, 12, 8), (1.5, 2.0, 1.0))])
    st = srv.stats()
    srv.close()
    assert all(r["status"] == L.TPT_OK for r in res)
    assert st["cache_misses"] == 2 and st["cache_hits"] == 4


def test_a_failed_request_reports_its_step_and_cuda_error():
    """A request that fails names the step it failed in; one that fails in
    host setup (an FFT transform asked for a stretched direction) carries no
    CUDA error.  Requests that succeed report neither."""
    srv = tpt.Server(device=-1, slots=2, setup_threads=1, memory_budget=1 << 30, cache_budget=0,
                     dry_run_ns_per_point=10.0)
    f, phi = np.zeros(8 * 8 * 8), np.zeros(8 * 8 * 8)
    bad = dict(_spec((8, 8, 8), (2.0, 2.0, 2.0)), xform=(tpt.FFT, tpt.GEMM))
    t_bad = srv.submit(f, phi, **bad)
    t_ok = srv.submit(f, phi, **_spec((8, 8, 8), (2.0, 2.0, 2.0)))
    r_bad, r_ok = srv.wait(t_bad, timeout=60.0), srv.wait(t_ok, timeout=60.0)
    srv.close()
    assert r_bad["status"] == L.TPT_ERR_UNSUPPORTED
    assert r_bad["failed_step"] == 1 and r_bad["cuda_error"] == 0   # TPT_STEP_PLAN
    assert r_ok["status"] == L.TPT_OK and r_ok["failed_step"] == 0 and r_ok["cuda_error"] == 0
    assert L.lib.tpt_cuda_error_name(0) == b"cudaSuccess"


def test_dry_run_merges_ready_requests_of_one_shape():
    """Same-shape batching on the host: with one slot busy, requests of one
    grid size that queue up are admitted together (at most `merge`, within
    the budget), others one at a time; every request completes and reports
    how many were solved with it."""
    mixed = dict(precision=L.TPT_PREC_MIXED_BF16X3, rtol=1e-10, max_refine=8)
    shapes = [(16, 12, 8)] * 9 + [(12, 16, 8)] * 2 + [(18, 12, 8)] * 2   # Nx = 18: not grouped
    srv = tpt.Server(device=-1, slots=1, setup_threads=1, memory_budget=1 << 40, cache_budget=0,
                     dry_run_ns_per_point=4000.0, merge=4)
    bufs, tickets = [], []
    for i, n in enumerate(shapes):
        f, phi = np.zeros(n[0] * n[1] * n[2]), np.zeros(n[0] * n[1] * n[2])
        bufs.append((f, phi))
        tickets.append(srv.submit(f, phi, **dict(_spec(n, (1.5, 2.0, 1.0)), **mixed)))
    res = [srv.wait(t, timeout=60.0) for t in tickets]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == L.TPT_OK for r in res)
    merged = [r["merged"] for r in res]
    assert max(merged) >= 3 and max(merged) <= 4, merged
    assert all(m == 1 or m >= 3 for m in merged), merged     # no pairs
    assert all(m == 1 for m, n in zip(merged, shapes) if n[0] == 18)
    # requests solved together were admitted and finished at the same moment
    for r in res:
        if r["merged"] > 1:
            same = [q for q in res if q["t_admit"] == r["t_admit"]]
            assert len(same) == r["merged"] and all(abs(q["t_done"] - r["t_done"]) < 1e-3 for q in same)
    assert st["completed"] == len(shapes)
