"""Failure detection on GB300, with no GPU fault: a bounded device-side wait
that runs out (a GEMM whose producer issues no loads) returns
TPT_ERR_TIMEOUT and leaves the context usable; a non-finite right-hand side
is reported as TPT_ERR_NONFINITE; device allocations that fail (injected on
the host) make plan creation and served requests return TPT_ERR_OOM cleanly,
and everything works again once the injection is off."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
import seeded_inputs as S
from _tpt import load

pytestmark = pytest.mark.gpu
tpt, L = load()

NNN = [(1, 1)] * 3


def _spec(n, prec, alpha=0.0, beta=1.0):
    dirs = O.make_dirs(n, (1.5, 2.0, 2.5), NNN)
    mixed = prec != L.TPT_PREC_FP64
    return dirs, dict(n=n, dxf=[d.dxf for d in dirs], dxc=[d.dxc for d in dirs], bc=NNN,
                      xform=(tpt.GEMM, tpt.GEMM), alpha=alpha, beta=beta, precision=prec,
                      rtol=1e-10 if mixed else 0.0, max_refine=30 if mixed else 1)


def _plan(spec):
    return tpt.Plan(spec["n"], spec["dxf"], spec["dxc"], spec["bc"], xform=spec["xform"], alpha=spec["alpha"],
                    beta=spec["beta"], precision=spec["precision"], rtol=spec["rtol"],
                    max_refine=spec["max_refine"])


def _solves_correctly(prec=L.TPT_PREC_MIXED_BF16X3):
    n = (48, 40, 36)
    dirs, spec = _spec(n, prec)
    f = S.remove_weighted_mean(S.uniform_rhs(n, 3), [d.dxf for d in dirs])
    phi, info = _plan(spec).solve(tpt.field_to_device(f))
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    err = np.abs(tpt.field_to_host(phi, n) - ref).max() / np.abs(ref).max()
    return info["status"] == L.TPT_OK and err <= 1e-9


def test_a_wait_that_runs_out_returns_timeout_and_the_next_solve_succeeds():
    work = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for polls in (1 << 10, 1 << 12):
        st = L.lib.tpt_test_gemm_timeout(polls, C.c_void_p(work.data_ptr()), work.numel(),
                                         C.c_void_p(stream.cuda_stream))
        assert st == L.TPT_ERR_TIMEOUT, L.lib.tpt_status_string(st)
    torch.cuda.synchronize()                 # no sticky error: the context is intact
    assert _solves_correctly()
    assert L.lib.tpt_test_gemm_timeout(0, C.c_void_p(work.data_ptr()), work.numel(), None) == L.TPT_ERR_INVALID_ARG


@pytest.mark.parametrize("prec,rtol", [(L.TPT_PREC_FP64, 1e-12), (L.TPT_PREC_MIXED_BF16X3, 1e-10)])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_a_non_finite_right_hand_side_is_reported(prec, rtol, bad):
    n = (40, 32, 24)
    dirs, spec = _spec(n, prec, alpha=1.0, beta=-5e-4)
    spec.update(rtol=rtol, max_refine=30)
    f = S.uniform_rhs(n, 5)
    f[7, 3, 11] = bad
    plan = _plan(spec)
    phi, work = plan.new_field(), plan.new_workspace()
    info = L.tpt_info()
    st = L.lib.tpt_solve(plan._h, C.c_void_p(tpt.field_to_device(f).data_ptr()), C.c_void_p(phi.data_ptr()),
                         C.c_void_p(work.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream),
                         C.byref(info))
    torch.cuda.synchronize()
    assert st == L.TPT_ERR_NONFINITE, L.lib.tpt_status_string(st)
    f[7, 3, 11] = 0.0                        # the same plan and buffers work on a finite one
    st = L.lib.tpt_solve(plan._h, C.c_void_p(tpt.field_to_device(f).data_ptr()), C.c_void_p(phi.data_ptr()),
                         C.c_void_p(work.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream),
                         C.byref(info))
    torch.cuda.synchronize()
    assert st == L.TPT_OK, L.lib.tpt_status_string(st)


def test_a_non_finite_right_hand_side_in_an_asynchronous_float64_solve_shows_in_its_info():
    n = (40, 32, 24)
    _, spec = _spec(n, L.TPT_PREC_FP64)          # rtol 0: no host synchronisation in the call
    f = S.uniform_rhs(n, 5)
    f[1, 2, 3] = float("nan")
    plan = _plan(spec)
    _, info = plan.solve(tpt.field_to_device(f))  # reads info after synchronising the stream
    assert info["status"] == L.TPT_OK and not np.isfinite(info["rel_residual"])


@pytest.mark.parametrize("prec", [L.TPT_PREC_FP64, L.TPT_PREC_MIXED_BF16X3])
@pytest.mark.parametrize("after", [0, 3])
def test_failed_device_allocations_make_plan_creation_return_oom(prec, after):
    _, spec = _spec((32, 24, 16), prec)
    desc, keep = tpt.make_desc(spec["n"], spec["dxf"], spec["dxc"], spec["bc"], spec["xform"], spec["alpha"],
                               spec["beta"], spec["precision"], spec["rtol"], spec["max_refine"])
    h = C.c_void_p()
    try:
        assert L.lib.tpt_test_fail_allocations(after) == L.TPT_OK
        st = L.lib.tpt_plan_create(C.byref(desc), 0, C.byref(h))
    finally:
        L.lib.tpt_test_fail_allocations(-1)
    assert st == L.TPT_ERR_OOM, L.lib.tpt_status_string(st)
    assert not h.value
    assert _solves_correctly(prec)


def test_failed_allocations_fail_served_requests_with_oom_and_the_server_recovers():
    n = (32, 32, 24)
    dirs, spec = _spec(n, L.TPT_PREC_MIXED_BF16X3)
    f = S.remove_weighted_mean(S.uniform_rhs(n, 9), [d.dxf for d in dirs])
    f_pin = torch.from_numpy(np.ascontiguousarray(f.ravel(order="F"))).pin_memory()
    out = [torch.empty_like(f_pin).pin_memory() for _ in range(2)]
    srv = tpt.Server(device=0, slots=2, setup_threads=1, memory_budget=1 << 30, cache_budget=1 << 28)
    try:
        L.lib.tpt_test_fail_allocations(0)
        try:
            r_bad = srv.wait(srv.submit(f_pin, out[0], **spec), timeout=120.0)
        finally:
            L.lib.tpt_test_fail_allocations(-1)
        r_ok = srv.wait(srv.submit(f_pin, out[1], **spec), timeout=120.0)
    finally:
        srv.close()
    assert r_bad["status"] == L.TPT_ERR_OOM, r_bad
    assert r_bad["failed_step"] in (1, 2) and r_bad["cuda_error_name"] == "cudaErrorMemoryAllocation", r_bad
    assert r_ok["status"] == L.TPT_OK and r_ok["failed_step"] == 0, r_ok
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    got = out[1].numpy().reshape(n, order="F")
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
