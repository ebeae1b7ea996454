"""Batched solves of uneven instances as one CUDA graph, and the GEMM tile
autotuner.  Each instance in the batch must equal its standalone solve (the
same kernels in the same order; only the atomic sums of the mean removal and
of the gauge differ in rounding order, so the bar is 1e-12 of the max norm),
and the oracle: 1e-12 for float64 instances, the refined relative residual
for mixed ones."""
import numpy as np
import pytest
import torch

import oracle as O
import seeded_inputs as S
from _tpt import load

pytestmark = pytest.mark.gpu
tpt, L = load()

# Bars of the refined mixed path: its own float-pair residual stops the
# refinement at <= 1e-10 (relative 2-norm); the oracle's long-double residual
# of the returned phi differs from it by float-pair rounding of r (~1e-13 of
# |f| per point, measured below 2e-15 in the relative norm), hence 1e-10 plus
# 1e-14.  The element-wise distance to the oracle's float64 solution is at
# most ~1.2e-10 in these cases (measured), bounded here at 1e-9.
RES_BAR = 1e-10 + 1e-14
ERR_BAR = 1e-9

NNN = [(1, 1)] * 3
DND = [(2, 1), (1, 2), (2, 2)]
PNN = [(0, 0), (1, 1), (1, 1)]

# (n, stretch, bcs, alpha, beta, precision, max_refine)
CASES = [
    ((48, 40, 32), (1.5, 2.0, 2.5), NNN, 0.0, 1.0, L.TPT_PREC_MIXED_BF16X3, 6),
    ((40, 56, 24), (2.8, 1.1, 1.9), NNN, 1.0, -0.5 * 7e-3, L.TPT_PREC_MIXED_BF16X3, 6),
    ((32, 32, 32), (1.5, 2.0, 2.5), NNN, 0.0, 1.0, L.TPT_PREC_FP64, 1),
    ((24, 40, 48), (1.2, 2.2, 1.7), DND, 1.0, -0.5 * 3e-3, L.TPT_PREC_FP64, 1),
    ((70, 45, 33), (1.2, 2.0, 2.5), PNN, 0.0, 1.0, L.TPT_PREC_MIXED_TF32, 8),
    ((64, 48, 40), (3.0, 1.0, 2.0), DND, 1.0, -0.5 * 1e-2, L.TPT_PREC_MIXED_BF16X3, 6),
    ((16, 24, 8), (1.0, 1.0, 1.0), NNN, 0.0, 1.0, L.TPT_PREC_MIXED_BF16X3, 6),
]


def _spec(case):
    n, stretch, bcs, alpha, beta, prec, refine = case
    dirs = O.make_dirs(n, stretch, bcs)
    spec = dict(n=n, dxf=[d.dxf for d in dirs], dxc=[d.dxc for d in dirs], bc=bcs,
                xform=(tpt.GEMM, tpt.GEMM), alpha=alpha, beta=beta, precision=prec,
                rtol=1e-10 if prec != L.TPT_PREC_FP64 else 0.0, max_refine=refine)
    return spec, dirs


def _rhs(case, dirs, seed):
    n, alpha = case[0], case[3]
    f = S.uniform_rhs(n, seed)
    if O.is_singular(dirs, alpha):
        f = S.remove_weighted_mean(f, [d.dxf for d in dirs])
    return f


def _standalone(spec, f):
    # the same plan solved on its own: float64 runs its fixed 1 + max_refine
    # steps, mixed stops at rtol (in the batch the stopping test runs on the
    # device, so both stop after the same correction)
    plan = tpt.Plan(**spec)
    phi, info = plan.solve(tpt.field_to_device(f))
    return tpt.field_to_host(phi, spec["n"]), info


def _close(a, b, tol=1e-12):
    return np.abs(a - b).max() <= tol * np.abs(b).max()


@pytest.fixture(scope="module")
def batch():
    specs, dirs = zip(*[_spec(c) for c in CASES])
    b = tpt.Batch(list(specs), nstreams=3)
    yield b, list(specs), list(dirs)
    b.close()


def _run(b, specs, dirs, seed, fs_dev=None, phis=None, work=None):
    fs = [_rhs(c, d, seed + i) for i, (c, d) in enumerate(zip(CASES, dirs))]
    if fs_dev is None:
        fs_dev = [tpt.field_to_device(f) for f in fs]
    else:
        for t, f in zip(fs_dev, fs):
            t.copy_(tpt.field_to_device(f))
    phis = [torch.empty_like(t) for t in fs_dev] if phis is None else phis
    work = b.new_workspace() if work is None else work
    infos = b.solve(fs_dev, phis, work)
    return fs, fs_dev, phis, work, infos


def _check_instances(specs, dirs, fs, phis, infos):
    for i, (case, spec, d, f) in enumerate(zip(CASES, specs, dirs, fs)):
        got = tpt.field_to_host(phis[i], case[0])
        alone, ainfo = _standalone(spec, f)
        assert _close(got, alone), (i, np.abs(got - alone).max())
        alpha, beta, prec = case[3], case[4], case[5]
        if prec == L.TPT_PREC_FP64:
            assert infos[i]["iters"] == 1 + case[6]
        else:
            assert infos[i]["iters"] == ainfo["iters"] < 1 + case[6], (i, infos[i], ainfo)
        if prec == L.TPT_PREC_FP64:
            ref, _ = O.solve_tensor(f, d, alpha, beta)
            assert _close(got, ref), (i, np.abs(got - ref).max())
            assert infos[i]["status"] == L.TPT_OK
        else:
            r = O.residual(f, got, d, alpha, beta, np.longdouble)
            rel = float(np.sqrt(np.sum(r ** 2) / np.sum(f ** 2)))
            assert infos[i]["status"] == L.TPT_OK, infos[i]
            assert infos[i]["rel_residual"] <= 1e-10 and rel <= RES_BAR, (i, rel, infos[i])


def test_batch_instances_equal_standalone_and_oracle(batch):
    b, specs, dirs = batch
    fs, fs_dev, phis, work, infos = _run(b, specs, dirs, 100)      # eager run + capture
    _check_instances(specs, dirs, fs, phis, infos)
    assert b.launches_per_replay() > 0
    before = L.kernel_launches()
    fs, _, _, _, infos = _run(b, specs, dirs, 200, fs_dev, phis, work)   # graph replay, new data
    assert L.kernel_launches() - before == b.launches_per_replay()
    _check_instances(specs, dirs, fs, phis, infos)


def test_batch_recaptures_on_new_buffers_and_in_place(batch):
    b, specs, dirs = batch
    fs = [_rhs(c, d, 300 + i) for i, (c, d) in enumerate(zip(CASES, dirs))]
    fs_dev = [tpt.field_to_device(f) for f in fs]
    work = b.new_workspace()
    infos = b.solve(fs_dev, fs_dev, work)                          # phi = f, new pointers
    infos = b.solve([t.copy_(tpt.field_to_device(f)) for t, f in zip(fs_dev, fs)], fs_dev, work)
    _check_instances(specs, dirs, fs, fs_dev, infos)


def test_batch_autotune_keeps_results(batch):
    b, specs, dirs = batch
    fs, fs_dev, phis, work, infos0 = _run(b, specs, dirs, 400)
    ref = [p.clone() for p in phis]
    tiles = b.autotune(work)
    for i, t in enumerate(tiles):
        if CASES[i][5] == L.TPT_PREC_FP64:
            assert t == (0, 0, 0, 0)
        else:
            assert all(v in (32, 64, 128, 256) for v in t), t
    infos = b.solve(fs_dev, phis, work)
    for i in range(len(CASES)):
        a, r = phis[i].cpu().numpy(), ref[i].cpu().numpy()
        assert np.abs(a - r).max() <= 1e-12 * np.abs(r).max(), i
        assert infos[i]["status"] == L.TPT_OK


def test_plan_autotune_choices_and_solution():
    case = ((96, 80, 64), (1.5, 2.0, 2.5), NNN, 0.0, 1.0, L.TPT_PREC_MIXED_BF16X3, 6)
    spec, dirs = _spec(case)
    spec["rtol"] = 0.0
    f = _rhs(case, dirs, 7)
    plan = tpt.Plan(**spec)
    phi0, _ = plan.solve(tpt.field_to_device(f))
    tiles = plan.autotune()
    # the widths may not exceed the default one for the GEMM's column count:
    # x forward and y inverse have Nx / Ny columns, the other two Ny*Nz / ... many
    def top(n):
        return 32 if n <= 32 else 64 if n <= 64 else 128 if n <= 128 else 256
    assert tiles[0] <= top(96) and tiles[2] <= top(80), tiles
    assert all(t in (32, 64, 128, 256) for t in tiles)
    assert plan.tiles() == tiles
    phi1, _ = plan.solve(tpt.field_to_device(f))
    a, r = phi1.cpu().numpy(), phi0.cpu().numpy()
    assert np.abs(a - r).max() <= 1e-12 * np.abs(r).max()
    plan.set_tiles((32, 32, 32, 32))
    phi2, _ = plan.solve(tpt.field_to_device(f))
    assert np.abs(phi2.cpu().numpy() - r).max() <= 1e-12 * np.abs(r).max()


def test_calibrated_batch_stops_on_the_device_and_reports_misses():
    # calibrate leaves room for the corrections each instance used plus one;
    # in the captured batch the stopping test runs on the device, so the same
    # right-hand sides stop after the same corrections, and an instance
    # calibrated on a zero right-hand side (one correction, one spare) reports
    # NOT_CONVERGED for a right-hand side that needs more
    cases = [CASES[0], CASES[1]]
    specs, dirs = zip(*[_spec(c) for c in cases])
    b = tpt.Batch(list(specs), nstreams=2)
    try:
        fs = [_rhs(c, d, 500 + i) for i, (c, d) in enumerate(zip(cases, dirs))]
        fs_dev = [tpt.field_to_device(f) for f in fs]
        phis = [torch.empty_like(t) for t in fs_dev]
        work = b.new_workspace()
        used = b.calibrate(fs_dev, phis, work)
        infos = b.solve(fs_dev, phis, work)
        for i in range(2):
            assert infos[i]["status"] == L.TPT_OK and infos[i]["iters"] == used[i], (infos[i], used)
            r = O.residual(fs[i], tpt.field_to_host(phis[i], cases[i][0]), dirs[i], cases[i][3], cases[i][4],
                           np.longdouble)
            assert float(np.sqrt(np.sum(r ** 2) / np.sum(fs[i] ** 2))) <= RES_BAR
        zeros = [torch.zeros_like(t) for t in fs_dev]
        assert b.calibrate(zeros, phis, work) == [1, 1]
        infos = b.solve(fs_dev, phis, work, raise_errors=False)
        for i in range(2):
            assert infos[i]["status"] == L.TPT_ERR_NOT_CONVERGED and infos[i]["iters"] == 2, infos[i]
    finally:
        b.close()
