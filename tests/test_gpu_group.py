"""Grouped batch solves on GB300: every stage one kernel over all instances
(GEMM tiles, Thomas line tiles and residual plane tiles of every instance in
one launch, per-instance stops on the device).  Each instance must match the
same plan solved on its own with the same Thomas kernel (the arithmetic is
the same; only the order of float64 atomic sums differs: 1e-11 for refined
mixed solves, as for served requests), and the oracle (residual within the
refinement target, element error 1e-9); the batch replays O(10) kernels per
correction; the stream mode gives the same solutions; a batch the grouped
kernels cannot take reports UNSUPPORTED for the grouped mode."""
import numpy as np
import pytest
import torch

import oracle as O
import seeded_inputs as S
from _tpt import load

pytestmark = pytest.mark.gpu
tpt, L = load()

RES_BAR = 1e-10 + 1e-14
ERR_BAR = 1e-9
NNN = [(1, 1)] * 3
DND = [(2, 1), (1, 2), (2, 2)]

# (n, stretch, bcs, alpha, beta): Nz from 24 to 320 covers the segment
# lengths 4, 8 and 12 of the two-line Thomas kernel; Poisson (singular),
# Helmholtz and Dirichlet walls give three residual variants
CASES = [
    ((64, 48, 40), (1.5, 2.0, 2.5), NNN, 0.0, 1.0),
    ((96, 64, 160), (2.8, 1.1, 1.9), NNN, 1.0, -0.5 * 7e-3),
    ((32, 32, 32), (1.0, 1.0, 1.0), NNN, 0.0, 1.0),
    ((128, 96, 96), (3.0, 1.0, 2.0), DND, 1.0, -0.5 * 1e-2),
    ((48, 40, 320), (1.2, 2.2, 1.7), NNN, 0.0, 1.0),
    ((16, 24, 24), (2.0, 2.0, 2.0), NNN, 1.0, -0.5 * 4e-3),
    ((64, 64, 64), (1.5, 1.5, 1.5), DND, 0.0, 1.0),
]


def _spec(case):
    n, stretch, bcs, alpha, beta = case
    dirs = O.make_dirs(n, stretch, bcs)
    spec = dict(n=n, dxf=[d.dxf for d in dirs], dxc=[d.dxc for d in dirs], bc=bcs, xform=(tpt.GEMM, tpt.GEMM),
                alpha=alpha, beta=beta, precision=L.TPT_PREC_MIXED_BF16X3, rtol=1e-10, max_refine=12)
    return spec, dirs


def _rhs(case, dirs, seed):
    f = S.uniform_rhs(case[0], seed)
    if O.is_singular(dirs, case[3]):
        f = S.remove_weighted_mean(f, [d.dxf for d in dirs])
    return f


@pytest.fixture(scope="module")
def group():
    specs, dirs = zip(*[_spec(c) for c in CASES])
    b = tpt.Batch(list(specs))
    assert b.grouped
    fs = [_rhs(c, d, 70 + i) for i, (c, d) in enumerate(zip(CASES, dirs))]
    fs_dev = [tpt.field_to_device(f) for f in fs]
    yield b, list(specs), list(dirs), fs, fs_dev
    b.close()


def test_grouped_instances_match_standalone_and_the_oracle(group):
    b, specs, dirs, fs, fs_dev = group
    phis = [torch.full_like(t, float("nan")) for t in fs_dev]
    work = b.new_workspace()
    outs = []
    for call in range(3):                       # eager with capture, then replays
        infos = b.solve(fs_dev, phis, work)
        outs.append([tpt.field_to_host(p, s["n"]) for p, s in zip(phis, specs)])
        for i, inf in enumerate(infos):
            assert inf["status"] == L.TPT_OK and inf["rel_residual"] <= 1e-10, (call, i, inf)
    for o in outs[1:]:
        for a, c in zip(o, outs[0]):
            assert np.abs(a - c).max() <= 1e-11 * np.abs(c).max()
    for i, (spec, d, f) in enumerate(zip(specs, dirs, fs)):
        got = outs[-1][i]
        plan = tpt.Plan(**spec)
        plan.set_thomas_kernel(2)
        alone, _ = plan.solve(tpt.field_to_device(f))
        alone = tpt.field_to_host(alone, spec["n"])
        assert np.abs(got - alone).max() <= 1e-11 * np.abs(alone).max(), i
        r = O.residual(f, got, d, spec["alpha"], spec["beta"], np.longdouble)
        rel = float(np.sqrt(np.sum(r ** 2) / np.sum(f ** 2)))
        ref, _ = O.solve_tensor(f, d, spec["alpha"], spec["beta"])
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert rel <= RES_BAR and err <= ERR_BAR, (i, rel, err)


def test_grouped_batch_replays_few_kernels_per_correction(group):
    b, specs, dirs, fs, fs_dev = group
    phis = [torch.empty_like(t) for t in fs_dev]
    work = b.new_workspace()
    b.solve(fs_dev, phis, work)
    corrections = 1 + max(s["max_refine"] for s in specs)
    launches = b.launches_per_replay()
    # per correction: four GEMMs, a Thomas sweep per segment length (3), the
    # null lines, a residual per variant (3), the stopping test; plus 8 once
    assert launches <= corrections * 13 + 8, launches


def test_stream_mode_gives_the_same_solutions(group):
    b, specs, dirs, fs, fs_dev = group
    phis_g = [torch.empty_like(t) for t in fs_dev]
    b.solve(fs_dev, phis_g, b.new_workspace())
    b.set_grouped(False)
    try:
        for p in b.plans:
            p.set_thomas_kernel(2)
        phis_s = [torch.empty_like(t) for t in fs_dev]
        infos = b.solve(fs_dev, phis_s, b.new_workspace())
        assert all(i["status"] == L.TPT_OK for i in infos)
        for a, c in zip(phis_g, phis_s):
            assert (a - c).abs().max().item() <= 1e-11 * c.abs().max().item()
    finally:
        for p in b.plans:
            p.set_thomas_kernel(0)
        b.set_grouped(True)
    assert b.grouped


def test_a_batch_outside_the_grouped_kernels_stays_on_streams():
    specs = [_spec(CASES[0])[0], dict(_spec(CASES[2])[0], precision=L.TPT_PREC_MIXED_TF32)]
    b = tpt.Batch(specs)
    try:
        assert not b.grouped
        with pytest.raises(L.TptError) as e:
            b.set_grouped(True)
        assert e.value.status == L.TPT_ERR_UNSUPPORTED
    finally:
        b.close()
    odd = [dict(_spec(CASES[0])[0], n=(66, 48, 40), dxf=None)]
    d = O.make_dirs((66, 48, 40), (1.5, 2.0, 2.5), NNN)
    odd[0].update(dxf=[x.dxf for x in d], dxc=[x.dxc for x in d])
    b = tpt.Batch(odd)
    try:
        assert not b.grouped                   # Nx not a multiple of 4
    finally:
        b.close()
