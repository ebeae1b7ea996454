"""Pressure projection (Sec. 2.1) on GB300 against the oracle's projection:
float64 plans to 1e-12 (relative max norm of the corrected velocities and of
Phi), refined mixed plans to 1e-9; the corrected field is discretely
divergence-free, a second projection leaves it unchanged and wall faces keep
their values."""
import numpy as np
import pytest
import torch

import oracle as O
from _tpt import load

pytestmark = pytest.mark.gpu
tpt, L = load()

NNN = [(1, 1)] * 3
PNN = [(0, 0), (1, 1), (1, 1)]


def _velocity(n, dirs, seed, wall_flux=False):
    rng = np.random.default_rng(seed)
    vel = []
    for ax, d in enumerate(dirs):
        shp = list(n)
        shp[ax] = d.n + 1
        u = np.moveaxis(rng.uniform(-1, 1, shp), ax, 0)
        if d.periodic:
            u[d.n] = u[0]
        elif not wall_flux:
            u[0] = 0.0
            u[d.n] = 0.0
        vel.append(np.moveaxis(u, 0, ax))
    return vel


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).ravel(order="F"))).cuda()


def _host(t, shape):
    return t.cpu().numpy().reshape(shape, order="F")


def _plan(n, dirs, bcs, prec):
    mixed = prec != L.TPT_PREC_FP64
    return tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs, xform=(tpt.GEMM, tpt.GEMM),
                    alpha=0.0, beta=1.0, precision=prec, rtol=1e-12 if mixed else 0.0,
                    max_refine=40 if mixed else 1)


CASES = [("NNN", NNN, (1.5, 2.0, 2.5)), ("PNN", PNN, (0.0, 2.2, 1.8))]


@pytest.mark.parametrize("prec", [L.TPT_PREC_FP64, L.TPT_PREC_MIXED_BF16X3])
@pytest.mark.parametrize("name,bcs,stretch", CASES)
def test_projection_matches_oracle(prec, name, bcs, stretch):
    n = (40, 28, 24)
    dirs = O.make_dirs(n, stretch, bcs)
    vel = _velocity(n, dirs, 3)
    gdt = 0.125
    ref_vel, ref_phi, _ = O.project(vel, dirs, gdt)
    plan = _plan(n, dirs, bcs, prec)
    uvw = [_dev(a) for a in vel]
    phi, info = plan.project(*uvw, gdt)
    tol = 1e-12 if prec == L.TPT_PREC_FP64 else 1e-9
    got_phi = _host(phi, n)
    assert np.abs(got_phi - ref_phi).max() <= tol * np.abs(ref_phi).max()
    got = [_host(t, a.shape) for t, a in zip(uvw, vel)]
    for a in range(3):
        assert np.abs(got[a] - ref_vel[a]).max() <= tol * np.abs(vel[a]).max(), (a,)
    div0 = np.abs(O.divergence(vel, dirs)).max()
    assert np.abs(O.divergence(got, dirs)).max() <= 10 * tol * div0
    for ax, d in enumerate(dirs):        # wall faces unchanged
        if not d.periodic:
            g = np.moveaxis(got[ax], ax, 0)
            v0 = np.moveaxis(vel[ax], ax, 0)
            assert np.array_equal(g[0], v0[0]) and np.array_equal(g[d.n], v0[d.n])


def test_projection_is_idempotent_and_reports_wall_flux():
    n = (32, 24, 20)
    dirs = O.make_dirs(n, (1.5, 2.0, 2.5), NNN)
    plan = _plan(n, dirs, NNN, L.TPT_PREC_FP64)
    vel = _velocity(n, dirs, 5)
    uvw = [_dev(a) for a in vel]
    plan.project(*uvw, 0.5)
    once = [t.clone() for t in uvw]
    plan.project(*uvw, 0.5)
    for a, b in zip(uvw, once):
        assert (a - b).abs().max().item() <= 1e-12 * b.abs().max().item()
    # a net flux through the walls is incompatible: it is removed and reported
    velw = _velocity(n, dirs, 6, wall_flux=True)
    _, phi_ref, defect = O.project(velw, dirs, 0.5)
    _, info = plan.project(*[_dev(a) for a in velw], 0.5)
    # the defect is a volume-weighted mean with cancellation: round-off is
    # relative to the size of the right-hand side, not of the mean
    scale = np.abs(O.divergence(velw, dirs)).max() / 0.5
    assert abs(info["compat_defect"] - defect) <= 1e-13 * scale
    assert abs(defect) > 1e-3


def test_projection_argument_checks():
    n = (16, 12, 10)
    dirs = O.make_dirs(n, (1.0, 1.0, 1.0), NNN)
    helm = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], NNN, xform=(tpt.GEMM, tpt.GEMM),
                    alpha=1.0, beta=-1e-3)
    vel = [_dev(a) for a in _velocity(n, dirs, 1)]
    with pytest.raises(L.TptError) as e:
        helm.project(*vel, 0.1)
    assert e.value.status == L.TPT_ERR_INVALID_ARG
    dbc = [(2, 2), (1, 1), (1, 1)]
    dird = O.make_dirs(n, (1.0, 1.0, 1.0), dbc)
    dp = tpt.Plan(n, [d.dxf for d in dird], [d.dxc for d in dird], dbc, xform=(tpt.GEMM, tpt.GEMM))
    with pytest.raises(L.TptError) as e:
        dp.project(*vel, 0.1)
    assert e.value.status == L.TPT_ERR_UNSUPPORTED
