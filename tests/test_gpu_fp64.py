"""float64 CUDA path against the CPU oracle, element by element.

Every test calls libtpt.so through the C ABI (via the ctypes binding) on cuda:0
and compares with ``oracle`` on the same seeded inputs.  Bar: relative
max-norm 1e-12 for solves (the float64 target), tighter for single steps.
"""
import numpy as np
import pytest
import torch

import oracle as O
import seeded_inputs as S
from _tpt import load

pytestmark = pytest.mark.gpu
tpt, L = load()

N_, P_, D_ = O.NEUMANN, O.PERIODIC, O.DIRICHLET
TOL = 1e-12


def _plan(dirs, alpha, beta, **kw):
    kw.setdefault("xform", (tpt.GEMM, tpt.GEMM))
    return tpt.Plan(tuple(d.n for d in dirs), [d.dxf for d in dirs], [d.dxc for d in dirs],
                    [d.bc for d in dirs], alpha=alpha, beta=beta, **kw)


def _rhs(dirs, seed, singular):
    n = tuple(d.n for d in dirs)
    f = S.uniform_rhs(n, seed)
    return S.remove_weighted_mean(f, [d.dxf for d in dirs]) if singular else f


def _relerr(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def _solve_and_compare(n, stretch, bcs, alpha, beta, seed, tol=TOL, refine=1, f=None):
    dirs = O.make_dirs(n, stretch, bcs)
    sing = O.is_singular(dirs, alpha)
    if f is None:
        f = _rhs(dirs, seed, sing)
    plan = _plan(dirs, alpha, beta, max_refine=refine)
    phi, info = plan.solve(tpt.field_to_device(f))
    got = tpt.field_to_host(phi, n)
    ref, defect = O.solve_tensor(f, dirs, alpha, beta, refine=1)
    err = _relerr(got, ref)
    assert err <= tol, (n, bcs, alpha, beta, err)
    assert abs(info["compat_defect"] - defect) <= 1e-12 * max(1.0, np.abs(f).max())
    return err, info


BCS = {
    "NNN": [(N_, N_)] * 3,
    "PNN": [(P_, P_), (N_, N_), (N_, N_)],
    "DND": [(D_, N_), (N_, D_), (D_, D_)],
    "PPD": [(P_, P_), (P_, P_), (N_, D_)],
}


@pytest.mark.parametrize("bcs", list(BCS))
@pytest.mark.parametrize("coef", [(0.0, 1.0), (1.0, -5e-4), (1.0, -0.25)])
def test_solve_parity_ragged_tiles(bcs, coef):
    # 70 and 45 span two 64-wide GEMM tiles with ragged tails; Nz = 33 is odd
    stretch = (1.5, 2.0, 2.5) if not bcs.startswith("P") else (0.0, 2.0, 2.5)
    _solve_and_compare((70, 45, 33), stretch, BCS[bcs], *coef, seed=11)


@pytest.mark.parametrize("n", [(1, 1, 50), (1, 23, 17), (19, 1, 17), (21, 18, 1), (2, 3, 2), (1, 1, 1)])
def test_degenerate_sizes(n):
    for coef in [(0.0, 1.0), (1.0, -0.01)]:
        _solve_and_compare(n, (1.2, 1.7, 2.2), BCS["NNN"], *coef, seed=5)


def test_config1_32cube_white_noise_and_manufactured():
    n = (32, 32, 32)
    bcs = BCS["PNN"]
    _solve_and_compare(n, (0.0, 1.5, 1.5), bcs, 0.0, 1.0, seed=1)
    dirs = O.make_dirs(n, (0.0, 1.5, 1.5), bcs)
    cen = []
    for d in dirs:
        faces = np.concatenate([[0.0], np.cumsum(d.dxf)])
        cen.append(0.5 * (faces[1:] + faces[:-1]))
    u = np.einsum("i,j,k->ijk", np.cos(2 * np.pi * cen[0]), np.cos(np.pi * cen[1]), np.cos(np.pi * cen[2]))
    f = O.apply_operator(u, dirs, 0.0, 1.0)
    plan = _plan(dirs, 0.0, 1.0)
    phi, _ = plan.solve(tpt.field_to_device(f))
    assert _relerr(tpt.field_to_host(phi, n), u) <= TOL


@pytest.mark.parametrize("coef,seed", [((0.0, 1.0), 2), ((1.0, -5e-4), 3)])
def test_config2_256cube(coef, seed):
    _solve_and_compare((256, 256, 256), (2.0, 2.0, 2.0), BCS["NNN"], *coef, seed=seed)


def test_incompatible_rhs_reports_defect_and_keeps_gauge():
    n = (24, 20, 16)
    dirs = O.make_dirs(n, (1.5, 2.0, 2.5), BCS["NNN"])
    f = S.uniform_rhs(n, 9) + 0.3          # not mean-free: defect ~ 0.3
    err, info = _solve_and_compare(n, (1.5, 2.0, 2.5), BCS["NNN"], 0.0, 1.0, 9, f=f)
    assert abs(info["compat_defect"] - O.weighted_mean(f, dirs)) < 1e-13


def test_adaptive_refinement_and_in_place():
    n = (48, 40, 36)
    dirs = O.make_dirs(n, (2.0, 2.5, 3.0), BCS["NNN"])
    f = _rhs(dirs, 4, True)
    plan = _plan(dirs, 0.0, 1.0, rtol=1e-13, max_refine=4)
    buf = tpt.field_to_device(f)
    phi, info = plan.solve(buf, phi=buf)        # in place: phi overwrites f
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    assert _relerr(tpt.field_to_host(phi, n), ref) <= TOL
    assert info["rel_residual"] <= 1e-13 and 1 <= info["iters"] <= 5
    resid = O.residual(f, tpt.field_to_host(phi, n), dirs, 0.0, 1.0, np.longdouble)
    assert float(np.sqrt(np.sum(resid ** 2)) / np.sqrt(np.sum(f ** 2))) <= 1e-13


def test_solve_host_end_to_end():
    n = (40, 36, 30)
    dirs = O.make_dirs(n, (1.5, 2.0, 2.5), BCS["NNN"])
    f = _rhs(dirs, 7, True)
    plan = _plan(dirs, 0.0, 1.0)
    fh = torch.from_numpy(np.ascontiguousarray(f.ravel(order="F"))).pin_memory()
    ph = torch.empty_like(fh).pin_memory()
    fd, pd = plan.new_field(), plan.new_field()
    plan.solve_host(fh, ph, fd, pd, plan.new_workspace())
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    assert _relerr(ph.numpy().reshape(n, order="F"), ref) <= TOL


# ---------------------------------------------------------------- single steps

def test_transform_diagonalises_the_operator():
    # forward transform along x of (T_x f) equals lambda_p times the forward
    # transform of f (Q^{-1} T = Lambda Q^{-1}), in the plan's own mode order
    n = (70, 45, 9)
    dirs = O.make_dirs(n, (2.5, 1.5, 1.0), [(N_, N_), (D_, N_), (N_, N_)])
    plan = _plan(dirs, 0.0, 1.0)
    f = S.uniform_rhs(n, 3)
    for ax in (0, 1):
        d = dirs[ax]
        shape = [1, 1, 1]
        shape[ax] = n[ax]
        a, b, c = (v.reshape(shape) for v in (d.a, d.b, d.c))
        Tf = b * f + a * np.roll(f, 1, axis=ax) + c * np.roll(f, -1, axis=ax)
        lam = plan.eigenvalues(ax)
        fh = tpt.field_to_host(plan.transform(tpt.field_to_device(f), ax, False), n)
        tfh = tpt.field_to_host(plan.transform(tpt.field_to_device(Tf), ax, False), n)
        scale = np.abs(tfh).max()
        assert np.abs(tfh - lam.reshape(shape) * fh).max() <= 1e-12 * scale
        back = tpt.field_to_host(plan.transform(tpt.field_to_device(fh), ax, True), n)
        assert _relerr(back, f) <= 1e-13


def test_thomas_matches_oracle_recurrence():
    n = (37, 29, 41)
    for bcs, coef in [(BCS["NNN"], (0.0, 1.0)), (BCS["DND"], (1.0, -0.01)), (BCS["NNN"], (1.0, -5e-4))]:
        dirs = O.make_dirs(n, (1.5, 2.0, 2.5), bcs)
        plan = _plan(dirs, *coef)
        lx, ly = plan.eigenvalues(0), plan.eigenvalues(1)
        fh = S.uniform_rhs(n, 8)
        sing = O.is_singular(dirs, coef[0])
        ref_in = fh.copy()
        if sing:   # the kernel projects the null line; give the oracle the projected line
            w = dirs[2].dxf
            ref_in[0, 0, :] -= np.sum(w * ref_in[0, 0, :]) / np.sum(w)
        ref = O.thomas_modal(ref_in, lx, ly, dirs[2], coef[0], coef[1], (0, 0) if sing else None)
        if sing:
            w = dirs[2].dxf
            ref[0, 0, :] -= np.sum(w * ref[0, 0, :]) / np.sum(w)
        got = tpt.field_to_host(plan.thomas(tpt.field_to_device(fh)), n)
        assert _relerr(got, ref) <= 1e-13


def test_residual_matches_oracle_stencil():
    n = (33, 20, 17)
    for bcs in BCS.values():
        dirs = O.make_dirs(n, (0.0 if bcs[0][0] == P_ else 1.5, 2.0, 2.5), bcs)
        plan = _plan(dirs, 0.7, -1.3)
        f, phi = S.uniform_rhs(n, 1), S.uniform_rhs(n, 2)
        sums = torch.zeros(3, dtype=torch.float64, device="cuda")
        r = tpt.field_to_host(plan.residual(tpt.field_to_device(f), tpt.field_to_device(phi), sums=sums), n)
        ref = O.residual(f, phi, dirs, 0.7, -1.3)
        assert np.abs(r - ref).max() <= 1e-13 * np.abs(ref).max()
        s = sums.cpu().numpy()
        assert abs(s[0] - np.sum(ref ** 2)) <= 1e-12 * np.sum(ref ** 2)
        vol = O.cell_volumes(dirs)
        assert abs(s[2] - np.sum(vol * ref)) <= 1e-12 * np.sum(np.abs(vol * ref))
