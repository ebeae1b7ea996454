"""Fourier-based transforms (real DFT / DCT-II-III) of uniform directions on
GB300 against the CPU oracle, and against the eigenbasis-GEMM transforms on the
same uniform grid (the two must give the same solution)."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as S
from _tpt import load

pytestmark = pytest.mark.gpu
tpt, L = load()
N_, P_ = O.NEUMANN, O.PERIODIC
TOL = 1e-12


def _dirs(n, bcs, stretch):
    out = []
    for a in range(3):
        g = O.uniform_grid(n[a]) if stretch[a] == 0.0 else O.tanh_grid(n[a], 1.0, stretch[a])
        out.append(O.Direction(*g, bcs[a]))
    return out


def _plan(dirs, alpha, beta, xform):
    return tpt.Plan(tuple(d.n for d in dirs), [d.dxf for d in dirs], [d.dxc for d in dirs],
                    [d.bc for d in dirs], xform=xform, alpha=alpha, beta=beta, max_refine=1)


def _solve(plan, f, n):
    phi, info = plan.solve(tpt.field_to_device(f))
    return tpt.field_to_host(phi, n), info


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_config1_fft_x_gemm_y():
    n = (32, 32, 32)
    dirs = _dirs(n, [(P_, P_), (N_, N_), (N_, N_)], (0.0, 1.5, 1.5))
    f = S.remove_weighted_mean(S.uniform_rhs(n, 1), [d.dxf for d in dirs])
    plan = _plan(dirs, 0.0, 1.0, (tpt.AUTO, tpt.AUTO))
    assert plan.transforms() == (tpt.FFT, tpt.GEMM)
    got, info = _solve(plan, f, n)
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    assert _rel(got, ref) <= TOL
    # manufactured solution cos(2 pi x) cos(pi y) cos(pi z), discrete f = A u
    cen = []
    for d in dirs:
        faces = np.concatenate([[0.0], np.cumsum(d.dxf)])
        cen.append(0.5 * (faces[1:] + faces[:-1]))
    u = np.einsum("i,j,k->ijk", np.cos(2 * np.pi * cen[0]), np.cos(np.pi * cen[1]), np.cos(np.pi * cen[2]))
    got, _ = _solve(plan, O.apply_operator(u, dirs, 0.0, 1.0), n)
    assert _rel(got, u) <= TOL


@pytest.mark.parametrize("coef", [(0.0, 1.0), (1.0, -5e-4)])
@pytest.mark.parametrize("bcs", [[(N_, N_)] * 3, [(P_, P_), (P_, P_), (N_, N_)], [(N_, N_), (P_, P_), (N_, N_)]])
def test_uniform_fft_equals_gemm_equals_oracle(coef, bcs):
    n = (64, 32, 24)
    dirs = _dirs(n, bcs, (0.0, 0.0, 2.0))
    f = S.uniform_rhs(n, 13)
    if coef[0] == 0.0:
        f = S.remove_weighted_mean(f, [d.dxf for d in dirs])
    ref, _ = O.solve_tensor(f, dirs, *coef)
    ff = _plan(dirs, *coef, (tpt.FFT, tpt.FFT))
    gg = _plan(dirs, *coef, (tpt.GEMM, tpt.GEMM))
    a, _ = _solve(ff, f, n)
    b, _ = _solve(gg, f, n)
    assert _rel(a, ref) <= TOL and _rel(b, ref) <= TOL and _rel(a, b) <= TOL


@pytest.mark.parametrize("n", [(2, 4, 5), (1, 8, 3), (16, 1, 7), (4, 2, 1)])
def test_small_and_degenerate_fft_sizes(n):
    dirs = _dirs(n, [(P_, P_), (N_, N_), (N_, N_)], (0.0, 0.0, 1.3))
    f = S.remove_weighted_mean(S.uniform_rhs(n, 3), [d.dxf for d in dirs])
    plan = _plan(dirs, 0.0, 1.0, (tpt.FFT, tpt.FFT))
    got, _ = _solve(plan, f, n)
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    assert np.abs(got - ref).max() <= TOL * max(np.abs(ref).max(), 1e-30)


@pytest.mark.parametrize("bc", [(P_, P_), (N_, N_)])
def test_fft_transform_diagonalises_and_inverts(bc):
    n = (128, 64, 6)
    dirs = _dirs(n, [bc, bc, (N_, N_)], (0.0, 0.0, 1.0))
    plan = _plan(dirs, 0.0, 1.0, (tpt.FFT, tpt.FFT))
    f = S.uniform_rhs(n, 4)
    for ax in (0, 1):
        d = dirs[ax]
        shape = [1, 1, 1]
        shape[ax] = n[ax]
        a, b, c = (v.reshape(shape) for v in (d.a, d.b, d.c))
        Tf = b * f + a * np.roll(f, 1, axis=ax) + c * np.roll(f, -1, axis=ax)
        lam = plan.eigenvalues(ax)
        fh = tpt.field_to_host(plan.transform(tpt.field_to_device(f), ax, False), n)
        tfh = tpt.field_to_host(plan.transform(tpt.field_to_device(Tf), ax, False), n)
        assert np.abs(tfh - lam.reshape(shape) * fh).max() <= 1e-11 * np.abs(tfh).max()
        back = tpt.field_to_host(plan.transform(tpt.field_to_device(fh), ax, True), n)
        assert _rel(back, f) <= 1e-14


def test_config2_uniform_variant_fft_vs_gemm_256():
    # config 2's cross-check: the uniform 256^3 all-Neumann grid, eigenbasis GEMM
    # against DCT transforms, both against the oracle
    n = (256, 256, 256)
    dirs = _dirs(n, [(N_, N_)] * 3, (0.0, 0.0, 0.0))
    f = S.remove_weighted_mean(S.uniform_rhs(n, 2), [d.dxf for d in dirs])
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    a, _ = _solve(_plan(dirs, 0.0, 1.0, (tpt.FFT, tpt.FFT)), f, n)
    b, _ = _solve(_plan(dirs, 0.0, 1.0, (tpt.GEMM, tpt.GEMM)), f, n)
    assert _rel(a, ref) <= TOL and _rel(b, ref) <= TOL
