"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test ties one part of ``oracle/`` to something other than itself: values
printed in the paper (tests/golden/), closed-form eigenvalues, textbook or
library routines (dense LU, banded solve, FFT/DCT diagonalisation), exact
identities and a discretisation-convergence check.  No GPU is used.
"""
import os

import numpy as np
import pytest
import scipy.fft as sfft
import scipy.linalg as sla
import scipy.sparse as sp

import oracle as O
import seeded_inputs as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")
BC_N, BC_P, BC_D = O.NEUMANN, O.PERIODIC, O.DIRICHLET


def _rows(path):
    with open(path) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


# ------------------------------------------------------------------ inputs

def test_splitmix64_published_outputs():
    for seed, ctr, val in _rows(os.path.join(GOLD, "splitmix64.txt")):
        got = S.splitmix64(int(seed), np.array([int(ctr)], dtype=np.uint64))[0]
        assert int(got) == int(val)


def test_uniform_rhs_range_and_indexing():
    f = S.uniform_rhs((5, 4, 3), seed=7)
    assert f.shape == (5, 4, 3) and f.min() >= -1.0 and f.max() < 1.0
    # element (i, j, k) is the value at linear Fortran index i + 5*(j + 4*k)
    z = S.splitmix64(7, np.array([2 + 5 * (3 + 4 * 1)], dtype=np.uint64))[0]
    assert f[2, 3, 1] == (int(z) >> 11) * 2.0 ** -53 * 2.0 - 1.0


# -------------------------------------------------------------------- grid

def test_grading_ratios_printed_in_paper():
    for n, alpha, ratio, digits in _rows(os.path.join(GOLD, "grading_ratios.txt")):
        dxf, _ = O.tanh_grid(int(n), 1.0, float(alpha))
        got = dxf.max() / dxf.min()
        assert round(got, int(digits)) == float(ratio), (n, alpha, got)


@pytest.mark.parametrize("alpha", [1.0, 2.0, 3.0])
def test_grading_ratio_large_n_limit(alpha):
    # footnote to Eq. (tanh_stretching): Delta_max/Delta_min -> cosh^2(alpha/2)
    dxf, _ = O.tanh_grid(1 << 16, 1.0, alpha)
    assert abs(dxf.max() / dxf.min() / np.cosh(alpha / 2) ** 2 - 1.0) < 1e-4


def test_grid_geometry():
    dxf, dxc = O.tanh_grid(40, 2.0, 2.5)
    assert abs(dxf.sum() - 2.0) < 1e-14 and np.all(dxf > 0)
    # centre spacing is the mean of the two adjacent cell widths
    assert np.allclose(dxc[1:40], 0.5 * (dxf[1:] + dxf[:-1]), rtol=1e-14, atol=0)
    assert dxc[0] == dxc[40] == 0.5 * (dxf[0] + dxf[-1])
    u, uc = O.tanh_grid(16, 1.0, 0.0)
    assert np.allclose(u, 1 / 16, rtol=1e-15) and np.allclose(uc, 1 / 16, rtol=1e-14)


# -------------------------------------------------------------- operator

@pytest.mark.parametrize("bc", [(BC_N, BC_N), (BC_P, BC_P), (BC_D, BC_N), (BC_D, BC_D)])
def test_row_scaled_operator_is_symmetric(bc):
    # Sec. 2.2.1: dx_i c_i = dx_{i+1} a_{i+1}, hence D T symmetric
    d = O.Direction(*O.tanh_grid(33, 1.0, 2.0), bc)
    lhs = d.dxf[:-1] * d.c[:-1]
    rhs = d.dxf[1:] * d.a[1:]
    assert np.allclose(lhs, rhs, rtol=4e-16, atol=0)
    S_ = d.dxf[:, None] * d.dense()
    assert np.allclose(S_, S_.T, rtol=4e-16, atol=0)


def _staggered_div_grad(dirs):
    """Divergence and gradient on the staggered grid written from the geometry:
    face velocities, cell widths and centre spacings (not from the 1D rows)."""
    def grad(phi, ax, d):
        p = np.moveaxis(phi, ax, 0)
        g = np.zeros((d.n + 1,) + p.shape[1:])
        g[1:d.n] = (p[1:] - p[:-1]) / d.dxc[1:d.n].reshape((-1,) + (1,) * (p.ndim - 1))
        if d.periodic:
            g[0] = g[d.n] = (p[0] - p[-1]) / d.dxc[0]
        return np.moveaxis(g, 0, ax)

    def div(vel):
        out = 0.0
        for ax, d in enumerate(dirs):
            u = np.moveaxis(vel[ax], ax, 0)
            dd = (u[1:] - u[:-1]) / d.dxf.reshape((-1,) + (1,) * (u.ndim - 1))
            out = out + np.moveaxis(dd, 0, ax)
        return out
    return div, grad


@pytest.mark.parametrize("bcx", [(BC_N, BC_N), (BC_P, BC_P)])
def test_projection_of_white_noise_is_divergence_free(bcx):
    # Sec. 4.1: projecting a white-noise velocity gives a discretely
    # divergence-free field to machine precision (needs L = D o G).
    n = (12, 10, 9)
    dirs = O.make_dirs(n, (0.0 if bcx[0] == BC_P else 1.7, 2.2, 2.9),
                       [bcx, (BC_N, BC_N), (BC_N, BC_N)])
    div, grad = _staggered_div_grad(dirs)
    rng = np.random.default_rng(11)
    vel = []
    for ax, d in enumerate(dirs):
        shp = list(n)
        shp[ax] = d.n + 1
        u = rng.uniform(-1, 1, shp)
        u = np.moveaxis(u, ax, 0)
        if d.periodic:
            u[d.n] = u[0]
        else:
            u[0] = 0.0
            u[d.n] = 0.0
        vel.append(np.moveaxis(u, 0, ax))
    rhs = div(vel)
    phi, defect = O.solve_tensor(rhs, dirs, 0.0, 1.0)
    assert abs(defect) < 1e-13
    newvel = [vel[ax] - grad(phi, ax, d) for ax, d in enumerate(dirs)]
    assert np.abs(div(newvel)).max() < 1e-12 * np.abs(rhs).max()


def test_stencil_matches_dense_matvec():
    dirs = O.make_dirs((5, 6, 4), (1.0, 2.0, 3.0), [(BC_P, BC_P), (BC_D, BC_N), (BC_N, BC_N)])
    phi = S.uniform_rhs((5, 6, 4), 9)
    A = O.assemble_dense(dirs, 0.7, -1.3)
    ref = (A @ phi.ravel(order="F")).reshape(phi.shape, order="F")
    got = O.apply_operator(phi, dirs, 0.7, -1.3)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


# -------------------------------------------------------------- eigenbasis

def _uniform_dir(n, bc):
    return O.Direction(*O.uniform_grid(n), bc)


@pytest.mark.parametrize("n", [8, 32, 64])
def test_uniform_eigenvalues_closed_form(n):
    h = 1.0 / n
    k = np.arange(n)
    # 2(cos t - 1)/h^2 written as -4 sin^2(t/2)/h^2 to avoid cancellation
    cases = {
        (BC_N, BC_N): -4 * np.sin(np.pi * k / (2 * n)) ** 2 / h ** 2,           # DCT-II modes
        (BC_P, BC_P): -4 * np.sin(np.pi * k / n) ** 2 / h ** 2,                 # Fourier modes
        (BC_D, BC_D): -4 * np.sin(np.pi * (k + 1) / (2 * n)) ** 2 / h ** 2,     # DST-II modes
        (BC_D, BC_N): -4 * np.sin(np.pi * (k + 0.5) / (2 * n)) ** 2 / h ** 2,   # DST-IV modes
    }
    for bc, lam in cases.items():
        e = O.Eigenbasis(_uniform_dir(n, bc))
        got, ref = np.sort(e.lam), np.sort(lam)
        tol = 1e-13 * np.maximum(np.abs(ref), 1.0 / h ** 2 * 1e-3)
        assert np.all(np.abs(got - ref) <= tol), (bc, np.abs(got - ref).max())


@pytest.mark.parametrize("bc", [(BC_N, BC_N), (BC_P, BC_P), (BC_D, BC_N)])
def test_eigenbasis_identities(bc):
    d = O.Direction(*O.tanh_grid(48, 1.0, 2.5 if bc[0] != BC_P else 0.0), bc)
    e = O.Eigenbasis(d)
    T = d.dense()
    n = d.n
    normT = np.abs(T).max()
    assert np.abs(e.Qt.T @ e.Qt - np.eye(n)).max() < 1e-13
    assert np.abs(e.Qinv @ e.Q - np.eye(n)).max() < 1e-12
    # T Q = Q Lambda (Eq. q-from-tildeq with T = Q Lambda Q^{-1})
    res = T @ e.Q - e.Q * e.lam[None, :]
    assert np.abs(res).max() < 1e-12 * normT * np.abs(e.Q).max()
    if d.has_null_mode:
        assert e.lam[e.null] == 0.0
        v = e.Q[:, e.null]
        assert np.ptp(v) < 1e-13 * np.abs(v).max()     # null vector of T is constant


def test_smallest_eigenvalues_carry_relative_accuracy():
    # reading R7: Rayleigh quotients in long double recover the smallest
    # eigenvalues to relative accuracy, where the plain float64 eigensolver
    # carries absolute error ~eps*||T||.  The uniform grid has exact values.
    n = 512
    e = O.Eigenbasis(_uniform_dir(n, (BC_N, BC_N)))
    k = np.arange(n)
    ref = np.sort(-4 * np.sin(np.pi * k / (2 * n)) ** 2 * n * n)
    got = np.sort(e.lam)
    small = slice(n - 6, n - 1)   # five smallest nonzero magnitudes
    assert np.all(np.abs(got[small] - ref[small]) <= 1e-14 * np.abs(ref[small]))


# ------------------------------------------------------------------- solves

BC_COMBOS = [
    [(BC_N, BC_N)] * 3,
    [(BC_P, BC_P), (BC_N, BC_N), (BC_N, BC_N)],
    [(BC_P, BC_P), (BC_P, BC_P), (BC_D, BC_N)],
    [(BC_D, BC_D), (BC_N, BC_D), (BC_D, BC_N)],
]


@pytest.mark.parametrize("bcs", BC_COMBOS)
@pytest.mark.parametrize("coef", [(0.0, 1.0), (1.0, -5e-4), (1.0, -0.3)])
@pytest.mark.parametrize("stretch", [(0.0, 0.0, 0.0), (1.5, 2.0, 2.5)])
def test_tensor_solve_equals_dense_lu(bcs, coef, stretch):
    n = (7, 6, 8)
    dirs = O.make_dirs(n, stretch, bcs)
    f = S.uniform_rhs(n, 4)
    pd, mu = O.solve_dense(f, dirs, *coef)
    pt, defect = O.solve_tensor(f, dirs, *coef)
    assert np.abs(pt - pd).max() <= 1e-13 * np.abs(pd).max()
    assert abs(mu - defect) <= 1e-13


def test_z_only_case_is_one_tridiagonal_solve():
    # Nx = Ny = 1: both diagonalised directions are 1-point, so the solve is
    # one tridiagonal system along z (banded LAPACK solve as the reference).
    dirs = O.make_dirs((1, 1, 50), (0, 0, 2.0), [(BC_N, BC_N), (BC_N, BC_N), (BC_D, BC_N)])
    f = S.uniform_rhs((1, 1, 50), 2)
    alpha, beta = 1.0, -0.01
    dz = dirs[2]
    ab = np.zeros((3, 50))
    ab[0, 1:] = beta * dz.c[:-1]
    ab[1, :] = alpha + beta * dz.b
    ab[2, :-1] = beta * dz.a[1:]
    ref = sla.solve_banded((1, 1), ab, f[0, 0, :])
    got, _ = O.solve_tensor(f, dirs, alpha, beta)
    assert np.abs(got[0, 0] - ref).max() <= 1e-14 * np.abs(ref).max()


def test_identity_coefficients():
    dirs = O.make_dirs((6, 5, 4), (1.0, 2.0, 3.0), [(BC_N, BC_N)] * 3)
    f = S.uniform_rhs((6, 5, 4), 5)
    got, _ = O.solve_tensor(f, dirs, 1.0, 0.0)
    assert np.abs(got - f).max() < 1e-14


def test_gauge_and_compatibility_projection():
    dirs = O.make_dirs((9, 8, 7), (1.5, 2.0, 2.5), [(BC_N, BC_N)] * 3)
    f = S.remove_weighted_mean(S.uniform_rhs((9, 8, 7), 6), [d.dxf for d in dirs])
    p0, d0 = O.solve_tensor(f, dirs, 0.0, 1.0)
    p1, d1 = O.solve_tensor(f + 0.25, dirs, 0.0, 1.0)
    assert abs(d0) < 1e-15 and abs(d1 - 0.25) < 1e-14
    assert np.abs(p1 - p0).max() < 1e-13 * np.abs(p0).max()
    assert abs(O.weighted_mean(p0, dirs)) < 1e-15 * np.abs(p0).max() * 10


def _sparse_operator(dirs, alpha, beta):
    Tx, Ty, Tz = (sp.csr_matrix(d.dense()) for d in dirs)
    Ix, Iy, Iz = (sp.identity(d.n, format="csr") for d in dirs)
    L = sp.kron(Iz, sp.kron(Iy, Tx)) + sp.kron(Iz, sp.kron(Ty, Ix)) + sp.kron(Tz, sp.kron(Iy, Ix))
    return alpha * sp.identity(L.shape[0]) + beta * L


def _centres(d):
    faces = np.concatenate([[0.0], np.cumsum(d.dxf)])
    return 0.5 * (faces[1:] + faces[:-1])


def test_discrete_manufactured_solution_32cube():
    # config-1 grid: x periodic uniform, y and z tanh(1.5) Neumann; f = A u for
    # u = cos(2 pi x) cos(pi y) cos(pi z) at the cell centres.
    n = (32, 32, 32)
    dirs = O.make_dirs(n, (0.0, 1.5, 1.5), [(BC_P, BC_P), (BC_N, BC_N), (BC_N, BC_N)])
    x, y, z = (_centres(d) for d in dirs)
    u = np.einsum("i,j,k->ijk", np.cos(2 * np.pi * x), np.cos(np.pi * y), np.cos(np.pi * z))
    A = _sparse_operator(dirs, 0.0, 1.0)
    f = (A @ u.ravel(order="F")).reshape(n, order="F")
    phi, defect = O.solve_tensor(f, dirs, 0.0, 1.0)
    assert abs(defect) < 1e-12 * np.abs(f).max()
    assert np.abs(phi - u).max() < 1e-13


def test_continuous_manufactured_solution_converges_second_order():
    errs = []
    for m in (16, 32, 64):
        dirs = O.make_dirs((m, m, m), (0.0, 1.5, 1.5), [(BC_P, BC_P), (BC_N, BC_N), (BC_N, BC_N)])
        x, y, z = (_centres(d) for d in dirs)
        u = np.einsum("i,j,k->ijk", np.cos(2 * np.pi * x), np.cos(np.pi * y), np.cos(np.pi * z))
        phi, _ = O.solve_tensor(-6 * np.pi ** 2 * u, dirs, 0.0, 1.0)
        errs.append(np.abs(phi - u).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs


def test_uniform_grid_matches_fft_dct_diagonalisation():
    # Sec. 2.2.1: on a uniform grid the eigenbasis solve is the Fourier-based
    # solve.  Reference: FFT along periodic x, DCT-II along Neumann y and z.
    n = (16, 12, 10)
    dirs = [_uniform_dir(n[0], (BC_P, BC_P)), _uniform_dir(n[1], (BC_N, BC_N)),
            _uniform_dir(n[2], (BC_N, BC_N))]
    f = S.remove_weighted_mean(S.uniform_rhs(n, 8), [d.dxf for d in dirs])
    h = [1.0 / m for m in n]
    kx = np.arange(n[0])
    lx = 2 * (np.cos(2 * np.pi * kx / n[0]) - 1) / h[0] ** 2
    ly = 2 * (np.cos(np.pi * np.arange(n[1]) / n[1]) - 1) / h[1] ** 2
    lz = 2 * (np.cos(np.pi * np.arange(n[2]) / n[2]) - 1) / h[2] ** 2
    fh = sfft.fft(sfft.dctn(f, type=2, axes=(1, 2), norm="ortho"), axis=0)
    lam = lx[:, None, None] + ly[None, :, None] + lz[None, None, :]
    lam[0, 0, 0] = 1.0
    ph = fh / lam
    ph[0, 0, 0] = 0.0
    ref = np.real(sfft.idctn(sfft.ifft(ph, axis=0), type=2, axes=(1, 2), norm="ortho"))
    for alpha_beta in [(0.0, 1.0)]:
        got, _ = O.solve_tensor(f, dirs, *alpha_beta)
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_residual_is_at_round_off_in_long_double():
    # Sec. 4.1: the algebraic residual f - T phi is at round-off at every point.
    n = (20, 18, 16)
    dirs = O.make_dirs(n, (1.5, 2.0, 2.5), [(BC_N, BC_N)] * 3)
    f = S.remove_weighted_mean(S.uniform_rhs(n, 4), [d.dxf for d in dirs])
    phi, _ = O.solve_tensor(f, dirs, 0.0, 1.0, refine=2, residual_dtype=np.longdouble)
    r = O.residual(f, phi, dirs, 0.0, 1.0, np.longdouble)
    scale = max(d.b.__abs__().max() for d in dirs) * np.abs(phi).max()
    assert float(np.abs(r).max()) < 8 * np.finfo(float).eps * scale


# ------------------------------------------------ pressure projection (N4)

def _faces_of(d):
    """Face coordinates of a direction from its cell widths (R1)."""
    return np.concatenate([[0.0], np.cumsum(d.dxf)])


def _random_velocity(n, dirs, seed):
    rng = np.random.default_rng(seed)
    vel = []
    for ax, d in enumerate(dirs):
        shp = list(n)
        shp[ax] = d.n + 1
        u = np.moveaxis(rng.uniform(-1, 1, shp), ax, 0)
        if d.periodic:
            u[d.n] = u[0]
        else:
            u[0] = 0.0
            u[d.n] = 0.0
        vel.append(np.moveaxis(u, 0, ax))
    return vel


def test_divergence_and_gradient_of_linear_fields_are_one():
    # closed forms: D of u = x_face along x is 1 in every cell; G of p = x_centre
    # is 1 on every interior face (R9), exactly up to rounding
    n = (9, 7, 6)
    dirs = O.make_dirs(n, (2.0, 1.3, 2.7), [(BC_N, BC_N)] * 3)
    for ax, d in enumerate(dirs):
        xf = _faces_of(d)
        shp = [1, 1, 1]
        shp[ax] = d.n + 1
        vel = [np.zeros((n[0] + (a == 0), n[1] + (a == 1), n[2] + (a == 2))) for a in range(3)]
        vel[ax] = np.broadcast_to(xf.reshape(shp), vel[ax].shape).copy()
        assert np.allclose(O.divergence(vel, dirs), 1.0, rtol=0, atol=1e-13)
        xc = 0.5 * (xf[1:] + xf[:-1])
        shp2 = [1, 1, 1]
        shp2[ax] = d.n
        p = np.broadcast_to(xc.reshape(shp2), n).copy()
        g = np.moveaxis(O.gradient(p, dirs)[ax], ax, 0)
        assert np.allclose(g[1:d.n], 1.0, rtol=0, atol=1e-12)
        assert np.all(g[0] == 0.0) and np.all(g[d.n] == 0.0)          # walls


@pytest.mark.parametrize("bcs", [[(BC_N, BC_N)] * 3, [(BC_P, BC_P), (BC_N, BC_N), (BC_N, BC_N)]])
def test_divergence_of_gradient_is_the_operator(bcs):
    # D o G equals the 7-point operator of the paper's 1D rows (Eq. poisson-fd2)
    n = (8, 7, 6)
    dirs = O.make_dirs(n, (0.0 if bcs[0][0] == BC_P else 1.8, 2.4, 1.6), bcs)
    phi = S.uniform_rhs(n, 31)
    got = O.divergence(O.gradient(phi, dirs), dirs)
    ref = O.apply_operator(phi, dirs, 0.0, 1.0)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("bcx", [(BC_N, BC_N), (BC_P, BC_P)])
def test_oracle_projection_is_divergence_free_and_idempotent(bcx):
    n = (11, 9, 8)
    dirs = O.make_dirs(n, (0.0 if bcx[0] == BC_P else 1.5, 2.5, 3.0), [bcx, (BC_N, BC_N), (BC_N, BC_N)])
    vel = _random_velocity(n, dirs, 12)
    gdt = 0.37
    new, phi, defect = O.project(vel, dirs, gdt)
    div0 = np.abs(O.divergence(vel, dirs)).max()
    assert abs(defect) < 1e-12 * div0 / gdt
    assert np.abs(O.divergence(new, dirs)).max() <= 1e-12 * div0
    again, phi2, _ = O.project(new, dirs, gdt)
    for a in range(3):
        assert np.abs(again[a] - new[a]).max() <= 1e-12 * np.abs(new[a]).max()
    # wall faces keep their (zero) values
    for ax, d in enumerate(dirs):
        if not d.periodic:
            u = np.moveaxis(new[ax], ax, 0)
            assert np.all(u[0] == 0.0) and np.all(u[d.n] == 0.0)


# ------------------------------ N3: node Dirichlet, face grids, yz / z options

BC_DN, BC_X = O.DIRICHLET_NODE, O.NONE


def test_node_dirichlet_eigenvalues_closed_form():
    # uniform face-centred unknowns between two walls: m = n - 1 interior faces
    # of spacing h; the rows are tridiag(1, -2, 1)/h^2 whose eigenvalues are
    # -4/h^2 sin^2(k pi / (2 (m + 1))), k = 1..m
    n, L = 17, 1.0
    dxf, dxc = O.uniform_grid(n, L)
    wf, sf = O.face_grid(dxf, dxc, periodic=False)
    d = O.Direction(wf, sf, (BC_DN, BC_DN))
    lam = np.sort(np.linalg.eigvalsh(d.dense()))
    m, h = n - 1, L / n
    ref = np.sort(-4.0 / h ** 2 * np.sin(np.arange(1, m + 1) * np.pi / (2 * (m + 1))) ** 2)
    assert np.abs(lam - ref).max() <= 1e-12 * np.abs(ref).max()


def test_face_grid_control_volumes():
    dxf, dxc = O.tanh_grid(14, 1.0, 2.2)
    w, s = O.face_grid(dxf, dxc, periodic=False)
    # the face control volumes tile [centre 0, centre n-1]; neighbours are a cell apart
    assert w.size == 13 and s.size == 14
    assert abs(w.sum() - (1.0 - 0.5 * dxf[0] - 0.5 * dxf[-1])) <= 1e-14
    assert np.array_equal(s, dxf)
    wp, sp = O.face_grid(*O.uniform_grid(8), periodic=True)
    assert wp.size == 8 and sp.size == 9 and abs(wp.sum() - 1.0) <= 1e-14


def test_z_option_is_independent_line_solves():
    # only z in the operator: every (i, j) line is alpha + beta T_z alone
    n = (6, 5, 9)
    dirs = O.make_dirs(n, (1.5, 2.0, 2.5), [(BC_X, BC_X), (BC_X, BC_X), (BC_N, BC_D)])
    alpha, beta = 1.0, -7e-3
    f = S.uniform_rhs(n, 41)
    got, _ = O.solve_tensor(f, dirs, alpha, beta)
    dz = dirs[2]
    ab = np.zeros((3, n[2]))
    ab[0, 1:] = beta * dz.c[:-1]
    ab[1, :] = alpha + beta * dz.b
    ab[2, :-1] = beta * dz.a[1:]
    ref = np.empty(n)
    for i in range(n[0]):
        for j in range(n[1]):
            ref[i, j] = sla.solve_banded((1, 1), ab, f[i, j])
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_yz_option_is_independent_plane_solves():
    # y and z in the operator: every x-plane is a 2D problem alpha + beta (T_y + T_z)
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    n = (5, 7, 6)
    dirs = O.make_dirs(n, (1.0, 2.0, 1.5), [(BC_X, BC_X), (BC_P, BC_P), (BC_N, BC_N)])
    alpha, beta = 1.0, -3e-3
    f = S.uniform_rhs(n, 43)
    got, _ = O.solve_tensor(f, dirs, alpha, beta)
    ty, tz = sp.csr_matrix(dirs[1].dense()), sp.csr_matrix(dirs[2].dense())
    a2 = alpha * sp.identity(n[1] * n[2]) + beta * (sp.kron(sp.identity(n[2]), ty) + sp.kron(tz, sp.identity(n[1])))
    ref = np.empty(n)
    for i in range(n[0]):
        ref[i] = spla.spsolve(a2.tocsc(), f[i].ravel(order="F")).reshape(n[1], n[2], order="F")
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
