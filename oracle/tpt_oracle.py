"""Plain CPU oracle for the tensor-product--Thomas Poisson/Helmholtz solve.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The CUDA product path never imports, links or calls it, and this module
imports nothing from the product package.

What it computes (paper sections cited per function):

* the staggered cell-centred grid of Eq. (tanh_stretching), Sec. 4.1;
* the 1D second-difference rows of Eq. (poisson-fd2)/(tridiagonal-coefficients),
  Sec. 2.2.1, with boundary rows (Neumann, periodic, Dirichlet);
* the 3D Kronecker-sum operator of Sec. 2.2.2 applied as a 7-point stencil, and
  assembled densely for tiny grids;
* the pressure projection of a staggered velocity field, Sec. 2.1 (the
  pressure-correction equation Eq. poi_ns and the velocity correction that
  follows it): divergence D, gradient G and u = u* - g G Phi with
  L Phi = D u* / g;
* the solve of (alpha I + beta L) phi = f:
    - ``solve_dense``: Gaussian elimination with partial pivoting on the
      assembled matrix (bordered when singular) -- the plain definition;
    - ``solve_tensor``: the paper's procedure of Sec. 2.2.2 (init 1.1-1.3,
      solution 2.1-2.5) with plain numpy matmuls and a scalar-recurrence Thomas
      sweep, followed by iterative refinement against the assembled stencil.

Readings of points the paper leaves open:

R1 grid: faces at x(k/N), k = 0..N, from Eq. (tanh_stretching); cell widths are
   face spacings, centres are face midpoints, centre spacings are the
   distances between neighbouring centres.  The wrap spacing of a periodic
   direction is (dx_0 + dx_{N-1})/2.
R2 domain length L = 1 in every direction unless given.
R3 boundary rows: Neumann drops the outside coupling (a_0 = 0 or c_{N-1} = 0);
   periodic keeps it as the cyclic corner; homogeneous Dirichlet (wall value
   zero at the face) drops the coupling and adds 2/dx^2 to -b at that row.
   Coefficients are formed exactly as a_i = 1/(dx_i*dx_{i-1/2}),
   c_i = 1/(dx_i*dx_{i+1/2}), b_i = -((a_i + c_i) + w_i) in IEEE float64, where
   w_i is the Dirichlet wall term; any implementation using the same formula
   gets bit-identical rows.
R4 gauge: a singular problem (alpha = 0 and every direction periodic or
   Neumann-Neumann) is solved for the canonical solution with zero
   cell-volume-weighted mean; in the tensor solve the modal unknown at the
   vanishing final pivot of the null line is set to zero, as the paper does,
   before the gauge is applied.
R5 compatibility: the right-hand side of a singular problem is projected by
   removing its volume-weighted mean (the left null vector of the operator is
   the vector of cell volumes); the removed mean is returned as the defect.
R6 the eigenvalue of the null mode is set to exactly 0.
R7 eigenvalues are recomputed as Rayleigh quotients of the float64 eigenvectors
   in long double, in the energy form of the symmetric row-scaled operator, so
   that the smallest eigenvalues carry relative (not absolute) accuracy.
R10 two more boundary kinds.  DIRICHLET_NODE: homogeneous Dirichlet with the
   zero value at the neighbouring node a centre spacing away (dxc[0] below,
   dxc[n] above): the coupling is dropped and its coefficient kept on the
   diagonal -- the wall row of face-centred unknowns, whose wall face is a
   boundary node.  NONE: the direction is not in the operator (the
   implicit-diffusion options yz and z of Sec. 2.1): zero rows, so the
   problem decouples along it.
R9 staggered velocity (projection): the x-velocity lives on the Nx + 1 x-faces
   of each x-line (face i between cells i-1 and i), likewise v, w; D u is the
   cell's net face flux over its width, (u_{i+1} - u_i)/dx_i summed over the
   three directions, and (G phi) on face i is (phi_i - phi_{i-1})/dx_{i-1/2}
   at interior faces and, on a periodic direction, across the wrap face 0 = N
   with the wrap spacing; G is zero on wall faces (no penetration), so the wall
   values of u are left as given.  With these, D o G is the operator of the
   1D rows with Neumann walls.
R8 the tensor solve is followed by ``refine`` steps of iterative refinement,
   each computing r = f - A phi with the stencil (float64 by default, long
   double on request) and adding the tensor solve of r.  A float64 eigensolver
   gives eigenvectors whose errors move a single direct solve by 1e-12 to 6e-11
   (relative, max-norm) on 256-512 point stretched grids; one refinement step
   brings the result to the exact discrete solution up to rounding.
"""
from __future__ import annotations

import numpy as np

PERIODIC, NEUMANN, DIRICHLET, DIRICHLET_NODE, NONE = 0, 1, 2, 3, 4
_BC_NAMES = {"periodic": PERIODIC, "neumann": NEUMANN, "dirichlet": DIRICHLET,
             "dirichlet_node": DIRICHLET_NODE, "none": NONE}


def _bc(code):
    return _BC_NAMES[code] if isinstance(code, str) else int(code)


# ---------------------------------------------------------------- grid (Sec. 4.1)

def tanh_grid(n: int, L: float = 1.0, alpha: float = 0.0):
    """Cell widths and centre spacings of an n-cell grid on [0, L].

    Faces follow Eq. (tanh_stretching): x(xi) = L/2 (1 + tanh(alpha (xi - 1/2)) /
    tanh(alpha/2)) at xi = k/n; alpha = 0 is the uniform limit.  Returns
    ``dxf`` (n cell widths) and ``dxc`` (n+1 entries: dxc[i] is the distance
    between the centres of cells i-1 and i for 1 <= i <= n-1, and dxc[0] =
    dxc[n] is the periodic wrap spacing (dx_0 + dx_{n-1})/2), reading R1.
    """
    xi = np.arange(n + 1, dtype=np.float64) / n
    if alpha == 0.0:
        xf = L * xi
    else:
        xf = 0.5 * L * (1.0 + np.tanh(alpha * (xi - 0.5)) / np.tanh(0.5 * alpha))
    dxf = np.diff(xf)
    xc = 0.5 * (xf[1:] + xf[:-1])
    dxc = np.empty(n + 1)
    dxc[1:n] = np.diff(xc)
    dxc[0] = dxc[n] = 0.5 * (dxf[0] + dxf[-1])
    return dxf, dxc


def uniform_grid(n: int, L: float = 1.0):
    """Exactly uniform spacing dx = L/n (cell widths and centre spacings)."""
    d = L / n
    return np.full(n, d), np.full(n + 1, d)


# ------------------------------------------------- 1D operator (Sec. 2.2.1)

def operator_1d(dxf, dxc, bc):
    """Rows (a, b, c) of the 1D operator, Eq. (tridiagonal-coefficients) with the
    boundary rows of reading R3.

    Row i reads  a_i phi_{i-1} + b_i phi_i + c_i phi_{i+1}.  For a periodic
    direction a_0 couples phi_{n-1} and c_{n-1} couples phi_0 (cyclic corners).
    ``bc`` = (lower, upper) codes.
    """
    dxf = np.asarray(dxf, dtype=np.float64)
    dxc = np.asarray(dxc, dtype=np.float64)
    n = dxf.size
    lo, hi = _bc(bc[0]), _bc(bc[1])
    if (lo == PERIODIC) != (hi == PERIODIC):
        raise ValueError("periodic must be set on both ends")
    if (lo == NONE) != (hi == NONE):
        raise ValueError("a direction outside the operator is so on both ends")
    if lo == NONE:                   # R10: the direction is not in the operator
        return np.zeros(n), np.zeros(n), np.zeros(n)
    with np.errstate(divide="ignore"):
        a = 1.0 / (dxf * dxc[:n])        # a_i = 1/(dx_i dx_{i-1/2})
        c = 1.0 / (dxf * dxc[1:n + 1])   # c_i = 1/(dx_i dx_{i+1/2})
    w = np.zeros(n)
    if lo != PERIODIC:
        if lo == DIRICHLET:
            w[0] += 2.0 / (dxf[0] * dxf[0])
        if hi == DIRICHLET:
            w[n - 1] += 2.0 / (dxf[n - 1] * dxf[n - 1])
        if lo == DIRICHLET_NODE:     # R10: zero value at the node dxc[0] below
            w[0] += a[0]
        if hi == DIRICHLET_NODE:     # and at the node dxc[n] above
            w[n - 1] += c[n - 1]
        a[0] = 0.0
        c[n - 1] = 0.0
    b = -((a + c) + w)
    return a, b, c


def face_grid(dxf, dxc, periodic: bool):
    """Spacings of the face-centred unknowns of a direction (R10): each unknown
    sits on a face, its control volume spans the two neighbouring centres and
    its neighbours are the adjacent faces.  Returns (widths, centre spacings)
    in the convention of ``tanh_grid``."""
    dxf = np.asarray(dxf, dtype=np.float64)
    dxc = np.asarray(dxc, dtype=np.float64)
    n = dxf.size
    if periodic:                     # faces 0..n-1, face n is face 0
        w = dxc[:n].copy()
        s = np.empty(n + 1)
        s[1:n] = dxf[:n - 1]
        s[0] = s[n] = dxf[n - 1]
        return w, s
    return dxc[1:n].copy(), dxf.copy()   # interior faces 1..n-1, walls are nodes


def dense_1d(a, b, c, periodic: bool):
    """Dense n x n matrix of the 1D rows, cyclic corners included."""
    n = b.size
    T = np.diag(b).astype(np.float64)
    for i in range(n):
        if i > 0:
            T[i, i - 1] += a[i]
        elif periodic:
            T[i, n - 1] += a[i]
        if i < n - 1:
            T[i, i + 1] += c[i]
        elif periodic:
            T[i, 0] += c[i]
    return T


class Direction:
    """One grid direction: spacings, boundary codes and its 1D rows."""

    def __init__(self, dxf, dxc, bc):
        self.dxf = np.asarray(dxf, dtype=np.float64)
        self.dxc = np.asarray(dxc, dtype=np.float64)
        self.bc = (_bc(bc[0]), _bc(bc[1]))
        self.periodic = self.bc[0] == PERIODIC
        self.n = self.dxf.size
        self.a, self.b, self.c = operator_1d(self.dxf, self.dxc, self.bc)

    @property
    def has_null_mode(self) -> bool:
        """Periodic and Neumann-Neumann rows sum to zero: constants are in the kernel."""
        return self.periodic or self.bc == (NEUMANN, NEUMANN)

    @property
    def excluded(self) -> bool:
        return self.bc[0] == NONE

    def dense(self):
        return dense_1d(self.a, self.b, self.c, self.periodic)


def is_singular(dirs, alpha) -> bool:
    return alpha == 0.0 and all(d.has_null_mode for d in dirs)


# --------------------------------------------- 3D operator (Sec. 2.2.2)

def apply_operator(phi, dirs, alpha, beta, dtype=np.float64):
    """(alpha I + beta L) phi with L = Tx (x) I (x) I + I (x) Ty (x) I + I (x) I (x) Tz,
    evaluated as the 7-point stencil of the 1D rows; phi is indexed (i, j, k)."""
    p = np.asarray(phi).astype(dtype)
    lap = np.zeros_like(p)
    for ax, d in enumerate(dirs):
        shape = [1, 1, 1]
        shape[ax] = d.n
        a = d.a.astype(dtype).reshape(shape)
        b = d.b.astype(dtype).reshape(shape)
        c = d.c.astype(dtype).reshape(shape)
        # a_i multiplies phi_{i-1}; c_i multiplies phi_{i+1}.  Non-periodic end
        # coefficients are zero, so the wrapped neighbour of np.roll never counts.
        lap += b * p
        lap += a * np.roll(p, 1, axis=ax)
        lap += c * np.roll(p, -1, axis=ax)
    return dtype(alpha) * p + dtype(beta) * lap


def residual(f, phi, dirs, alpha, beta, dtype=np.float64):
    """r = f - (alpha I + beta L) phi (Sec. 4.1 verification uses f - T phi)."""
    return np.asarray(f).astype(dtype) - apply_operator(phi, dirs, alpha, beta, dtype)


def assemble_dense(dirs, alpha, beta):
    """Dense matrix of alpha I + beta L on the Fortran-ordered vector (x fastest).

    The paper writes the Kronecker factors as (x, y, z) left to right; with x as
    the fastest storage index the same operator reads Iz (x) Iy (x) Tx + ...
    """
    Tx, Ty, Tz = (d.dense() for d in dirs)
    Ix, Iy, Iz = (np.eye(d.n) for d in dirs)
    L = (np.kron(Iz, np.kron(Iy, Tx)) + np.kron(Iz, np.kron(Ty, Ix))
         + np.kron(Tz, np.kron(Iy, Ix)))
    return alpha * np.eye(L.shape[0]) + beta * L


def cell_volumes(dirs):
    dx, dy, dz = (d.dxf for d in dirs)
    return np.einsum("i,j,k->ijk", dx, dy, dz)


def weighted_mean(f, dirs):
    w = cell_volumes(dirs)
    return float(np.sum(np.asarray(f, dtype=np.float64) * w) / np.sum(w))


# ------------------------------------------------------------ dense mode

def solve_dense(f, dirs, alpha, beta):
    """Plain definition: solve the assembled system by LU with partial pivoting.

    Singular case (reading R4/R5): the bordered system
        [A 1; v^T 0] [phi; mu] = [f; 0],   v = cell volumes,
    whose solution has zero weighted mean and absorbs the weighted mean of f
    in mu (A phi = f - mu).  Returns (phi, mu).
    """
    f = np.asarray(f, dtype=np.float64)
    A = assemble_dense(dirs, alpha, beta)
    fv = f.ravel(order="F")
    if is_singular(dirs, alpha):
        n = fv.size
        v = cell_volumes(dirs).ravel(order="F")
        M = np.zeros((n + 1, n + 1))
        M[:n, :n] = A
        M[:n, n] = 1.0
        M[n, :n] = v
        sol = np.linalg.solve(M, np.concatenate([fv, [0.0]]))
        return sol[:n].reshape(f.shape, order="F"), float(sol[n])
    return np.linalg.solve(A, fv).reshape(f.shape, order="F"), 0.0


# ------------------------------------------------------------ tensor mode

def rayleigh_eigenvalues(Qt, d: Direction):
    """Reading R7: lambda_k = v^T S v / v^T D v for v = D^{-1/2} q_k, in long double.

    S = D T is symmetric (Sec. 2.2.1: dx_i c_i = dx_{i+1} a_{i+1}); its quadratic
    form is written as  sum_i r_i v_i^2 - sum_{i<j} S_ij (v_i - v_j)^2  with r_i
    the row sums of S, which avoids the cancellation of the plain product.
    """
    ld = np.longdouble
    n = d.n
    S = d.dense().astype(ld) * d.dxf.astype(ld)[:, None]
    S = 0.5 * (S + S.T)
    v = Qt.astype(ld) / np.sqrt(d.dxf.astype(ld))[:, None]
    rows = S.sum(axis=1)
    num = np.sum(rows[:, None] * v * v, axis=0)
    iu, ju = np.triu_indices(n, 1)
    mask = S[iu, ju] != 0
    iu, ju = iu[mask], ju[mask]
    diff = v[iu, :] - v[ju, :]
    num -= np.sum(S[iu, ju][:, None] * diff * diff, axis=0)
    den = np.sum(d.dxf.astype(ld)[:, None] * v * v, axis=0)
    return (num / den).astype(np.float64)


class Eigenbasis:
    """Init steps 1.1-1.3 of Sec. 2.2.2 for one diagonalised direction.

    1.1  T~ = D^{1/2} T D^{-1/2}   (Eq. reverse-similarity-transform)
    1.2  T~ = Q~ Lambda Q~^T       (numpy.linalg.eigh: LAPACK symmetric eigensolver)
    1.3  Q = D^{-1/2} Q~, Q^{-1} = Q~^T D^{1/2}   (Eq. q-from-tildeq)
    Eigenvalues are then refined (R7) and the null eigenvalue set to 0 (R6).
    """

    def __init__(self, d: Direction):
        s = np.sqrt(d.dxf)
        T = d.dense()
        Tt = (s[:, None] * T) / s[None, :]
        lam, Qt = np.linalg.eigh(Tt)          # reads the lower triangle of T~
        lam = rayleigh_eigenvalues(Qt, d)
        self.null = -1
        if d.has_null_mode:
            self.null = int(np.argmax(lam))   # all eigenvalues are <= 0
            lam[self.null] = 0.0
        self.lam = lam
        self.Qt = Qt
        self.Q = Qt / s[:, None]
        self.Qinv = Qt.T * s[None, :]


def thomas_modal(fhat, lam_x, lam_y, dz: Direction, alpha, beta, null=None):
    """Step 2.3: (alpha + beta(lam_x_i + lam_y_j)) phi + beta T_z phi = fhat on every
    (i, j) line along z, by the Thomas recurrence (vectorised over lines,
    sequential in k).  ``null`` = (i0, j0) marks the singular line: its last
    modal unknown is set to zero (reading R4).
    """
    nx, ny, nz = fhat.shape
    shift = alpha + beta * (lam_x[:, None] + lam_y[None, :])
    sub = beta * dz.a
    sup = beta * dz.c
    diag0 = beta * dz.b
    cp = np.empty((nx, ny, nz))
    dp = np.empty((nx, ny, nz))
    last_pivot = 0.0
    m = diag0[0] + shift
    if nz == 1 and null is not None:
        last_pivot = m[null]
        m = m.copy()
        m[null] = 1.0
    cp[:, :, 0] = sup[0] / m
    dp[:, :, 0] = fhat[:, :, 0] / m
    for k in range(1, nz):
        m = (diag0[k] + shift) - sub[k] * cp[:, :, k - 1]
        if k == nz - 1 and null is not None:
            last_pivot = m[null]
            m = m.copy()
            m[null] = 1.0
        cp[:, :, k] = sup[k] / m
        dp[:, :, k] = (fhat[:, :, k] - sub[k] * dp[:, :, k - 1]) / m
    if null is not None:
        dp[null + (nz - 1,)] = 0.0
        scale = max(float(np.max(np.abs(diag0))), abs(beta))
        if abs(last_pivot) > 1e-10 * scale:
            raise AssertionError("null line final pivot %.3e does not vanish" % last_pivot)
    x = np.empty((nx, ny, nz))
    x[:, :, nz - 1] = dp[:, :, nz - 1]
    for k in range(nz - 2, -1, -1):
        x[:, :, k] = dp[:, :, k] - cp[:, :, k] * x[:, :, k + 1]
    return x


class TensorSolver:
    """The paper's 3D procedure (Sec. 2.2.2), x and y diagonalised, z by Thomas."""

    def __init__(self, dirs, alpha, beta):
        self.dirs = [d if isinstance(d, Direction) else Direction(*d) for d in dirs]
        if self.dirs[2].periodic:
            raise NotImplementedError("periodic z needs a cyclic tridiagonal solve")
        self.alpha, self.beta = float(alpha), float(beta)
        self.ex = Eigenbasis(self.dirs[0])
        self.ey = Eigenbasis(self.dirs[1])
        self.singular = is_singular(self.dirs, self.alpha)
        self.null = (self.ex.null, self.ey.null) if self.singular else None

    def direct(self, f):
        """Steps 2.1-2.5 on one right-hand side (float64 throughout)."""
        f = np.asarray(f, dtype=np.float64)
        fx = np.einsum("pi,ijk->pjk", self.ex.Qinv, f, optimize=True)       # 2.1
        fxy = np.einsum("qj,pjk->pqk", self.ey.Qinv, fx, optimize=True)     # 2.2
        ph = thomas_modal(fxy, self.ex.lam, self.ey.lam, self.dirs[2],
                          self.alpha, self.beta, self.null)                 # 2.3
        px = np.einsum("jq,pqk->pjk", self.ey.Q, ph, optimize=True)         # 2.4
        return np.einsum("ip,pjk->ijk", self.ex.Q, px, optimize=True)       # 2.5

    def solve(self, f, refine: int = 1, residual_dtype=np.float64):
        """Returns (phi, defect): phi in the canonical gauge, defect the weighted
        mean removed from f for compatibility (0 when non-singular)."""
        f = np.asarray(f, dtype=np.float64)
        defect = 0.0
        if self.singular:
            defect = weighted_mean(f, self.dirs)
            f = f - defect
        phi = self.direct(f)
        for _ in range(refine):
            r = residual(f, phi, self.dirs, self.alpha, self.beta, residual_dtype)
            r = r.astype(np.float64)
            if self.singular:
                r = r - weighted_mean(r, self.dirs)
            phi = phi + self.direct(r)
        if self.singular:
            phi = phi - weighted_mean(phi, self.dirs)
        return phi, defect


def solve_tensor(f, dirs, alpha, beta, refine: int = 1, residual_dtype=np.float64):
    return TensorSolver(dirs, alpha, beta).solve(f, refine, residual_dtype)


def make_dirs(n, stretch, bcs, L=(1.0, 1.0, 1.0)):
    """Directions for sizes n, tanh factors ``stretch`` and boundary pairs ``bcs``."""
    return [Direction(*tanh_grid(n[a], L[a], stretch[a]), bcs[a]) for a in range(3)]


# ------------------------------------- pressure projection (Sec. 2.1)

def divergence(vel, dirs):
    """D u on the cells (R9): vel = (u, v, w) with u of shape (Nx+1, Ny, Nz),
    v (Nx, Ny+1, Nz), w (Nx, Ny, Nz+1)."""
    out = 0.0
    for ax, d in enumerate(dirs):
        u = np.moveaxis(np.asarray(vel[ax], dtype=np.float64), ax, 0)
        flux = (u[1:] - u[:-1]) / d.dxf.reshape((-1,) + (1,) * (u.ndim - 1))
        out = out + np.moveaxis(flux, 0, ax)
    return out


def gradient(phi, dirs):
    """G phi on the faces of each direction (R9): zero on wall faces, the wrap
    difference on the shared boundary face of a periodic direction."""
    out = []
    for ax, d in enumerate(dirs):
        p = np.moveaxis(np.asarray(phi, dtype=np.float64), ax, 0)
        g = np.zeros((d.n + 1,) + p.shape[1:])
        g[1:d.n] = (p[1:] - p[:-1]) / d.dxc[1:d.n].reshape((-1,) + (1,) * (p.ndim - 1))
        if d.periodic:
            g[0] = (p[0] - p[-1]) / d.dxc[0]
            g[d.n] = g[0]
        out.append(np.moveaxis(g, 0, ax))
    return out


def project(vel, dirs, gdt, refine: int = 1):
    """The projection of Sec. 2.1 with g = gamma_k dt: Phi solves L Phi = D u / g
    (Poisson, zero volume-weighted mean), and the result is u - g G Phi.
    Returns (new velocity, Phi, the compatibility defect of D u / g)."""
    rhs = divergence(vel, dirs) / gdt
    phi, defect = solve_tensor(rhs, dirs, 0.0, 1.0, refine)
    grad = gradient(phi, dirs)
    return [np.asarray(vel[a], dtype=np.float64) - gdt * grad[a] for a in range(3)], phi, defect
