// Host setup of a plan (float64 with long-double refinement): grid helper, 1D
// operator rows with boundary rows, symmetrisation and symmetric
// eigendecomposition of each diagonalised direction.
//
// Paper: Sec. 2.2.1 (Eq. poisson-fd2, Eq. tridiagonal-coefficients,
// Eq. reverse-similarity-transform, Eq. q-from-tildeq, initialisation steps
// 1.1-1.3), Sec. 3 (eigendecomposition once per direction on the CPU, then
// copied to the GPU; Algorithm 1 initialisation), Sec. 4.1 (Eq. tanh_stretching).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <numeric>
#include <vector>

#include "tpt_internal.h"

namespace tpt {

int grid_faces(int n, const double* dxf, const double* dxc, int periodic, int* n_out, double* dxf_out,
               double* dxc_out) {
  if (n < 1 || !dxf || !dxc || !n_out || !dxf_out || !dxc_out) return TPT_ERR_INVALID_ARG;
  if (periodic) {
    for (int j = 0; j < n; ++j) dxf_out[j] = dxc[j];            // face j spans centres j-1 .. j
    dxc_out[0] = dxc_out[n] = dxf[n - 1];                       // faces n-1 and n = 0 across the wrap
    for (int j = 1; j < n; ++j) dxc_out[j] = dxf[j - 1];        // faces j-1 and j
    *n_out = n;
    return TPT_OK;
  }
  if (n < 2) return TPT_ERR_INVALID_ARG;
  for (int j = 0; j < n - 1; ++j) dxf_out[j] = dxc[j + 1];      // interior face j + 1
  for (int j = 0; j <= n - 1; ++j) dxc_out[j] = dxf[j];         // faces j and j + 1 (walls at the ends)
  *n_out = n - 1;
  return TPT_OK;
}

int grid_tanh(int n, double L, double stretch, double* dxf, double* dxc) {
  if (n < 1 || !(L > 0.0) || !(stretch >= 0.0) || !dxf || !dxc) return TPT_ERR_INVALID_ARG;
  std::vector<double> xf(n + 1);
  for (int k = 0; k <= n; ++k) {
    const double xi = static_cast<double>(k) / n;
    xf[k] = (stretch == 0.0) ? L * xi
                             : 0.5 * L * (1.0 + std::tanh(stretch * (xi - 0.5)) / std::tanh(0.5 * stretch));
  }
  for (int i = 0; i < n; ++i) dxf[i] = xf[i + 1] - xf[i];
  // centres are face midpoints; centre spacing i is between cells i-1 and i
  for (int i = 1; i < n; ++i) {
    const double c_lo = 0.5 * (xf[i - 1] + xf[i]);
    const double c_hi = 0.5 * (xf[i] + xf[i + 1]);
    dxc[i] = c_hi - c_lo;
  }
  dxc[0] = dxc[n] = 0.5 * (dxf[0] + dxf[n - 1]);
  return TPT_OK;
}

int build_dir(int n, const double* dxf, const double* dxc, const int bc[2], Dir1D* out) {
  if (n < 1 || !dxf || !dxc) return TPT_ERR_INVALID_ARG;
  for (int e = 0; e < 2; ++e)
    if (bc[e] < TPT_BC_PERIODIC || bc[e] > TPT_BC_NONE) return TPT_ERR_INVALID_ARG;
  if ((bc[0] == TPT_BC_PERIODIC) != (bc[1] == TPT_BC_PERIODIC)) return TPT_ERR_INVALID_ARG;
  if ((bc[0] == TPT_BC_NONE) != (bc[1] == TPT_BC_NONE)) return TPT_ERR_INVALID_ARG;
  Dir1D& d = *out;
  d.n = n;
  d.bc[0] = bc[0];
  d.bc[1] = bc[1];
  d.periodic = bc[0] == TPT_BC_PERIODIC;
  d.dxf.assign(dxf, dxf + n);
  d.dxc.assign(dxc, dxc + n + 1);
  for (int i = 0; i < n; ++i)
    if (!(dxf[i] > 0.0) || !std::isfinite(dxf[i])) return TPT_ERR_INVALID_ARG;
  d.a.assign(n, 0.0);
  d.b.assign(n, 0.0);
  d.c.assign(n, 0.0);
  if (bc[0] == TPT_BC_NONE) {   // not in the operator: zero rows, spacings only for volumes
    d.uniform = false;
    return TPT_OK;
  }
  // centre spacings in use: interior ones, plus the ends of a periodic
  // direction or of a node-Dirichlet wall
  const int c0 = (d.periodic || bc[0] == TPT_BC_DIRICHLET_NODE) ? 0 : 1;
  const int c1 = (d.periodic || bc[1] == TPT_BC_DIRICHLET_NODE) ? n : n - 1;
  for (int i = c0; i <= c1; ++i)
    if (!(dxc[i] > 0.0) || !std::isfinite(dxc[i])) return TPT_ERR_INVALID_ARG;
  std::vector<double> wall(n, 0.0);
  for (int i = 0; i < n; ++i) {
    d.a[i] = 1.0 / (dxf[i] * dxc[i]);       // 1/(dx_i dx_{i-1/2})
    d.c[i] = 1.0 / (dxf[i] * dxc[i + 1]);   // 1/(dx_i dx_{i+1/2})
  }
  if (!d.periodic) {
    if (bc[0] == TPT_BC_DIRICHLET) wall[0] += 2.0 / (dxf[0] * dxf[0]);
    if (bc[1] == TPT_BC_DIRICHLET) wall[n - 1] += 2.0 / (dxf[n - 1] * dxf[n - 1]);
    if (bc[0] == TPT_BC_DIRICHLET_NODE) wall[0] += d.a[0];        // zero value at the node below
    if (bc[1] == TPT_BC_DIRICHLET_NODE) wall[n - 1] += d.c[n - 1];
    d.a[0] = 0.0;
    d.c[n - 1] = 0.0;
  }
  for (int i = 0; i < n; ++i) d.b[i] = -((d.a[i] + d.c[i]) + wall[i]);
  // a direction is uniform when every width and every used centre spacing
  // equals dx_0 to a relative 1e-12
  bool uni = true;
  for (int i = 0; i < n && uni; ++i) uni = std::fabs(dxf[i] - dxf[0]) <= 1e-12 * dxf[0];
  for (int i = c0; i <= c1 && uni; ++i) uni = std::fabs(dxc[i] - dxf[0]) <= 1e-12 * dxf[0];
  d.uniform = uni;
  return TPT_OK;
}

namespace {

// Implicit QL iteration with Wilkinson-type shifts on a symmetric tridiagonal
// matrix (diagonal dd[0..n-1], off-diagonal ee[i] coupling i and i+1), with the
// rotations accumulated into the column-major n x n matrix z (starts as I).
// This is the classic public-domain algorithm of EISPACK's imtql2 (Bowdler,
// Martin, Reinsch and Wilkinson, 1968), in its common textbook form; the
// steps and the scalar names (g, r, s, c, p, f, b) follow that published
// listing.
bool ql_implicit(int n, std::vector<double>& dd, std::vector<double>& ee, std::vector<double>& z) {
  ee.resize(n);
  ee[n - 1] = 0.0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      int m = l;
      for (; m < n - 1; ++m) {
        const double scale = std::fabs(dd[m]) + std::fabs(dd[m + 1]);
        if (std::fabs(ee[m]) <= DBL_EPSILON * scale) break;
      }
      if (m == l) break;
      if (++iter > 200) return false;
      double g = (dd[l + 1] - dd[l]) / (2.0 * ee[l]);
      double r = std::hypot(g, 1.0);
      g = dd[m] - dd[l] + ee[l] / (g + std::copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      bool deflated = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = s * ee[i], b = c * ee[i];
        r = std::hypot(f, g);
        ee[i + 1] = r;
        if (r == 0.0) {
          dd[i + 1] -= p;
          ee[m] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = dd[i + 1] - p;
        r = (dd[i] - g) * s + 2.0 * c * b;
        p = s * r;
        dd[i + 1] = g + p;
        g = c * r - b;
        double* zi = &z[static_cast<size_t>(i) * n];
        double* zj = &z[static_cast<size_t>(i + 1) * n];
        for (int k = 0; k < n; ++k) {
          const double t = zj[k];
          zj[k] = s * zi[k] + c * t;
          zi[k] = c * zi[k] - s * t;
        }
      }
      if (deflated) continue;
      dd[l] -= p;
      ee[l] = g;
      ee[m] = 0.0;
    }
  }
  return true;
}

// Cyclic Jacobi eigensolver for a dense symmetric matrix a (column-major,
// destroyed); eigenvectors into v (column-major), eigenvalues into lam.
bool jacobi_dense(int n, std::vector<double>& a, std::vector<double>& v, std::vector<double>& lam) {
  v.assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) v[static_cast<size_t>(i) * n + i] = 1.0;
  auto A = [&](int r, int c) -> double& { return a[static_cast<size_t>(c) * n + r]; };
  double norm2 = 0.0;
  for (double x : a) norm2 += x * x;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int q = 0; q < n; ++q)
      for (int p = 0; p < q; ++p) off += A(p, q) * A(p, q);
    if (off <= 1e-31 * norm2) break;
    if (sweep == 99) return false;
    for (int q = 1; q < n; ++q) {
      for (int p = 0; p < q; ++p) {
        const double apq = A(p, q);
        if (std::fabs(apq) <= 1e-18 * std::sqrt(norm2)) continue;
        const double theta = (A(q, q) - A(p, p)) / (2.0 * apq);
        const double t = std::copysign(1.0, theta) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q
          const double akp = A(k, p), akq = A(k, q);
          A(k, p) = c * akp - s * akq;
          A(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          const double apk = A(p, k), aqk = A(q, k);
          A(p, k) = c * apk - s * aqk;
          A(q, k) = s * apk + c * aqk;
        }
        double* vp = &v[static_cast<size_t>(p) * n];
        double* vq = &v[static_cast<size_t>(q) * n];
        for (int k = 0; k < n; ++k) {
          const double x = vp[k], y = vq[k];
          vp[k] = c * x - s * y;
          vq[k] = s * x + c * y;
        }
      }
    }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A(i, i);
  return true;
}

// Rayleigh quotient of the generalised pair (S, D), S = D T symmetric, for
// v = D^{-1/2} q, evaluated in long double in the energy form
//   v^T S v = sum_i rowsum_i v_i^2 - sum_{couplings i<j} S_ij (v_i - v_j)^2,
// so that the smallest eigenvalues keep relative accuracy.
double rayleigh(const Dir1D& d, const double* q) {
  typedef long double ld;
  const int n = d.n;
  std::vector<ld> v(n);
  for (int i = 0; i < n; ++i) v[i] = static_cast<ld>(q[i]) / std::sqrt(static_cast<ld>(d.dxf[i]));
  // symmetric couplings between i and i+1 (and the wrap pair when periodic)
  auto coupling = [&](int i, int j) -> ld {  // j = i+1 mod n
    const ld sij = static_cast<ld>(d.dxf[i]) * static_cast<ld>(d.c[i]);
    const ld sji = static_cast<ld>(d.dxf[j]) * static_cast<ld>(d.a[j]);
    return 0.5L * (sij + sji);
  };
  ld num = 0.0L, den = 0.0L;
  std::vector<ld> rowsum(n, 0.0L);
  const int ncpl = d.periodic ? n : n - 1;
  for (int i = 0; i < n; ++i) rowsum[i] = static_cast<ld>(d.dxf[i]) * static_cast<ld>(d.b[i]);
  for (int i = 0; i < ncpl && n > 1; ++i) {
    const int j = (i + 1) % n;
    const ld s = coupling(i, j);
    rowsum[i] += s;
    rowsum[j] += s;
    const ld dv = v[i] - v[j];
    num -= s * dv * dv;
  }
  for (int i = 0; i < n; ++i) {
    num += rowsum[i] * v[i] * v[i];
    den += static_cast<ld>(d.dxf[i]) * v[i] * v[i];
  }
  return static_cast<double>(num / den);
}

}  // namespace

int eigen_dir(const Dir1D& d, Eigen1D* out) {
  const int n = d.n;
  if (d.excluded()) {   // identity eigenbasis, zero eigenvalues: no transform along d
    out->lam.assign(n, 0.0);
    out->qt.assign(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i) out->qt[static_cast<size_t>(i) * n + i] = 1.0;
    out->null_mode = -1;
    return TPT_OK;
  }
  std::vector<double> s(n);
  for (int i = 0; i < n; ++i) s[i] = std::sqrt(d.dxf[i]);
  std::vector<double> lam, vec;
  if (n == 1) {
    const double t = d.periodic ? d.a[0] + d.b[0] + d.c[0] : d.b[0];
    lam.assign(1, t);
    vec.assign(1, 1.0);
  } else if (!d.periodic) {
    // step 1.1: T~ = D^{1/2} T D^{-1/2}; off-diagonal (i, i+1) = sqrt(dx_i/dx_{i+1}) c_i
    std::vector<double> dd(d.b), ee(n, 0.0);
    for (int i = 0; i < n - 1; ++i) ee[i] = std::sqrt(d.dxf[i] / d.dxf[i + 1]) * d.c[i];
    vec.assign(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i) vec[static_cast<size_t>(i) * n + i] = 1.0;
    if (!ql_implicit(n, dd, ee, vec)) return TPT_ERR_NUMERICAL;   // step 1.2
    lam = dd;
  } else {
    // cyclic operator: dense symmetric T~ with the corner couplings
    std::vector<double> a(static_cast<size_t>(n) * n, 0.0);
    auto A = [&](int r, int c) -> double& { return a[static_cast<size_t>(c) * n + r]; };
    for (int i = 0; i < n; ++i) A(i, i) += d.b[i];
    for (int i = 0; i < n; ++i) {
      const int j = (i + 1) % n;
      const double e = std::sqrt(d.dxf[i] / d.dxf[j]) * d.c[i];
      A(i, j) += e;
      A(j, i) += e;
    }
    if (!jacobi_dense(n, a, vec, lam)) return TPT_ERR_NUMERICAL;
  }
  // refine every eigenvalue (Rayleigh quotient in long double), then sort the
  // modes by decreasing refined eigenvalue, so a null mode comes first
  std::vector<double> ref(n);
  for (int p = 0; p < n; ++p) ref[p] = rayleigh(d, &vec[static_cast<size_t>(p) * n]);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ref[x] > ref[y]; });
  out->lam.resize(n);
  out->qt.resize(static_cast<size_t>(n) * n);
  for (int p = 0; p < n; ++p) {
    const double* src = &vec[static_cast<size_t>(order[p]) * n];
    std::copy(src, src + n, &out->qt[static_cast<size_t>(p) * n]);
    out->lam[p] = ref[order[p]];
  }
  out->null_mode = -1;
  if (d.has_null()) {
    out->null_mode = 0;
    out->lam[0] = 0.0;
  }
  for (int p = 0; p < n; ++p)
    if (!std::isfinite(out->lam[p])) return TPT_ERR_NUMERICAL;
  return TPT_OK;
}

bool fft_supported(const Dir1D& d) {
  if (d.excluded()) return false;
  const int n = d.n;
  const bool pow2 = n >= 1 && (n & (n - 1)) == 0;
  const bool bcs = d.periodic || (d.bc[0] == TPT_BC_NEUMANN && d.bc[1] == TPT_BC_NEUMANN);
  return pow2 && d.uniform && bcs;
}

int fft_dir(const Dir1D& d, Eigen1D* out, int* kind) {
  if (!fft_supported(d)) return TPT_ERR_UNSUPPORTED;
  const int n = d.n;
  *kind = d.periodic ? 0 : 1;
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<double> v(n);
  out->lam.assign(n, 0.0);
  out->qt.clear();
  for (int p = 0; p < n; ++p) {
    for (int i = 0; i < n; ++i) {
      long double x;
      if (*kind == 1) {
        x = std::cos(pi * p * (2.0L * i + 1.0L) / (2.0L * n));
      } else if (p == 0) {
        x = 1.0L;
      } else if (p == n - 1) {
        x = (i % 2 == 0) ? 1.0L : -1.0L;
      } else {
        const int k = (p + 1) / 2;
        const long double arg = 2.0L * pi * i * k / n;
        x = (p % 2 == 1) ? std::cos(arg) : std::sin(arg);
      }
      v[i] = static_cast<double>(x);
    }
    // the Rayleigh quotient takes D^{1/2} v; on a uniform grid that is a constant factor
    out->lam[p] = (p == 0) ? 0.0 : rayleigh(d, v.data());
  }
  out->null_mode = 0;
  return TPT_OK;
}

}  // namespace tpt
