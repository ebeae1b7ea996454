// Pressure projection of a staggered velocity field (Sec. 2.1: the
// pressure-correction Poisson equation Eq. poi_ns and the velocity correction
// that follows it).  Declarations and contracts: include/tpt.h.
//
//   D u* / g  (div_kernel)  ->  L Phi = rhs (tpt_solve)  ->  u -= g G Phi (grad_kernel)
//
// Both kernels stream float64 fields once with coalesced accesses along x;
// the divergence uses the plan's reciprocal cell widths and the gradient its
// reciprocal centre spacings, so no division runs on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "tpt_internal.h"

namespace {

int cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return TPT_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TPT_ERR_OOM : TPT_ERR_CUDA;
}

// Per-call coefficient tables with g folded in: tab[d][i] = (1/dx_i) / g for
// the divergence (n entries) and tab[3+d][f] = -g / dx_{f-1/2} for the
// gradient (n + 1 entries), so each cell and face costs one float64 multiply
// or fused multiply-add less.
__global__ void coef_kernel(int n, const double* __restrict__ ixf, const double* __restrict__ ixc, double g,
                            double* __restrict__ div_tab, double* __restrict__ grad_tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) div_tab[i] = ixf[i] / g;
  if (i <= n) grad_tab[i] = -g * ixc[i];
}

// rhs = (D u) / g on every cell; block 128 along x, grid (x, y, z)
__global__ void __launch_bounds__(128)
div_kernel(int nx, int ny, const double* __restrict__ u, const double* __restrict__ v,
           const double* __restrict__ w, const double* __restrict__ ix, const double* __restrict__ iy,
           const double* __restrict__ iz, double* __restrict__ rhs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= nx) return;
  const long long ou = i + static_cast<long long>(nx + 1) * (j + static_cast<long long>(ny) * k);
  const long long ov = i + static_cast<long long>(nx) * (j + static_cast<long long>(ny + 1) * k);
  const long long ow = i + static_cast<long long>(nx) * (j + static_cast<long long>(ny) * k);
  const long long sz = static_cast<long long>(nx) * ny;
  double d = (u[ou + 1] - u[ou]) * ix[i];
  d = fma(v[ov + nx] - v[ov], iy[j], d);
  rhs[ow] = fma(w[ow + sz] - w[ow], iz[k], d);
}

// vel -= g G Phi on the faces of direction DIR: interior faces, and the shared
// boundary face of a periodic direction (written at both ends).  Block 128
// along x of the velocity's own shape, grid (x, y, z) over it.
template <int DIR>
__global__ void __launch_bounds__(128)
grad_kernel(int nx, int ny, int nz, int periodic, const double* __restrict__ phi, const double* __restrict__ cg,
            double* __restrict__ vel) {
  const int sx = nx + (DIR == 0), sy = ny + (DIR == 1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= sx) return;
  const int f = (DIR == 0) ? i : (DIR == 1 ? j : k);
  const int nn = (DIR == 0) ? nx : (DIR == 1 ? ny : nz);
  int lo = f - 1, hi = f;   // cells on both sides of the face
  if (f == 0 || f == nn) {
    if (!periodic) return;  // wall face: no penetration, value kept
    lo = nn - 1;
    hi = 0;
  }
  const long long step = (DIR == 0) ? 1 : (DIR == 1 ? nx : static_cast<long long>(nx) * ny);
  const long long base = (DIR == 0 ? 0 : i) + (DIR == 1 ? 0 : static_cast<long long>(j) * nx) +
                         (DIR == 2 ? 0 : static_cast<long long>(k) * nx * ny);
  const double dp = phi[base + hi * step] - phi[base + lo * step];
  const long long o = i + static_cast<long long>(sx) * (j + static_cast<long long>(sy) * k);
  vel[o] = fma(cg[f], dp, vel[o]);
}

}  // namespace

extern "C" {

size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

// Workspace: rhs field | coefficient tables (6 x (n + 1) doubles) | solve workspace.
size_t tables_bytes(const tpt_plan_s* p) {
  return align256(6 * sizeof(double) * (1 + std::max(p->n[0], std::max(p->n[1], p->n[2]))));
}

int tpt_project_workspace_bytes(tpt_plan p, size_t* bytes) {
  if (!p || !bytes) return TPT_ERR_INVALID_ARG;
  size_t ws = 0;
  const int st = tpt_workspace_bytes(p, &ws);
  if (st != TPT_OK) return st;
  *bytes = align256(tpt::npts(p) * sizeof(double)) + tables_bytes(p) + ws;
  return TPT_OK;
}

int tpt_project(tpt_plan p, double* u, double* v, double* w, double gamma_dt, double* phi, void* work,
                void* stream, tpt_info* info) {
  if (!p || p->dev < 0 || !p->d_scal || !u || !v || !w || !phi || !work) return TPT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0 || !(gamma_dt > 0.0)) return TPT_ERR_INVALID_ARG;
  if (p->alpha != 0.0 || p->beta != 1.0) return TPT_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (p->dir[d].bc[0] == TPT_BC_DIRICHLET || p->dir[d].bc[1] == TPT_BC_DIRICHLET) return TPT_ERR_UNSUPPORTED;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int nmax = 1 + std::max(nx, std::max(ny, nz));
  double* rhs = static_cast<double*>(work);
  double* tab = reinterpret_cast<double*>(static_cast<char*>(work) + align256(tpt::npts(p) * sizeof(double)));
  char* solve_work = reinterpret_cast<char*>(tab) + tables_bytes(p);
  int st = TPT_OK;
  for (int d = 0; d < 3 && st == TPT_OK; ++d) {
    tpt::note_launch(1);
    coef_kernel<<<(p->n[d] + 1 + 127) / 128, 128, 0, s>>>(p->n[d], p->d_inv_dxf[d], p->d_inv_dxc[d], gamma_dt,
                                                          tab + d * nmax, tab + (3 + d) * nmax);
    st = cuda_st(cudaGetLastError());
  }
  if (st == TPT_OK) {
    dim3 grid((nx + 127) / 128, ny, nz);
    tpt::note_launch(1);
    div_kernel<<<grid, 128, 0, s>>>(nx, ny, u, v, w, tab, tab + nmax, tab + 2 * nmax, rhs);
    st = cuda_st(cudaGetLastError());
  }
  bool converged = true;
  if (st == TPT_OK) {
    st = tpt_solve(p, rhs, phi, solve_work, stream, info);
    if (st == TPT_ERR_NOT_CONVERGED) {   // Phi holds the last iterate: correct with it, then report
      converged = false;
      st = TPT_OK;
    }
  }
  double* vel[3] = {u, v, w};
  for (int d = 0; d < 3 && st == TPT_OK; ++d) {
    const int per = p->dir[d].periodic ? 1 : 0;
    const double* cg = tab + (3 + d) * nmax;
    dim3 grid((nx + (d == 0) + 127) / 128, ny + (d == 1), nz + (d == 2));
    tpt::note_launch(1);
    if (d == 0) grad_kernel<0><<<grid, 128, 0, s>>>(nx, ny, nz, per, phi, cg, vel[d]);
    else if (d == 1) grad_kernel<1><<<grid, 128, 0, s>>>(nx, ny, nz, per, phi, cg, vel[d]);
    else grad_kernel<2><<<grid, 128, 0, s>>>(nx, ny, nz, per, phi, cg, vel[d]);
    st = cuda_st(cudaGetLastError());
  }
  if (prev >= 0) cudaSetDevice(prev);
  return (st == TPT_OK && !converged) ? TPT_ERR_NOT_CONVERGED : st;
}

}  // extern "C"
