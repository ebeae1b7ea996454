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

#include <cstdint>

#include "tpt_internal.h"

namespace {

int cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return TPT_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TPT_ERR_OOM : TPT_ERR_CUDA;
}

// rhs = (D u) / g on every cell; block (128, 1, 1) along x, grid (x, y, z)
__global__ void __launch_bounds__(128)
div_kernel(int nx, int ny, int nz, const double* __restrict__ u, const double* __restrict__ v,
           const double* __restrict__ w, const double* __restrict__ ix, const double* __restrict__ iy,
           const double* __restrict__ iz, double inv_g, double* __restrict__ rhs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= nx) return;
  const long long ou = i + static_cast<long long>(nx + 1) * (j + static_cast<long long>(ny) * k);
  const long long ov = i + static_cast<long long>(nx) * (j + static_cast<long long>(ny + 1) * k);
  const long long ow = i + static_cast<long long>(nx) * (j + static_cast<long long>(ny) * k);
  const long long sz = static_cast<long long>(nx) * ny;
  double d = (u[ou + 1] - u[ou]) * ix[i];
  d = fma(v[ov + nx] - v[ov], iy[j], d);
  d = fma(w[ow + sz] - w[ow], iz[k], d);
  rhs[ow] = d * inv_g;
}

// u -= g G Phi on the faces of direction `dir`: interior faces, and the
// shared boundary face of a periodic direction (written at both ends).
// Face (f, a, b) of the direction, f = 0..n, a/b the other two indices.
__global__ void __launch_bounds__(128)
grad_kernel(int dir, int nx, int ny, int nz, int periodic, const double* __restrict__ phi,
            const double* __restrict__ ic, double g, double* __restrict__ vel) {
  const int n[3] = {nx, ny, nz};
  const int ext = n[dir] + 1;   // faces along dir
  // thread index over the face array, x fastest in the velocity's own shape
  const long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  const int sx = (dir == 0) ? ext : nx, sy = (dir == 1) ? ext : ny, szz = (dir == 2) ? ext : nz;
  const long long total = static_cast<long long>(sx) * sy * szz;
  if (t >= total) return;
  const int i = static_cast<int>(t % sx);
  const int j = static_cast<int>((t / sx) % sy);
  const int k = static_cast<int>(t / (static_cast<long long>(sx) * sy));
  const int f = (dir == 0) ? i : (dir == 1 ? j : k);
  const int nn = n[dir];
  int lo = f - 1, hi = f;   // cells on both sides of the face
  if (f == 0 || f == nn) {
    if (!periodic) return;   // wall face: no penetration, value kept
    lo = nn - 1;
    hi = 0;
  }
  const long long s[3] = {1, static_cast<long long>(nx), static_cast<long long>(nx) * ny};
  const long long base = (dir == 0 ? 0 : i) + (dir == 1 ? 0 : static_cast<long long>(j) * nx) +
                         (dir == 2 ? 0 : static_cast<long long>(k) * nx * ny);
  const double dp = phi[base + hi * s[dir]] - phi[base + lo * s[dir]];
  vel[t] = fma(-g * ic[f], dp, vel[t]);
}

}  // namespace

extern "C" {

int tpt_project_workspace_bytes(tpt_plan p, size_t* bytes) {
  if (!p || !bytes) return TPT_ERR_INVALID_ARG;
  size_t ws = 0;
  const int st = tpt_workspace_bytes(p, &ws);
  if (st != TPT_OK) return st;
  *bytes = ((tpt::npts(p) * sizeof(double) + 255) & ~static_cast<size_t>(255)) + ws;
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
  double* rhs = static_cast<double*>(work);
  char* solve_work = static_cast<char*>(work) + ((tpt::npts(p) * sizeof(double) + 255) & ~static_cast<size_t>(255));
  int st = TPT_OK;
  {
    dim3 grid((nx + 127) / 128, ny, nz);
    tpt::note_launch(1);
    div_kernel<<<grid, 128, 0, s>>>(nx, ny, nz, u, v, w, p->d_inv_dxf[0], p->d_inv_dxf[1], p->d_inv_dxf[2],
                                    1.0 / gamma_dt, rhs);
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
    const long long faces = static_cast<long long>(nx + (d == 0)) * (ny + (d == 1)) * (nz + (d == 2));
    tpt::note_launch(1);
    grad_kernel<<<static_cast<unsigned>((faces + 127) / 128), 128, 0, s>>>(
        d, nx, ny, nz, p->dir[d].periodic ? 1 : 0, phi, p->d_inv_dxc[d], gamma_dt, vel[d]);
    st = cuda_st(cudaGetLastError());
  }
  if (prev >= 0) cudaSetDevice(prev);
  return (st == TPT_OK && !converged) ? TPT_ERR_NOT_CONVERGED : st;
}

}  // extern "C"
