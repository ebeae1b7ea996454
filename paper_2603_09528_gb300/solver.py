"""Python face of the C ABI: a Plan object over torch device memory and streams.

Fields are float64 in Fortran order (Nx, Ny, Nz), x fastest.  On the torch side
a field is a contiguous float64 CUDA tensor with Nx*Ny*Nz elements (any shape;
``field_to_device`` / ``field_to_host`` convert from/to numpy (Nx, Ny, Nz)
arrays).  This module only marshals arguments: every computation runs in
libtpt.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check, lib

AUTO, GEMM, FFT = _lib.TPT_XFORM_AUTO, _lib.TPT_XFORM_GEMM, _lib.TPT_XFORM_FFT
PERIODIC, NEUMANN, DIRICHLET = _lib.TPT_BC_PERIODIC, _lib.TPT_BC_NEUMANN, _lib.TPT_BC_DIRICHLET
DIRICHLET_NODE, NONE = _lib.TPT_BC_DIRICHLET_NODE, _lib.TPT_BC_NONE
FP64 = _lib.TPT_PREC_FP64
MIXED_BF16, MIXED_BF16X3, MIXED_TF32 = (_lib.TPT_PREC_MIXED_BF16, _lib.TPT_PREC_MIXED_BF16X3,
                                        _lib.TPT_PREC_MIXED_TF32)
_BC = {"periodic": PERIODIC, "neumann": NEUMANN, "dirichlet": DIRICHLET, "dirichlet_node": DIRICHLET_NODE,
       "none": NONE}


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def grid_tanh(n: int, L: float = 1.0, stretch: float = 0.0):
    """tpt_grid_tanh: (dxf, dxc) of Eq. (tanh_stretching) as float64 numpy arrays."""
    dxf = np.empty(n)
    dxc = np.empty(n + 1)
    check(lib.tpt_grid_tanh(n, L, stretch, dxf.ctypes.data_as(_lib._dp),
                            dxc.ctypes.data_as(_lib._dp)), "tpt_grid_tanh")
    return dxf, dxc


def grid_faces(dxf, dxc, periodic: bool):
    """tpt_grid_faces: (widths, centre spacings) of the face-centred unknowns."""
    dxf = np.ascontiguousarray(dxf, dtype=np.float64)
    dxc = np.ascontiguousarray(dxc, dtype=np.float64)
    n = dxf.size
    wf, sc = np.empty(n), np.empty(n + 1)
    m = C.c_int()
    check(lib.tpt_grid_faces(n, dxf.ctypes.data_as(_lib._dp), dxc.ctypes.data_as(_lib._dp), int(bool(periodic)),
                             C.byref(m), wf.ctypes.data_as(_lib._dp), sc.ctypes.data_as(_lib._dp)),
          "tpt_grid_faces")
    return wf[:m.value].copy(), sc[:m.value + 1].copy()


def field_to_device(f: np.ndarray, device="cuda") -> torch.Tensor:
    """numpy (Nx, Ny, Nz) -> flat contiguous float64 tensor in Fortran order."""
    flat = np.asarray(f, dtype=np.float64).ravel(order="F")
    return torch.from_numpy(np.ascontiguousarray(flat)).to(device)


def field_to_host(t: torch.Tensor, n) -> np.ndarray:
    return t.detach().cpu().numpy().reshape(tuple(n), order="F")


def make_desc(n, dxf, dxc, bc, xform=(AUTO, AUTO), alpha=0.0, beta=1.0, precision=FP64, rtol=0.0,
              max_refine=1, desc=None):
    """Fill a tpt_desc; returns (desc, arrays that must stay alive until the
    plan is created)."""
    desc = _lib.tpt_desc() if desc is None else desc
    keep = []
    for a in range(3):
        f = np.ascontiguousarray(dxf[a], dtype=np.float64)
        c = np.ascontiguousarray(dxc[a], dtype=np.float64)
        keep += [f, c]
        desc.n[a] = int(n[a])
        desc.dxf[a] = f.ctypes.data_as(_lib._dp)
        desc.dxc[a] = c.ctypes.data_as(_lib._dp)
        lo, hi = bc[a]
        desc.bc[a][0] = _BC.get(lo, lo) if isinstance(lo, str) else int(lo)
        desc.bc[a][1] = _BC.get(hi, hi) if isinstance(hi, str) else int(hi)
    desc.xform[0], desc.xform[1] = int(xform[0]), int(xform[1])
    desc.alpha, desc.beta = float(alpha), float(beta)
    desc.precision = int(precision)
    desc.rtol = float(rtol)
    desc.max_refine = int(max_refine)
    return desc, keep


def _info_dict(info, status):
    return dict(iters=info.iters, rel_residual=info.rel_residual, compat_defect=info.compat_defect,
                status=status, ms_stage=[float(x) for x in info.ms_stage])


class Plan:
    """tpt_plan_create / tpt_solve / tpt_plan_destroy on one CUDA device."""

    def __init__(self, n, dxf, dxc, bc, xform=(AUTO, AUTO), alpha=0.0, beta=1.0,
                 precision=FP64, rtol=0.0, max_refine=1, device: int = 0, cache: "Cache" = None):
        desc, keep = make_desc(n, dxf, dxc, bc, xform, alpha, beta, precision, rtol, max_refine)
        h = C.c_void_p()
        if cache is not None:
            self.device = cache.device
            check(lib.tpt_plan_create_cached(C.byref(desc), cache._h, C.byref(h)), "tpt_plan_create_cached")
            self._cache = cache          # the cache outlives its plans
        else:
            self.device = int(device)
            check(lib.tpt_plan_create(C.byref(desc), self.device, C.byref(h)), "tpt_plan_create")
        del keep
        self._owned = True
        self._attach(h, n)

    @classmethod
    def borrowed(cls, handle: C.c_void_p, n, device: int) -> "Plan":
        """View of a plan owned elsewhere (a batch instance); never destroyed here."""
        obj = cls.__new__(cls)
        obj.device = int(device)
        obj._owned = False
        obj._attach(handle, n)
        return obj

    def _attach(self, h, n):
        self._h = h
        self.n = tuple(int(v) for v in n)
        nb = C.c_size_t()
        check(lib.tpt_workspace_bytes(self._h, C.byref(nb)), "tpt_workspace_bytes")
        self.workspace_bytes = int(nb.value)
        self.npts = self.n[0] * self.n[1] * self.n[2]

    # ------------------------------------------------------------------
    def new_workspace(self) -> torch.Tensor:
        return torch.empty(self.workspace_bytes, dtype=torch.uint8, device="cuda:%d" % self.device)

    def new_field(self) -> torch.Tensor:
        return torch.empty(self.npts, dtype=torch.float64, device="cuda:%d" % self.device)

    def solve(self, f: torch.Tensor, phi: torch.Tensor = None, work: torch.Tensor = None,
              stream=None, want_info: bool = True, raise_not_converged: bool = True):
        """tpt_solve.  Returns (phi, info dict or None); info is read after a
        stream synchronisation when the plan runs a fixed number of steps."""
        phi = self.new_field() if phi is None else phi
        work = self.new_workspace() if work is None else work
        info = _lib.tpt_info() if want_info else None
        st = lib.tpt_solve(self._h, _ptr(f), _ptr(phi), _ptr(work), _stream(stream),
                           C.byref(info) if info is not None else None)
        if st == _lib.TPT_ERR_NOT_CONVERGED and not raise_not_converged:
            pass
        else:
            check(st, "tpt_solve")
        if info is None:
            return phi, None
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return phi, dict(iters=info.iters, rel_residual=info.rel_residual,
                         compat_defect=info.compat_defect, status=st,
                         ms_stage=[float(x) for x in info.ms_stage])

    def project_workspace(self) -> torch.Tensor:
        nb = C.c_size_t()
        check(lib.tpt_project_workspace_bytes(self._h, C.byref(nb)), "tpt_project_workspace_bytes")
        return torch.empty(int(nb.value), dtype=torch.uint8, device="cuda:%d" % self.device)

    def project(self, u: torch.Tensor, v: torch.Tensor, w: torch.Tensor, gamma_dt: float,
                phi: torch.Tensor = None, work: torch.Tensor = None, stream=None,
                raise_not_converged: bool = True):
        """tpt_project: u, v, w (face velocities, flat float64 CUDA tensors of
        (Nx+1)NyNz, Nx(Ny+1)Nz, NxNy(Nz+1) values) are corrected in place;
        returns (phi, info dict)."""
        phi = self.new_field() if phi is None else phi
        work = self.project_workspace() if work is None else work
        info = _lib.tpt_info()
        st = lib.tpt_project(self._h, _ptr(u), _ptr(v), _ptr(w), float(gamma_dt), _ptr(phi), _ptr(work),
                             _stream(stream), C.byref(info))
        if not (st == _lib.TPT_ERR_NOT_CONVERGED and not raise_not_converged):
            check(st, "tpt_project")
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return phi, _info_dict(info, st)

    def set_stage_timing(self, enable: bool):
        check(lib.tpt_set_stage_timing(self._h, int(bool(enable))), "tpt_set_stage_timing")

    def solve_host(self, f_host: torch.Tensor, phi_host: torch.Tensor, f_dev: torch.Tensor,
                   phi_dev: torch.Tensor, work: torch.Tensor, stream=None):
        info = _lib.tpt_info()
        st = lib.tpt_solve_host(self._h, _ptr(f_host), _ptr(phi_host), _ptr(f_dev), _ptr(phi_dev),
                                _ptr(work), _stream(stream), C.byref(info))
        check(st, "tpt_solve_host")
        return dict(iters=info.iters, rel_residual=info.rel_residual,
                    compat_defect=info.compat_defect)

    def set_refinement(self, rtol: float, max_refine: int):
        check(lib.tpt_set_refinement(self._h, float(rtol), int(max_refine)), "tpt_set_refinement")

    def set_coefficients(self, alpha: float, beta: float):
        check(lib.tpt_set_coefficients(self._h, float(alpha), float(beta)), "tpt_set_coefficients")

    # ------------------------------------------------------------ single steps
    def transform(self, x: torch.Tensor, direction: int, inverse: bool, out=None, stream=None):
        out = self.new_field() if out is None else out
        check(lib.tpt_transform(self._h, int(direction), int(bool(inverse)), _ptr(x), _ptr(out),
                                _stream(stream)), "tpt_transform")
        return out

    def thomas(self, fhat: torch.Tensor, out=None, scratch=None, stream=None):
        out = self.new_field() if out is None else out
        scratch = self.new_field() if scratch is None else scratch
        check(lib.tpt_thomas(self._h, _ptr(fhat), _ptr(out), _ptr(scratch), _stream(stream)),
              "tpt_thomas")
        return out

    def residual(self, f: torch.Tensor, phi: torch.Tensor, out=None, sums=None, stream=None):
        out = self.new_field() if out is None else out
        check(lib.tpt_residual(self._h, _ptr(f), _ptr(phi), _ptr(out), _ptr(sums), _stream(stream)),
              "tpt_residual")
        return out

    def eigenvalues(self, direction: int) -> np.ndarray:
        lam = np.empty(self.n[direction])
        check(lib.tpt_plan_eigenvalues(self._h, int(direction), lam.ctypes.data_as(_lib._dp)),
              "tpt_plan_eigenvalues")
        return lam

    def transforms(self):
        x = (C.c_int * 2)()
        check(lib.tpt_plan_transforms(self._h, x), "tpt_plan_transforms")
        return int(x[0]), int(x[1])

    def rows(self, direction: int):
        m = self.n[direction]
        a, b, c = np.empty(m), np.empty(m), np.empty(m)
        check(lib.tpt_plan_rows(self._h, int(direction), a.ctypes.data_as(_lib._dp),
                                b.ctypes.data_as(_lib._dp), c.ctypes.data_as(_lib._dp)),
              "tpt_plan_rows")
        return a, b, c

    def autotune(self, work: torch.Tensor = None, stream=None):
        """tpt_plan_autotune: the four transform column-tile widths it keeps."""
        work = self.new_workspace() if work is None else work
        t = (C.c_int * 4)()
        check(lib.tpt_plan_autotune(self._h, _ptr(work), _stream(stream), t), "tpt_plan_autotune")
        return tuple(int(v) for v in t)

    def set_tiles(self, tiles):
        t = (C.c_int * 4)(*[int(v) for v in tiles])
        check(lib.tpt_plan_set_tiles(self._h, t), "tpt_plan_set_tiles")

    def tiles(self):
        t = (C.c_int * 4)()
        check(lib.tpt_plan_get_tiles(self._h, t), "tpt_plan_get_tiles")
        return tuple(int(v) for v in t)

    def set_pairing(self, pairs):
        t = (C.c_int * 4)(*[int(v) for v in pairs])
        check(lib.tpt_plan_set_pairing(self._h, t), "tpt_plan_set_pairing")

    def set_thomas_kernel(self, variant):
        check(lib.tpt_plan_set_thomas_kernel(self._h, int(variant)), "tpt_plan_set_thomas_kernel")

    def set_residual_kernel(self, variant):
        """0 automatic, 1 direct loads, 2 TMA-staged plane tiles (mixed plans)."""
        check(lib.tpt_plan_set_residual_kernel(self._h, int(variant)), "tpt_plan_set_residual_kernel")

    def pairing(self):
        t = (C.c_int * 4)()
        check(lib.tpt_plan_get_pairing(self._h, t), "tpt_plan_get_pairing")
        return tuple(int(v) for v in t)

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                lib.tpt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cache:
    """tpt_cache_*: shared direction eigenbases for plans created through it."""

    def __init__(self, device: int = 0, budget_bytes: int = 1 << 30):
        self.device = int(device)
        h = C.c_void_p()
        check(lib.tpt_cache_create(self.device, int(budget_bytes), C.byref(h)), "tpt_cache_create")
        self._h = h

    def stats(self):
        hits, misses = C.c_ulonglong(), C.c_ulonglong()
        nb, ne = C.c_size_t(), C.c_size_t()
        check(lib.tpt_cache_stats(self._h, C.byref(hits), C.byref(misses), C.byref(nb), C.byref(ne)),
              "tpt_cache_stats")
        return dict(hits=int(hits.value), misses=int(misses.value), device_bytes=int(nb.value),
                    entries=int(ne.value))

    def close(self):
        if getattr(self, "_h", None):
            lib.tpt_cache_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """tpt_server_*: continuous-batching request server on one device.

    ``submit`` takes Plan keyword arguments (n, dxf, dxc, bc, xform, alpha,
    beta, precision, rtol, max_refine) and host tensors for f and phi (pinned
    for full copy bandwidth); the tensors are kept alive until the request
    is waited for.  ``device < 0`` runs the dry-run executor on the host."""

    def __init__(self, device: int = 0, slots: int = 4, setup_threads: int = 4,
                 memory_budget: int = 64 << 30, cache_budget: int = 4 << 30,
                 dry_run_ns_per_point: float = 0.0, merge: int = 8):
        cfg = _lib.tpt_server_config(int(device), int(slots), int(setup_threads), int(memory_budget),
                                     int(cache_budget), float(dry_run_ns_per_point), int(merge))
        h = C.c_void_p()
        check(lib.tpt_server_create(C.byref(cfg), C.byref(h)), "tpt_server_create")
        self._h = h
        self._held = {}

    def submit(self, f_host, phi_host, **spec) -> int:
        desc, keep = make_desc(**spec)
        t = C.c_ulonglong()
        fp = C.c_void_p(f_host.data_ptr() if hasattr(f_host, "data_ptr") else f_host.ctypes.data)
        pp = C.c_void_p(phi_host.data_ptr() if hasattr(phi_host, "data_ptr") else phi_host.ctypes.data)
        check(lib.tpt_server_submit(self._h, C.byref(desc), fp, pp, C.byref(t)), "tpt_server_submit")
        del keep                        # the server copied the descriptor
        self._held[int(t.value)] = (f_host, phi_host)
        return int(t.value)

    def warm(self, **spec):
        """tpt_server_warm: build the eigenbases of spec's x and y directions now."""
        desc, keep = make_desc(**spec)
        check(lib.tpt_server_warm(self._h, C.byref(desc)), "tpt_server_warm")

    def wait(self, ticket: int, timeout: float = -1.0):
        """The request's result dict, or None if it is still running after timeout."""
        r = _lib.tpt_result()
        st = lib.tpt_server_wait(self._h, int(ticket), float(timeout), C.byref(r))
        if st == _lib.TPT_PENDING:
            return None
        check(st, "tpt_server_wait")
        self._held.pop(int(ticket), None)
        return dict(status=int(r.status), iters=r.info.iters, rel_residual=r.info.rel_residual,
                    compat_defect=r.info.compat_defect, t_submit=r.t_submit, t_planned=r.t_planned,
                    t_admit=r.t_admit, t_done=r.t_done, device_bytes=int(r.device_bytes),
                    failed_step=int(r.failed_step), cuda_error=int(r.cuda_error),
                    t_copied=r.t_copied, t_solved=r.t_solved, merged=int(r.merged),
                    cuda_error_name=(lib.tpt_cuda_error_name(int(r.cuda_error)) or b"?").decode())

    def now(self) -> float:
        t = C.c_double()
        check(lib.tpt_server_now(self._h, C.byref(t)), "tpt_server_now")
        return float(t.value)

    def stats(self):
        st = _lib.tpt_serving_stats()
        check(lib.tpt_server_stats(self._h, C.byref(st)), "tpt_server_stats")
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib.tpt_server_destroy(self._h)
            self._h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """tpt_batch_*: independent instances of uneven size solved as one CUDA
    graph.  ``specs`` is a list of dicts of Plan's keyword arguments (n, dxf,
    dxc, bc, xform, alpha, beta, precision, rtol, max_refine)."""

    def __init__(self, specs, nstreams: int = 0, device: int = 0):
        self.device = int(device)
        self.count = len(specs)
        descs = (_lib.tpt_desc * self.count)()
        keep = []
        for i, sp in enumerate(specs):
            _, k = make_desc(desc=descs[i], **sp)
            keep.append(k)
        h = C.c_void_p()
        check(lib.tpt_batch_create(descs, self.count, self.device, int(nstreams), C.byref(h)),
              "tpt_batch_create")
        self._h = h
        del keep
        nb = C.c_size_t()
        check(lib.tpt_batch_workspace_bytes(self._h, C.byref(nb)), "tpt_batch_workspace_bytes")
        self.workspace_bytes = int(nb.value)
        self.plans = []
        for i, sp in enumerate(specs):
            ph = C.c_void_p()
            check(lib.tpt_batch_plan(self._h, i, C.byref(ph)), "tpt_batch_plan")
            self.plans.append(Plan.borrowed(ph, sp["n"], self.device))

    def new_workspace(self) -> torch.Tensor:
        return torch.empty(self.workspace_bytes, dtype=torch.uint8, device="cuda:%d" % self.device)

    @property
    def grouped(self) -> bool:
        v = C.c_int()
        check(lib.tpt_batch_get_grouped(self._h, C.byref(v)), "tpt_batch_get_grouped")
        return bool(v.value)

    def set_grouped(self, on: bool):
        """tpt_batch_set_grouped: grouped launches (True) or capture streams
        (False); the workspace size follows the mode."""
        check(lib.tpt_batch_set_grouped(self._h, int(bool(on))), "tpt_batch_set_grouped")
        nb = C.c_size_t()
        check(lib.tpt_batch_workspace_bytes(self._h, C.byref(nb)), "tpt_batch_workspace_bytes")
        self.workspace_bytes = int(nb.value)

    def autotune(self, work: torch.Tensor, stream=None):
        check(lib.tpt_batch_autotune(self._h, _ptr(work), _stream(stream)), "tpt_batch_autotune")
        return [p.tiles() for p in self.plans]

    def calibrate(self, fs, phis, work: torch.Tensor, rtol: float = 1e-10, max_refine: int = 40,
                  stream=None, spare: int = 1):
        """Size each instance's corrections for capture: one adaptive solve to
        ``rtol`` per instance, then room for the corrections it used plus
        ``spare``.  In the captured batch the stopping test runs on the
        device, so an instance stops as soon as it reaches rtol; a spare
        correction only computes for a right-hand side that needs it (past
        convergence its kernels return at entry, at the cost of their
        launches).  Returns the corrections per instance."""
        used = []
        for p, f, phi in zip(self.plans, fs, phis):
            p.set_refinement(rtol, max_refine)
            _, info = p.solve(f, phi, work, stream=stream, raise_not_converged=False)
            used.append(int(info["iters"]))
            p.set_refinement(rtol, min(max_refine, max(0, used[-1] - 1 + int(spare))))
        return used

    def solve(self, fs, phis, work: torch.Tensor, stream=None, want_info: bool = True,
              raise_errors: bool = True):
        """tpt_batch_solve.  Returns a list of info dicts (with per-instance
        status) after a stream synchronisation, or None when want_info is
        False (the call is then asynchronous)."""
        n = self.count
        fa = (C.c_void_p * n)(*[f.data_ptr() for f in fs])
        pa = (C.c_void_p * n)(*[p.data_ptr() for p in phis])
        infos = (_lib.tpt_info * n)() if want_info else None
        sts = (C.c_int * n)() if want_info else None
        st = lib.tpt_batch_solve(self._h, fa, pa, _ptr(work), _stream(stream), infos, sts)
        if raise_errors and st not in (_lib.TPT_OK, _lib.TPT_ERR_NOT_CONVERGED):
            check(st, "tpt_batch_solve")
        if not want_info:
            return None
        return [_info_dict(infos[i], int(sts[i])) for i in range(n)]

    def launches_per_replay(self) -> int:
        v = C.c_ulonglong()
        check(lib.tpt_batch_launches(self._h, C.byref(v)), "tpt_batch_launches")
        return int(v.value)

    def close(self):
        if getattr(self, "_h", None):
            for p in self.plans:
                p._h = None
            lib.tpt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
