"""Host-side checks of libtpt.so: exported symbols, descriptor validation and
the host setup (rows, eigenvalues) against the oracle.  No GPU needed: these
use host-only plans (cuda_device < 0)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from _tpt import ROOT, load

tpt, L = load()


def _declared():
    src = open(os.path.join(ROOT, "include", "tpt.h")).read()
    return re.findall(r"^(?:int|const char\*)\s+(tpt_\w+)\s*\(", src, flags=re.M)


def test_every_declared_symbol_is_exported_and_bound():
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L.lib, name), name
    bound = {s[0] for s in L.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def _desc(n, grids, bcs, alpha=0.0, beta=1.0, prec=0, xform=(1, 1)):
    d = L.tpt_desc()
    keep = []
    for a in range(3):
        dxf = np.ascontiguousarray(grids[a][0], dtype=np.float64)
        dxc = np.ascontiguousarray(grids[a][1], dtype=np.float64)
        keep += [dxf, dxc]
        d.n[a] = n[a]
        d.dxf[a] = dxf.ctypes.data_as(L._dp)
        d.dxc[a] = dxc.ctypes.data_as(L._dp)
        d.bc[a][0], d.bc[a][1] = bcs[a]
    d.xform[0], d.xform[1] = xform
    d.alpha, d.beta, d.precision, d.rtol, d.max_refine = alpha, beta, prec, 0.0, 1
    return d, keep


def _host_plan(n, stretch, bcs, **kw):
    grids = [O.tanh_grid(n[a], 1.0, stretch[a]) for a in range(3)]
    d, keep = _desc(n, grids, bcs, **kw)
    h = C.c_void_p()
    st = L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h))
    return st, h, grids


def test_descriptor_validation():
    h = C.c_void_p()
    assert L.lib.tpt_plan_create(None, -1, C.byref(h)) == L.TPT_ERR_INVALID_ARG
    grids = [O.tanh_grid(8, 1.0, 1.0)] * 3
    d, keep = _desc((8, 8, 8), grids, [(1, 1)] * 3)
    d.n[1] = 0
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_INVALID_ARG
    d, keep = _desc((8, 8, 8), grids, [(0, 1), (1, 1), (1, 1)])   # periodic on one end only
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_INVALID_ARG
    d, keep = _desc((8, 8, 8), grids, [(1, 1), (1, 1), (0, 0)])   # periodic z
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_UNSUPPORTED
    d, keep = _desc((8, 8, 8), grids, [(1, 1)] * 3, alpha=0.0, beta=0.0)
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_INVALID_ARG
    bad = [g for g in grids]
    neg = (grids[0][0].copy(), grids[0][1])
    neg[0][3] = -1.0
    d, keep = _desc((8, 8, 8), [neg, grids[1], grids[2]], [(1, 1)] * 3)
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_INVALID_ARG
    assert not h.value


def test_host_plan_rejected_by_device_entry_points():
    st, h, _ = _host_plan((6, 6, 6), (1, 1, 1), [(1, 1)] * 3)
    assert st == L.TPT_OK
    x = C.c_void_p(256)
    assert L.lib.tpt_solve(h, x, x, x, None, None) == L.TPT_ERR_INVALID_ARG
    assert L.lib.tpt_transform(h, 0, 0, x, C.c_void_p(512), None) == L.TPT_ERR_INVALID_ARG
    assert L.lib.tpt_plan_destroy(h) == L.TPT_OK


@pytest.mark.parametrize("bcs", [[(1, 1), (1, 1), (1, 1)], [(0, 0), (2, 1), (1, 2)],
                                 [(2, 2), (1, 2), (2, 1)]])
def test_rows_bitwise_equal_to_oracle(bcs):
    n, stretch = (21, 17, 13), (1.5, 2.0, 2.5)
    st, h, grids = _host_plan(n, stretch, bcs)
    assert st == L.TPT_OK
    for a in range(3):
        ref = O.Direction(*grids[a], bcs[a])
        ra, rb, rc = (np.empty(n[a]) for _ in range(3))
        assert L.lib.tpt_plan_rows(h, a, ra.ctypes.data_as(L._dp), rb.ctypes.data_as(L._dp),
                                   rc.ctypes.data_as(L._dp)) == L.TPT_OK
        assert np.array_equal(ra, ref.a) and np.array_equal(rb, ref.b) and np.array_equal(rc, ref.c)
    L.lib.tpt_plan_destroy(h)


@pytest.mark.parametrize("n,stretch,bc", [(64, 2.0, (1, 1)), (200, 2.5, (1, 1)), (33, 1.0, (2, 1)),
                                          (40, 0.0, (0, 0)), (24, 1.5, (0, 0)), (1, 0.0, (1, 1))])
def test_eigenvalues_match_oracle(n, stretch, bc):
    st, h, grids = _host_plan((n, n, 4), (stretch, stretch, 1.0), [bc, bc, (1, 1)])
    assert st == L.TPT_OK
    lam = np.empty(n)
    assert L.lib.tpt_plan_eigenvalues(h, 0, lam.ctypes.data_as(L._dp)) == L.TPT_OK
    ref = O.Eigenbasis(O.Direction(*grids[0], bc)).lam
    got, exp = np.sort(lam), np.sort(ref)
    scale = np.abs(exp).max() if n > 1 else 1.0
    assert np.all(np.abs(got - exp) <= 1e-13 * np.maximum(np.abs(exp), 1e-3 * scale))
    # modes are ordered by decreasing eigenvalue; a null mode is mode 0 and exactly 0
    assert np.all(np.diff(lam) <= 0)
    if bc != (2, 1):
        assert lam[0] == 0.0
    L.lib.tpt_plan_destroy(h)


def test_grid_helper_matches_oracle_grid():
    for n, s in [(128, 2.0), (128, 4.0), (37, 1.3), (16, 0.0)]:
        dxf, dxc = tpt.grid_tanh(n, 1.0, s)
        rf, rc = O.tanh_grid(n, 1.0, s)
        # face differences near x = L lose a few bits to cancellation
        assert np.allclose(dxf, rf, rtol=1e-12, atol=0) and np.allclose(dxc, rc, rtol=1e-12, atol=0)
    assert L.lib.tpt_grid_tanh(0, 1.0, 1.0, None, None) == L.TPT_ERR_INVALID_ARG


def _xforms(h):
    x = (C.c_int * 2)()
    assert L.lib.tpt_plan_transforms(h, x) == L.TPT_OK
    return int(x[0]), int(x[1])


def test_fft_eigenvalues_in_transform_order():
    # periodic N = 32 (real DFT, half-complex order) and Neumann N = 64 (DCT-II order)
    for n, bc, kind in [(32, (0, 0), "dft"), (64, (1, 1), "dct"), (2, (0, 0), "dft"), (1, (1, 1), "dct")]:
        grids = [O.uniform_grid(n), O.uniform_grid(n), O.tanh_grid(8, 1.0, 1.0)]
        d, keep = _desc((n, n, 8), grids, [bc, bc, (1, 1)], xform=(L.TPT_XFORM_FFT, L.TPT_XFORM_AUTO))
        h = C.c_void_p()
        assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_OK
        assert _xforms(h) == (L.TPT_XFORM_FFT, L.TPT_XFORM_FFT)
        lam = np.empty(n)
        assert L.lib.tpt_plan_eigenvalues(h, 0, lam.ctypes.data_as(L._dp)) == L.TPT_OK
        hh = 1.0 / n
        if kind == "dct":
            ref = -4 * np.sin(np.pi * np.arange(n) / (2 * n)) ** 2 / hh ** 2
        else:
            ks = [0] + [(p + 1) // 2 for p in range(1, n - 1)] + ([n // 2] if n > 1 else [])
            ref = -4 * np.sin(np.pi * np.array(ks[:n]) / n) ** 2 / hh ** 2
        assert np.allclose(lam, ref, rtol=1e-13, atol=1e-9), (n, kind, lam[:4], ref[:4])
        assert lam[0] == 0.0
        L.lib.tpt_plan_destroy(h)


def test_transform_selection_rules():
    st_grid = O.tanh_grid(32, 1.0, 1.5)
    un = O.uniform_grid(32)
    h = C.c_void_p()
    # AUTO: FFT on uniform power of two, GEMM on stretched or non-power-of-two
    d, keep = _desc((32, 32, 8), [un, st_grid, O.tanh_grid(8, 1.0, 1.0)], [(0, 0), (1, 1), (1, 1)],
                    xform=(L.TPT_XFORM_AUTO, L.TPT_XFORM_AUTO))
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_OK
    assert _xforms(h) == (L.TPT_XFORM_FFT, L.TPT_XFORM_GEMM)
    L.lib.tpt_plan_destroy(h)
    d, keep = _desc((24, 32, 8), [O.uniform_grid(24), un, O.tanh_grid(8, 1.0, 1.0)], [(1, 1), (2, 1), (1, 1)],
                    xform=(L.TPT_XFORM_AUTO, L.TPT_XFORM_AUTO))
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_OK
    assert _xforms(h) == (L.TPT_XFORM_GEMM, L.TPT_XFORM_GEMM)   # 24 not a power of two; Dirichlet y
    L.lib.tpt_plan_destroy(h)
    # explicit FFT where it does not apply
    d, keep = _desc((32, 32, 8), [st_grid, un, O.tanh_grid(8, 1.0, 1.0)], [(1, 1), (1, 1), (1, 1)],
                    xform=(L.TPT_XFORM_FFT, L.TPT_XFORM_GEMM))
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_UNSUPPORTED
    # mixed-precision plans: explicit FFT from 16 points (float32 transforms in
    # the corrections), AUTO keeps the GEMM, fewer than 16 points are refused
    for prec in (L.TPT_PREC_MIXED_BF16X3, L.TPT_PREC_MIXED_BF16, L.TPT_PREC_MIXED_TF32):
        d, keep = _desc((32, 16, 8), [un, O.uniform_grid(16), O.tanh_grid(8, 1.0, 1.0)], [(0, 0), (1, 1), (1, 1)],
                        prec=prec, xform=(L.TPT_XFORM_FFT, L.TPT_XFORM_FFT))
        assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_OK
        assert _xforms(h) == (L.TPT_XFORM_FFT, L.TPT_XFORM_FFT)
        L.lib.tpt_plan_destroy(h)
        d, keep = _desc((32, 16, 8), [un, O.uniform_grid(16), O.tanh_grid(8, 1.0, 1.0)], [(0, 0), (1, 1), (1, 1)],
                        prec=prec, xform=(L.TPT_XFORM_AUTO, L.TPT_XFORM_AUTO))
        assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_OK
        assert _xforms(h) == (L.TPT_XFORM_GEMM, L.TPT_XFORM_GEMM)
        L.lib.tpt_plan_destroy(h)
        d, keep = _desc((32, 8, 8), [un, O.uniform_grid(8), O.tanh_grid(8, 1.0, 1.0)], [(1, 1), (1, 1), (1, 1)],
                        prec=prec, xform=(L.TPT_XFORM_GEMM, L.TPT_XFORM_FFT))
        assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_UNSUPPORTED
    # ... and more than 4096 points
    d, keep = _desc((8192, 16, 4), [O.uniform_grid(8192), O.uniform_grid(16), O.tanh_grid(4, 1.0, 1.0)],
                    [(0, 0), (1, 1), (1, 1)], prec=L.TPT_PREC_MIXED_BF16X3, xform=(L.TPT_XFORM_FFT, L.TPT_XFORM_FFT))
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_UNSUPPORTED


def test_tile_setters_and_batch_argument_checks():
    st, h, _ = _host_plan((6, 6, 6), (1, 1, 1), [(1, 1)] * 3, prec=L.TPT_PREC_MIXED_BF16X3)
    assert st == L.TPT_OK
    t = (C.c_int * 4)(32, 64, 0, 256)
    assert L.lib.tpt_plan_set_tiles(h, t) == L.TPT_OK
    got = (C.c_int * 4)()
    assert L.lib.tpt_plan_get_tiles(h, got) == L.TPT_OK
    assert list(got) == [32, 64, 0, 256]
    bad = (C.c_int * 4)(32, 48, 0, 0)
    assert L.lib.tpt_plan_set_tiles(h, bad) == L.TPT_ERR_INVALID_ARG
    assert list(got) == [32, 64, 0, 256]
    # host-only plans are rejected by the device entry points
    x = C.c_void_p(256)
    assert L.lib.tpt_plan_autotune(h, x, None, got) == L.TPT_ERR_INVALID_ARG
    L.lib.tpt_plan_destroy(h)
    st, h, _ = _host_plan((6, 6, 6), (1, 1, 1), [(1, 1)] * 3)
    assert L.lib.tpt_plan_set_tiles(h, t) == L.TPT_OK       # float64 plan: nothing to tune
    assert L.lib.tpt_plan_get_tiles(h, got) == L.TPT_OK and list(got) == [0, 0, 0, 0]
    L.lib.tpt_plan_destroy(h)
    # a batch needs a device, at least one instance and an output handle
    grids = [O.tanh_grid(8, 1.0, 1.0)] * 3
    d, keep = _desc((8, 8, 8), grids, [(1, 1)] * 3)
    b = C.c_void_p()
    assert L.lib.tpt_batch_create(C.byref(d), 1, -1, 0, C.byref(b)) == L.TPT_ERR_INVALID_ARG
    assert L.lib.tpt_batch_create(C.byref(d), 0, 0, 0, C.byref(b)) == L.TPT_ERR_INVALID_ARG
    assert L.lib.tpt_batch_create(None, 1, 0, 0, C.byref(b)) == L.TPT_ERR_INVALID_ARG
    assert L.lib.tpt_batch_create(C.byref(d), 1, 0, -1, C.byref(b)) == L.TPT_ERR_INVALID_ARG
    assert not b.value
    n = C.c_size_t()
    assert L.lib.tpt_batch_workspace_bytes(None, C.byref(n)) == L.TPT_ERR_INVALID_ARG
    assert L.lib.tpt_batch_destroy(None) == L.TPT_ERR_INVALID_ARG


def test_node_dirichlet_rows_and_face_grid_match_the_oracle():
    dxf, dxc = O.tanh_grid(20, 1.0, 2.3)
    for periodic in (False, True):
        wf, sc = tpt.grid_faces(dxf, dxc, periodic)
        rw, rs = O.face_grid(dxf, dxc, periodic)
        assert np.array_equal(wf, rw) and np.array_equal(sc, rs)
    wf, sc = O.face_grid(dxf, dxc, False)
    m = wf.size
    grids = [(wf, sc), O.tanh_grid(8, 1.0, 1.0), O.tanh_grid(6, 1.0, 1.0)]
    bcs = [(O.DIRICHLET_NODE, O.DIRICHLET_NODE), (1, 1), (1, 2)]
    d, keep = _desc((m, 8, 6), grids, bcs, alpha=1.0, beta=-1e-3)
    h = C.c_void_p()
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_OK
    a, b, c = np.empty(m), np.empty(m), np.empty(m)
    assert L.lib.tpt_plan_rows(h, 0, a.ctypes.data_as(L._dp), b.ctypes.data_as(L._dp),
                               c.ctypes.data_as(L._dp)) == L.TPT_OK
    ra, rb, rc = O.operator_1d(wf, sc, bcs[0])
    assert np.array_equal(a, ra) and np.array_equal(b, rb) and np.array_equal(c, rc)
    L.lib.tpt_plan_destroy(h)


def test_excluded_direction_rules():
    grids = [O.tanh_grid(8, 1.0, 1.0)] * 3
    h = C.c_void_p()
    X = O.NONE
    d, keep = _desc((8, 8, 8), grids, [(X, X), (1, 1), (1, 1)], alpha=1.0, beta=-1e-3)
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_OK       # yz option
    lam = np.empty(8)
    assert L.lib.tpt_plan_eigenvalues(h, 0, lam.ctypes.data_as(L._dp)) == L.TPT_OK
    assert np.all(lam == 0.0)
    L.lib.tpt_plan_destroy(h)
    d, keep = _desc((8, 8, 8), grids, [(X, X), (X, X), (1, 1)], alpha=1.0, beta=-1e-3)
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_OK       # z option
    L.lib.tpt_plan_destroy(h)
    d, keep = _desc((8, 8, 8), grids, [(X, X), (1, 1), (1, 1)])                 # Poisson: degenerate
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_INVALID_ARG
    d, keep = _desc((8, 8, 8), grids, [(X, 1), (1, 1), (1, 1)], alpha=1.0, beta=-1e-3)
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_INVALID_ARG
    d, keep = _desc((8, 8, 8), grids, [(1, 1), (1, 1), (X, X)], alpha=1.0, beta=-1e-3)
    assert L.lib.tpt_plan_create(C.byref(d), -1, C.byref(h)) == L.TPT_ERR_UNSUPPORTED


def test_pointer_guard_keeps_multicast_to_own_device_memory():
    """The transform GEMMs share operand tiles between paired CTAs by TMA
    multicast only for operands in the current GPU's own memory; host memory
    (and anything on a machine without that device) never qualifies."""
    buf = np.zeros(64, dtype=np.float64)
    flag = C.c_int(7)
    assert L.lib.tpt_pointer_on_device(C.c_void_p(buf.ctypes.data), 0, C.byref(flag)) == L.TPT_OK
    assert flag.value == 0
    flag.value = 7
    assert L.lib.tpt_pointer_on_device(None, 0, C.byref(flag)) == L.TPT_OK
    assert flag.value == 0
    assert L.lib.tpt_pointer_on_device(C.c_void_p(buf.ctypes.data), -1, C.byref(flag)) == L.TPT_ERR_INVALID_ARG
    assert L.lib.tpt_pointer_on_device(C.c_void_p(buf.ctypes.data), 0, None) == L.TPT_ERR_INVALID_ARG
