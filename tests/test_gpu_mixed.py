"""Mixed-precision path on GB300: the tcgen05 GEMM on its own against float64
matmuls, then the refined mixed solve against the CPU oracle."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
import seeded_inputs as S
from _tpt import load

pytestmark = pytest.mark.gpu
tpt, L = load()

# Bars of the refined mixed path: its own float-pair residual stops the
# refinement at <= 1e-10 (relative 2-norm); the oracle's long-double residual
# of the returned phi differs from it by float-pair rounding of r (~1e-13 of
# |f| per point, measured below 2e-15 in the relative norm), hence 1e-10 plus
# 1e-14.  The element-wise distance to the oracle's float64 solution is at
# most ~1.2e-10 in these cases (measured), bounded here at 1e-9.
RES_BAR = 1e-10 + 1e-14
ERR_BAR = 1e-9

PRECS = {"bf16": L.TPT_PREC_MIXED_BF16, "bf16x3": L.TPT_PREC_MIXED_BF16X3, "tf32": L.TPT_PREC_MIXED_TF32}


def _tc_gemm(prec, A, B, tile=0, pair=0):
    M, K = A.shape
    N = B.shape[0]
    a = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    d = torch.full((N, M), float("nan"), dtype=torch.float64, device="cuda")
    work = torch.empty(8 * (M + N) * (K + 8) + 1024, dtype=torch.uint8, device="cuda")
    st = L.lib.tpt_tc_gemm(PRECS[prec], M, N, K, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                           C.c_void_p(d.data_ptr()), C.c_void_p(work.data_ptr()),
                           C.c_void_p(torch.cuda.current_stream().cuda_stream), tile, pair)
    assert st == L.TPT_OK, L.lib.tpt_status_string(st)
    torch.cuda.synchronize()
    return d.cpu().numpy().T          # column-major D -> (M, N)


SHAPES = [(128, 256, 64), (128, 32, 64), (256, 512, 512), (200, 150, 72), (96, 45, 40), (1000, 96, 128),
          (130, 300, 200)]


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("shape", SHAPES)
def test_tc_gemm_exact_on_representable_inputs(prec, shape):
    # small integers are exact in bf16 / tf32 and their products and sums are
    # exact in float32, so any layout, swizzle, K-step or edge mistake shows
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.integers(-8, 9, size=(M, K)).astype(np.float64)
    B = rng.integers(-8, 9, size=(N, K)).astype(np.float64)
    got = _tc_gemm(prec, A, B)
    assert np.array_equal(got, A @ B.T), (prec, shape, np.abs(got - A @ B.T).max())


@pytest.mark.parametrize("prec,rel", [("bf16", 2e-2), ("bf16x3", 2e-4), ("tf32", 4e-3)])
def test_tc_gemm_random_within_format_error(prec, rel):
    # relative to sum_k |A_mk||B_nk|: bf16 ~2^-8, split bf16 ~2^-16, tf32 ~2^-10
    M, N, K = 384, 256, 512
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, (M, K))
    B = rng.uniform(-1, 1, (N, K))
    got = _tc_gemm(prec, A, B)
    ref = A @ B.T
    scale = np.abs(A) @ np.abs(B).T
    err = np.max(np.abs(got - ref) / scale)
    assert err <= rel, err


def _dirs(n, stretch, bcs):
    return O.make_dirs(n, stretch, bcs)


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("case", ["poisson", "helmholtz"])
def test_mixed_solve_reaches_rtol(prec, case):
    n = (64, 48, 40)
    bcs = [(1, 1)] * 3
    alpha, beta = (0.0, 1.0) if case == "poisson" else (1.0, -5e-4)
    dirs = _dirs(n, (1.5, 2.0, 2.5), bcs)
    f = S.uniform_rhs(n, 21)
    if alpha == 0.0:
        f = S.remove_weighted_mean(f, [d.dxf for d in dirs])
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs, xform=(tpt.GEMM, tpt.GEMM),
                    alpha=alpha, beta=beta, precision=PRECS[prec], rtol=1e-10, max_refine=30)
    phi, info = plan.solve(tpt.field_to_device(f))
    got = tpt.field_to_host(phi, n)
    ref, _ = O.solve_tensor(f, dirs, alpha, beta)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    r = O.residual(f, got, dirs, alpha, beta, np.longdouble)
    rel = float(np.sqrt(np.sum(r ** 2) / np.sum(f ** 2)))
    print("mixed", prec, case, "iters", info["iters"], "rel_res(gpu)", info["rel_residual"],
          "rel_res(oracle)", rel, "err vs fp64", err)
    assert info["rel_residual"] <= 1e-10
    assert rel <= RES_BAR
    assert err <= ERR_BAR, err


@pytest.mark.parametrize("prec", list(PRECS))
def test_mixed_identity_operator_returns_rhs(prec):
    # alpha = 1, beta = 0: the refined solution is f itself; exercises the
    # float64 <-> float-pair conversions end to end
    n = (40, 24, 16)
    dirs = _dirs(n, (1.0, 2.0, 3.0), [(1, 1)] * 3)
    f = S.uniform_rhs(n, 5) * 1e3
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], [(1, 1)] * 3,
                    xform=(tpt.GEMM, tpt.GEMM), alpha=1.0, beta=0.0, precision=PRECS[prec],
                    rtol=1e-13, max_refine=10)
    phi, info = plan.solve(tpt.field_to_device(f))
    got = tpt.field_to_host(phi, n)
    assert np.abs(got - f).max() <= 1e-12 * np.abs(f).max(), np.abs(got - f).max()


MIXED_BCS = {
    "NNN": [(1, 1)] * 3,
    "DND": [(2, 1), (1, 2), (2, 2)],
    "PNN": [(0, 0), (1, 1), (1, 1)],
}


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("bcs", list(MIXED_BCS))
@pytest.mark.parametrize("coef", [(0.0, 1.0), (1.0, -5e-4)])
def test_mixed_ragged_sizes_and_boundaries(prec, bcs, coef):
    # 70 and 45 are not multiples of 8 (padded operand rows) and span two
    # 128-row tiles / partial 256-column tiles; Nz = 33 leaves identity rows in
    # the partition Thomas; periodic x uses the cyclic (Jacobi) eigenbasis
    n = (70, 45, 33)
    stretch = (1.5 if bcs != "PNN" else 1.2, 2.0, 2.5)
    dirs = _dirs(n, stretch, MIXED_BCS[bcs])
    f = S.uniform_rhs(n, 17)
    if O.is_singular(dirs, coef[0]):
        f = S.remove_weighted_mean(f, [d.dxf for d in dirs])
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], MIXED_BCS[bcs],
                    xform=(tpt.GEMM, tpt.GEMM), alpha=coef[0], beta=coef[1], precision=PRECS[prec],
                    rtol=1e-10, max_refine=40)
    phi, info = plan.solve(tpt.field_to_device(f))
    got = tpt.field_to_host(phi, n)
    r = O.residual(f, got, dirs, *coef, np.longdouble)
    rel = float(np.sqrt(np.sum(r ** 2) / np.sum(f ** 2)))
    ref, _ = O.solve_tensor(f, dirs, *coef)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print("ragged", prec, bcs, coef, "iters", info["iters"], "rel_res", rel, "err", err)
    assert info["rel_residual"] <= 1e-10 and rel <= RES_BAR
    assert err <= ERR_BAR, err


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_mixed_refined_to_float64_accuracy_matches_oracle(prec):
    # refining the tensor-core correction solves to rtol 1e-13 gives a
    # float64-accurate result: the 1e-12 parity bar of the float64 path
    n = (96, 80, 64)
    dirs = _dirs(n, (1.5, 2.0, 2.5), [(1, 1)] * 3)
    f = S.remove_weighted_mean(S.uniform_rhs(n, 29), [d.dxf for d in dirs])
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], [(1, 1)] * 3,
                    xform=(tpt.GEMM, tpt.GEMM), alpha=0.0, beta=1.0, precision=PRECS[prec],
                    rtol=1e-13, max_refine=40)
    phi, info = plan.solve(tpt.field_to_device(f))
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    err = np.abs(tpt.field_to_host(phi, n) - ref).max() / np.abs(ref).max()
    print("fp64-accurate", prec, "iters", info["iters"], "err", err)
    assert err <= 1e-12


PAIR_CASES = [((512, 512, 128), 256, 1), ((512, 512, 128), 256, 2), ((1024, 256, 96), 128, 1),
              ((256, 768, 200), 128, 2), ((384, 512, 64), 256, 1),      # odd m-tile count: one CTA per tile
              ((512, 640, 64), 256, 2)]                                # odd n-tile count: one CTA per tile


@pytest.mark.parametrize("shape,tile,pair", PAIR_CASES)
def test_tc_gemm_two_cta_pairs_exact(shape, tile, pair):
    # clusters of two CTAs sharing an operand tile by TMA multicast must give
    # exactly the products of small integers, as the single-CTA kernel does
    M, N, K = shape
    rng = np.random.default_rng(M + 3 * N + 7 * K + pair)
    A = rng.integers(-8, 9, size=(M, K)).astype(np.float64)
    B = rng.integers(-8, 9, size=(N, K)).astype(np.float64)
    got = _tc_gemm("bf16x3", A, B, tile=tile, pair=pair)
    assert np.array_equal(got, A @ B.T), (shape, tile, pair, np.abs(got - A @ B.T).max())


def test_mixed_solve_with_two_cta_pairs_equals_default():
    n = (256, 128, 64)
    dirs = _dirs(n, (1.5, 2.0, 2.5), [(1, 1)] * 3)
    f = S.remove_weighted_mean(S.uniform_rhs(n, 23), [d.dxf for d in dirs])
    kw = dict(xform=(tpt.GEMM, tpt.GEMM), alpha=0.0, beta=1.0, precision=PRECS["bf16x3"], rtol=0.0, max_refine=3)
    ref_plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], [(1, 1)] * 3, **kw)
    ref, _ = ref_plan.solve(tpt.field_to_device(f))
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], [(1, 1)] * 3, **kw)
    plan.set_tiles((256, 128, 128, 256))
    plan.set_pairing((1, 2, 1, 2))
    assert plan.pairing() == (1, 2, 1, 2)
    got, info = plan.solve(tpt.field_to_device(f))
    a, r = got.cpu().numpy(), ref.cpu().numpy()
    assert np.abs(a - r).max() <= 1e-12 * np.abs(r).max()


def _tc_gemm_out(prec, A, B, kind, rm, sm, sn, size, tile, tma_out, pair=0):
    M, K = A.shape
    N = B.shape[0]
    a = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dt = torch.float32 if kind == L.TPT_GEMM_OUT_F32 else torch.bfloat16
    # sentinel everywhere: elements outside the index set must stay untouched
    o0 = torch.full((size,), -7.25, dtype=dt, device="cuda")
    o1 = torch.full((size,), -7.25, dtype=dt, device="cuda")
    work = torch.empty(8 * (M + N) * (K + 8) + 1024, dtype=torch.uint8, device="cuda")
    st = L.lib.tpt_tc_gemm_out(PRECS[prec], M, N, K, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), kind,
                               rm, sm, sn, C.c_void_p(o0.data_ptr()), C.c_void_p(o1.data_ptr()),
                               C.c_void_p(work.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream),
                               tile, tma_out, pair)
    assert st == L.TPT_OK, L.lib.tpt_status_string(st)
    torch.cuda.synchronize()
    return o0.float().cpu().numpy(), o1.float().cpu().numpy()


# (M, N, K), rm, sm, sn: one block of rows (rm >= M), blocks of 32/64/96 rows
# with padded block strides (the transforms' T1/T3 layouts), ragged M and N
# edges, and a column stride that is not 16-byte aligned (direct stores)
OUT_CASES = [((384, 512, 64), 1 << 30, 0, 400), ((200, 300, 72), 1 << 30, 0, 208),
             ((256, 384, 96), 64, 64 * 384 + 32, 64), ((384, 256, 64), 96, 96 * 256 + 32, 96),
             ((192, 200, 40), 32, 32 * 200 + 32, 32), ((160, 140, 64), 1 << 30, 0, 161)]


@pytest.mark.parametrize("kind", ["f32", "bf16", "split"])
@pytest.mark.parametrize("case", OUT_CASES)
@pytest.mark.parametrize("tile", [128, 256])
@pytest.mark.parametrize("pair", [0, 1, 2])
def test_tc_gemm_output_formats_and_layouts(kind, case, tile, pair):
    # the bulk-tensor-store epilogue and the per-thread stores must write the
    # same values to the same indices and nothing else; the values are the
    # exact integer products, rounded once to the output format
    (M, N, K), rm, sm, sn = case
    k = {"f32": L.TPT_GEMM_OUT_F32, "bf16": L.TPT_GEMM_OUT_BF16, "split": L.TPT_GEMM_OUT_SPLIT_BF16}[kind]
    rng = np.random.default_rng(M + N + K + tile)
    A = rng.integers(-40, 41, size=(M, K)).astype(np.float64)
    B = rng.integers(-40, 41, size=(N, K)).astype(np.float64)
    m = np.arange(M)[:, None]
    n = np.arange(N)[None, :]
    idx = (m % rm) + (m // rm) * sm + n * sn
    size = int(idx.max()) + 1 + 64
    # pair 1: clusters of two m-tiles share B (even m-tile count), pair 2: two
    # n-tiles share A (even n-tile count, float32 out); otherwise one CTA per tile
    outs = [_tc_gemm_out("bf16x3", A, B, k, rm, sm, sn, size, tile, t, pair) for t in (1, 0)]
    (t0, t1), (d0, d1) = outs
    assert np.array_equal(t0, d0) and (kind != "split" or np.array_equal(t1, d1)), (kind, case, tile)
    hi, lo = outs[0]
    D = A @ B.T                                     # exact: |D| < 2^24
    if kind == "f32":
        assert np.array_equal(hi[idx], D)
    else:
        hb = torch.from_numpy(D).to(torch.bfloat16)
        assert np.array_equal(hi[idx], hb.float().numpy())
        if kind == "split":
            lb = torch.from_numpy(D - hb.double().numpy()).to(torch.bfloat16)
            assert np.array_equal(lo[idx], lb.float().numpy())
    untouched = np.ones(size, bool)
    untouched[idx.ravel()] = False
    assert np.all(hi[untouched] == -7.25)
    if kind == "split":
        assert np.all(lo[untouched] == -7.25)


# (n, boundaries, (alpha, beta)): full 64 x 8 tiles with three z segments
# (64 + 64 + 2 planes); periodic x and y (edge points load the wrapped
# neighbours) with ragged x and y tiles; Dirichlet walls (diagonal remainder)
# with Helmholtz; a grid narrower than one tile in every direction
RES_CASES = [((128, 64, 130), [(1, 1)] * 3, (0.0, 1.0)),
             ((132, 44, 70), [(0, 0), (0, 0), (1, 1)], (0.0, 1.0)),
             ((100, 36, 66), [(2, 1), (1, 2), (2, 2)], (1.0, -5e-4)),
             ((4, 9, 3), [(0, 0), (0, 0), (2, 1)], (1.0, -1e-3))]


@pytest.mark.parametrize("case", RES_CASES, ids=["full", "periodic-xy", "walls-helmholtz", "tiny"])
def test_tma_residual_equals_direct_loads_and_the_oracle(case):
    # both residual kernels apply the same float-pair operations to every
    # point, so three fixed corrections give the same phi (to the bit where
    # the problem is not singular); the TMA-staged solve refined to 1e-10 must
    # then match the oracle
    n, bcs, coef = case
    dirs = _dirs(n, (1.5, 2.0, 2.5), bcs)
    f = S.uniform_rhs(n, 31)
    if O.is_singular(dirs, coef[0]):
        f = S.remove_weighted_mean(f, [d.dxf for d in dirs])
    kw = dict(xform=(tpt.GEMM, tpt.GEMM), alpha=coef[0], beta=coef[1], precision=PRECS["bf16x3"])
    out = []
    for variant in (1, 2):
        plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs, rtol=0.0, max_refine=3, **kw)
        plan.set_residual_kernel(variant)
        phi, info = plan.solve(tpt.field_to_device(f))
        out.append((phi.cpu().numpy(), info))
    (a, ia), (b, ib) = out
    assert ia["iters"] == ib["iters"]
    if O.is_singular(dirs, coef[0]):
        # the mean removal and the gauge sum with float64 atomics, whose order
        # changes from run to run: equal to rounding of those sums (the
        # residual, near the float-pair floor, to a few of its digits)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max(), np.abs(a - b).max()
        assert abs(ia["rel_residual"] - ib["rel_residual"]) <= 1e-3 * ia["rel_residual"] + 1e-16
    else:
        assert np.array_equal(a, b)
        # r^2 is summed in float32 per thread over its plane segment (64
        # planes for the tiles, 32 for direct loads), then in float64
        assert abs(ia["rel_residual"] - ib["rel_residual"]) <= 1e-5 * ia["rel_residual"]
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs, rtol=1e-10, max_refine=40, **kw)
    plan.set_residual_kernel(2)
    phi, info = plan.solve(tpt.field_to_device(f))
    got = tpt.field_to_host(phi, n)
    r = O.residual(f, got, dirs, *coef, np.longdouble)
    rel = float(np.sqrt(np.sum(r ** 2) / np.sum(f ** 2)))
    ref, _ = O.solve_tensor(f, dirs, *coef)
    print("tma-res", case, "rel", rel, "gpu", info["rel_residual"], "err", np.abs(got - ref).max() / np.abs(ref).max())
    assert info["rel_residual"] <= 1e-10 and rel <= RES_BAR, (info, rel)
    assert np.abs(got - ref).max() <= ERR_BAR * np.abs(ref).max()


def test_adaptive_solve_replayed_as_graph_and_continued_past_the_planned_corrections():
    # the adaptive solve stops on the device (converge_kernel) and is replayed
    # from a CUDA graph once the same call repeats: repeated calls must give
    # the first call's result, a new right-hand side in the same buffer must
    # give that right-hand side's solution, and a plan whose previous solve
    # needed one correction must continue past it when the next one needs more
    n = (64, 48, 40)
    dirs = _dirs(n, (1.5, 2.0, 2.5), [(1, 1)] * 3)
    kw = dict(xform=(tpt.GEMM, tpt.GEMM), alpha=0.0, beta=1.0, precision=PRECS["bf16x3"], rtol=1e-10,
              max_refine=8)
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], [(1, 1)] * 3, **kw)
    f1 = S.remove_weighted_mean(S.uniform_rhs(n, 41), [d.dxf for d in dirs])
    f2 = S.remove_weighted_mean(S.uniform_rhs(n, 42), [d.dxf for d in dirs])
    f_dev = tpt.field_to_device(f1)
    phi = plan.new_field()
    work = plan.new_workspace()
    outs = []
    for _ in range(4):                      # direct, direct + capture, replay, replay
        _, info = plan.solve(f_dev, phi, work)
        outs.append((phi.cpu().numpy().copy(), info))
    for o, inf in outs[1:]:
        assert np.abs(o - outs[0][0]).max() <= 1e-12 * np.abs(outs[0][0]).max()
        assert inf["iters"] == outs[0][1]["iters"] and inf["rel_residual"] <= 1e-10
    f_dev.copy_(tpt.field_to_device(f2))
    _, info2 = plan.solve(f_dev, phi, work)
    ref2, _ = O.solve_tensor(f2, dirs, 0.0, 1.0)
    got2 = tpt.field_to_host(phi, n)
    print("graph-rhs2 err", np.abs(got2 - ref2).max() / np.abs(ref2).max(), "gpu", info2["rel_residual"])
    assert info2["rel_residual"] <= 1e-10
    assert np.abs(got2 - ref2).max() <= ERR_BAR * np.abs(ref2).max()
    # a zero right-hand side converges at once (one correction); the next,
    # non-zero one must then run past that plan
    plan0 = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], [(1, 1)] * 3, **kw)
    _, i0 = plan0.solve(tpt.field_to_device(np.zeros(n)))
    assert i0["iters"] == 1
    _, i1 = plan0.solve(tpt.field_to_device(f1))
    assert i1["iters"] > 1 and i1["rel_residual"] <= 1e-10


def test_concurrent_solves_on_one_plan_from_two_threads():
    # two host threads solve on one plan with their own workspaces and
    # streams: the shared null-line fork/join and the plan's graph are taken
    # in turn, so every result equals the same solve made alone
    import threading
    n = (64, 48, 40)
    dirs = _dirs(n, (1.5, 2.0, 2.5), [(1, 1)] * 3)
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], [(1, 1)] * 3, xform=(tpt.GEMM, tpt.GEMM),
                    alpha=0.0, beta=1.0, precision=PRECS["bf16x3"], rtol=1e-10, max_refine=8)
    fs = [tpt.field_to_device(S.remove_weighted_mean(S.uniform_rhs(n, 60 + t), [d.dxf for d in dirs]))
          for t in range(2)]
    refs = [plan.solve(f)[0].cpu().numpy() for f in fs]
    errors = []

    def worker(t):
        try:
            stream = torch.cuda.Stream()
            work = plan.new_workspace()
            phi = plan.new_field()
            for _ in range(6):
                _, info = plan.solve(fs[t], phi, work, stream=stream)
                stream.synchronize()
                got = phi.cpu().numpy()
                if not (np.abs(got - refs[t]).max() <= 1e-12 * np.abs(refs[t]).max() and
                        info["rel_residual"] <= 1e-10):
                    errors.append((t, float(np.abs(got - refs[t]).max()), info))
        except Exception as e:   # noqa: BLE001 (reported below)
            errors.append((t, repr(e)))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors


def test_device_stopping_test_reports_misses_and_continues_after_a_graph_replay():
    # a plan allowed one correction reports NOT_CONVERGED with its residual;
    # a plan whose solve was captured as a graph for a zero right-hand side
    # (one correction) replays that graph for a random one in the same
    # buffer and continues with further corrections until rtol
    n = (48, 40, 32)
    bcs = [(2, 1), (1, 2), (2, 2)]            # walls: not singular
    dirs = _dirs(n, (1.5, 2.0, 2.5), bcs)
    kw = dict(xform=(tpt.GEMM, tpt.GEMM), alpha=0.0, beta=1.0, precision=PRECS["bf16x3"])
    f = S.uniform_rhs(n, 71)
    one = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs, rtol=1e-10, max_refine=0, **kw)
    _, info = one.solve(tpt.field_to_device(f), raise_not_converged=False)
    assert info["iters"] == 1 and info["rel_residual"] > 1e-10 and info["status"] == L.TPT_ERR_NOT_CONVERGED

    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs, rtol=1e-10, max_refine=8, **kw)
    f_dev = tpt.field_to_device(np.zeros(n))
    phi = plan.new_field()
    work = plan.new_workspace()
    easy = [plan.solve(f_dev, phi, work)[1]["iters"] for _ in range(4)]   # captured, then replayed
    assert easy == [1, 1, 1, 1], easy
    f_dev.copy_(tpt.field_to_device(f))
    _, info = plan.solve(f_dev, phi, work)
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    got = tpt.field_to_host(phi, n)
    print("stop-test err", np.abs(got - ref).max() / np.abs(ref).max(), "gpu", info["rel_residual"])
    assert info["status"] == L.TPT_OK and info["rel_residual"] <= 1e-10 and info["iters"] > 1, info
    assert np.abs(got - ref).max() <= ERR_BAR * np.abs(ref).max()


def test_pointer_guard_on_the_gpu():
    """Device memory of this GPU qualifies for multicast operand sharing;
    pinned host memory and a device index past the last GPU do not."""
    dev = torch.empty(256, dtype=torch.float64, device="cuda")
    pin = torch.empty(256, dtype=torch.float64).pin_memory()
    flag = C.c_int(-1)
    cur = torch.cuda.current_device()
    assert L.lib.tpt_pointer_on_device(C.c_void_p(dev.data_ptr()), cur, C.byref(flag)) == L.TPT_OK
    assert flag.value == 1
    assert L.lib.tpt_pointer_on_device(C.c_void_p(pin.data_ptr()), cur, C.byref(flag)) == L.TPT_OK
    assert flag.value == 0
    assert L.lib.tpt_pointer_on_device(C.c_void_p(dev.data_ptr()), torch.cuda.device_count(),
                                       C.byref(flag)) == L.TPT_OK
    assert flag.value == 0



def _thomas_f32_sequential(fh, lx, ly, dz, alpha, beta):
    """The plain Thomas recurrence in float32 (numpy, vectorised over lines):
    the accuracy a float32 modal solve can be expected to reach per line."""
    f32 = np.float32
    shift = (f32(alpha) + f32(beta) * (lx.astype(f32)[:, None] + ly.astype(f32)[None, :])).astype(f32)
    a, b, c = (f32(beta) * dz.a.astype(f32)), (f32(beta) * dz.b.astype(f32)), (f32(beta) * dz.c.astype(f32))
    nz = fh.shape[2]
    cp = np.zeros(fh.shape, f32)
    dp = np.zeros(fh.shape, f32)
    m = b[0] + shift
    cp[:, :, 0] = c[0] / m
    dp[:, :, 0] = fh[:, :, 0] / m
    for k in range(1, nz):
        m = (b[k] + shift) - a[k] * cp[:, :, k - 1]
        cp[:, :, k] = c[k] / m
        dp[:, :, k] = (fh[:, :, k] - a[k] * dp[:, :, k - 1]) / m
    x = np.zeros(fh.shape, f32)
    x[:, :, -1] = dp[:, :, -1]
    for k in range(nz - 2, -1, -1):
        x[:, :, k] = dp[:, :, k] - cp[:, :, k] * x[:, :, k + 1]
    return x.astype(np.float64)


def _line_errors(got, ref):
    scale = np.abs(ref).max(axis=2)
    return np.abs(got - ref).max(axis=2) / np.where(scale > 0, scale, 1.0)


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("nz", [33, 200, 256, 387, 512])
@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
@pytest.mark.parametrize("coef", [(1.0, -5e-4), (0.0, 1.0)])
def test_mixed_thomas_kernels_match_the_oracle_recurrence(variant, nz, prec, coef):
    """The float32 modal Thomas step of the mixed path (partition method, both
    kernels) against the oracle's float64 recurrence on the same float32
    inputs: every line within a small multiple of what a plain sequential
    float32 Thomas sweep reaches on that line (near-singular Poisson lines
    lose digits in any float32 solve), and the bulk near float32 rounding.
    Nx = 20 with Ny = 12 (padded to 16 operand rows) gives 10 tiles of 32
    lines with dummy padding lines; Nz = 33, 200 and 387 leave padding rows."""
    n = (20, 12, nz)
    bcs = [(1, 1)] * 3
    dirs = O.make_dirs(n, (1.5, 2.0, 2.5), bcs)
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs, xform=(tpt.GEMM, tpt.GEMM),
                    alpha=coef[0], beta=coef[1], precision=PRECS[prec], rtol=1e-10, max_refine=30)
    plan.set_thomas_kernel(variant)
    lx, ly = plan.eigenvalues(0), plan.eigenvalues(1)
    fh = S.uniform_rhs(n, 31).astype(np.float32).astype(np.float64)
    sing = O.is_singular(dirs, coef[0])
    nx, ny = n[0], n[1]
    ldy = (ny + 7) // 8 * 8
    t2 = np.zeros((nz, nx, ldy), np.float32)
    t2[:, :, :ny] = fh.transpose(2, 0, 1)
    t2d = torch.from_numpy(t2.ravel()).cuda()
    if prec == "bf16x3":
        o0 = torch.zeros(t2.size, dtype=torch.int16, device="cuda")
        o1 = torch.zeros(t2.size, dtype=torch.int16, device="cuda")
    else:
        o0 = torch.zeros(t2.size, dtype=torch.float32, device="cuda")
        o1 = None
    work = plan.new_workspace()
    st = L.lib.tpt_mixed_thomas(plan._h, C.c_void_p(t2d.data_ptr()), C.c_void_p(o0.data_ptr()),
                                C.c_void_p(o1.data_ptr() if o1 is not None else 0), C.c_void_p(work.data_ptr()),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.TPT_OK, L.lib.tpt_status_string(st)
    if prec == "bf16x3":
        def bf(t):
            u = t.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
            return u.view(np.float32).astype(np.float64)
        out = bf(o0) + bf(o1)
    else:
        out = o0.cpu().numpy().astype(np.float64)
    got = out.reshape(nz, nx, ldy)[:, :, :ny].transpose(1, 2, 0)
    ref_in = fh.copy()
    if sing:   # the kernel projects the null line; give the references the projected line
        w = dirs[2].dxf
        ref_in[0, 0, :] -= np.sum(w * ref_in[0, 0, :]) / np.sum(w)
    ref = O.thomas_modal(ref_in, lx, ly, dirs[2], coef[0], coef[1], (0, 0) if sing else None)
    seq = _thomas_f32_sequential(ref_in, lx, ly, dirs[2], coef[0], coef[1])
    if sing:
        w = dirs[2].dxf
        ref[0, 0, :] -= np.sum(w * ref[0, 0, :]) / np.sum(w)
        seq[0, 0, :] = ref[0, 0, :]       # the null line is solved in float64 by its own kernel
    e_got, e_seq = _line_errors(got, ref), _line_errors(seq, ref)
    print("thomas", variant, nz, prec, coef, "max", e_got.max(), "median", np.median(e_got),
          "seq max", e_seq.max(), "seq median", np.median(e_seq))
    # the T3 format rounds each value once more: a bf16 hi/lo pair keeps ~16
    # significant bits (2^-17 relative), float32 (the tf32 path) all 24
    fmt = 2.0 ** -16 if prec == "bf16x3" else 0.0
    assert np.all(e_got <= 16.0 * e_seq + 4e-6 + fmt), (e_got.max(), e_seq.max())
    assert np.median(e_got) <= 2.0 * np.median(e_seq) + 1e-6 + fmt / 2
    if sing:   # the float64 null line: only the output format's rounding
        assert e_got[0, 0] <= 1e-7 + fmt, e_got[0, 0]
