"""Float32 Fourier-based transforms inside the mixed-precision corrections
(uniform power-of-two directions, Sec. 2.2.1 "U grid"): the refined solve with
FFT/DCT directions against the CPU oracle, against the same plan with
eigenbasis GEMMs in those directions, and refined to float64 accuracy."""
import numpy as np
import pytest

import oracle as O
import seeded_inputs as S
from _tpt import load

pytestmark = pytest.mark.gpu
tpt, L = load()

PRECS = {"bf16": L.TPT_PREC_MIXED_BF16, "bf16x3": L.TPT_PREC_MIXED_BF16X3, "tf32": L.TPT_PREC_MIXED_TF32}
# the bars of the refined mixed path (its float-pair residual stops the
# refinement at <= 1e-10; the oracle's long-double residual of the result
# differs from it by the float-pair rounding of r), and its element-wise
# distance to the oracle's float64 solution
RES_BAR = 1e-10 + 1e-14
ERR_BAR = 1e-9

P_, N_ = O.PERIODIC, O.NEUMANN
# (x, y) boundary pairs and stretch factors: which of x and y are uniform
CASES = {
    "FG": ([(P_, P_), (N_, N_), (N_, N_)], (0.0, 1.5, 2.0), ("fft", "gemm")),   # config-1 layout
    "GF": ([(N_, N_), (N_, N_), (N_, N_)], (2.0, 0.0, 2.5), ("gemm", "fft")),   # DCT in y
    "FF": ([(N_, N_), (P_, P_), (N_, N_)], (0.0, 0.0, 2.0), ("fft", "fft")),    # DCT x, DFT y
}


def _xf(names):
    return tuple(tpt.FFT if a == "fft" else tpt.GEMM for a in names)


def _solve(n, dirs, bcs, coef, prec, xform, f, rtol=1e-10):
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs, xform=xform, alpha=coef[0],
                    beta=coef[1], precision=PRECS[prec], rtol=rtol, max_refine=40)
    assert plan.transforms() == xform
    phi, info = plan.solve(tpt.field_to_device(f))
    return tpt.field_to_host(phi, n), info, plan


def _rhs(n, dirs, coef, seed):
    f = S.uniform_rhs(n, seed)
    if O.is_singular(dirs, coef[0]):
        f = S.remove_weighted_mean(f, [d.dxf for d in dirs])
    return f


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("coef", [(0.0, 1.0), (1.0, -5e-4)])
def test_mixed_fft_solve_matches_oracle(prec, case, coef):
    # 64 / 32 points in the Fourier directions; 45 and 33 leave ragged blocks
    # of lines (64 lines per block at these lengths) and odd line counts
    bcs, stretch, xf = CASES[case]
    n = (64 if xf[0] == "fft" else 45, 32 if xf[1] == "fft" else 45, 33)
    dirs = O.make_dirs(n, stretch, bcs)
    f = _rhs(n, dirs, coef, 41)
    got, info, _ = _solve(n, dirs, bcs, coef, prec, _xf(xf), f)
    r = O.residual(f, got, dirs, *coef, np.longdouble)
    rel = float(np.sqrt(np.sum(r ** 2) / np.sum(f ** 2)))
    ref, _ = O.solve_tensor(f, dirs, *coef)
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    print("fft-mixed", prec, case, coef, "iters", info["iters"], "rel_res", rel, "err", err)
    assert info["status"] == L.TPT_OK and info["rel_residual"] <= 1e-10 and rel <= RES_BAR, (info, rel)
    assert err <= ERR_BAR, err


@pytest.mark.parametrize("case", list(CASES))
def test_mixed_fft_equals_mixed_gemm_on_the_same_grid(case):
    # the Fourier transforms and the eigenbasis GEMMs diagonalise the same
    # operator: the refined solutions agree to the refinement's accuracy, and
    # the float32 transforms need no more corrections than the tensor cores
    bcs, stretch, xf = CASES[case]
    n = (128 if xf[0] == "fft" else 96, 64 if xf[1] == "fft" else 80, 48)
    dirs = O.make_dirs(n, stretch, bcs)
    f = _rhs(n, dirs, (0.0, 1.0), 43)
    a, ia, _ = _solve(n, dirs, bcs, (0.0, 1.0), "bf16x3", _xf(xf), f)
    b, ib, _ = _solve(n, dirs, bcs, (0.0, 1.0), "bf16x3", (tpt.GEMM, tpt.GEMM), f)
    d = float(np.abs(a - b).max() / np.abs(b).max())
    print("fft vs gemm", case, ia["iters"], ib["iters"], d)
    assert ia["rel_residual"] <= 1e-10 and ib["rel_residual"] <= 1e-10
    assert d <= 2 * ERR_BAR and ia["iters"] <= ib["iters"]


@pytest.mark.parametrize("case", ["FG", "FF"])
def test_mixed_fft_refined_to_float64_accuracy(case):
    # rtol 1e-13: the 1e-12 parity bar of the float64 path, over several
    # blocks of lines in both Fourier directions
    bcs, stretch, xf = CASES[case]
    n = (256, 128 if xf[1] == "fft" else 72, 40)
    dirs = O.make_dirs(n, stretch, bcs)
    f = _rhs(n, dirs, (0.0, 1.0), 47)
    got, info, _ = _solve(n, dirs, bcs, (0.0, 1.0), "bf16x3", _xf(xf), f, rtol=1e-13)
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    print("fft-mixed fp64-accurate", case, info["iters"], err)
    assert err <= 1e-12


def test_mixed_fft_manufactured_solution_and_graph_replay():
    # config-1 grid (periodic uniform x by FFT, stretched Neumann y by GEMM,
    # stretched z by Thomas) with the manufactured u = cos(2 pi x) cos(pi y)
    # cos(pi z): f = A u recovered to the refinement's accuracy; the third
    # identical call replays the solve graph and gives the same phi
    bcs, stretch, xf = CASES["FG"]
    n = (32, 32, 32)
    dirs = O.make_dirs(n, stretch, bcs)
    cen = []
    for d in dirs:
        faces = np.concatenate([[0.0], np.cumsum(d.dxf)])
        cen.append(0.5 * (faces[1:] + faces[:-1]))
    u = np.einsum("i,j,k->ijk", np.cos(2 * np.pi * cen[0]), np.cos(np.pi * cen[1]), np.cos(np.pi * cen[2]))
    f = O.apply_operator(u, dirs, 0.0, 1.0)
    plan = tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs, xform=_xf(xf), alpha=0.0, beta=1.0,
                    precision=PRECS["bf16x3"], rtol=1e-12, max_refine=40)
    fd = tpt.field_to_device(f)
    outs = []
    for _ in range(3):
        phi, info = plan.solve(fd)
        assert info["status"] == L.TPT_OK and info["rel_residual"] <= 1e-12
        outs.append(tpt.field_to_host(phi, n))
    err = float(np.abs(outs[0] - u).max() / np.abs(u).max())
    assert err <= 1e-10, err
    assert np.array_equal(outs[1], outs[2])


@pytest.mark.parametrize("n,prec", [((16, 32, 7), "bf16x3"), ((2048, 16, 6), "tf32"), ((4096, 16, 5), "bf16x3")])
def test_mixed_fft_shortest_and_longest_lines(n, prec):
    # 16 points: 64 lines per block, the last pass one stage; 2048 points in
    # float32 operands and 4096 in bf16 pairs: rows read in more than 256
    # vectors (the one-vector-at-a-time path), a block of two or four lines
    bcs = [(N_, N_), (P_, P_), (N_, N_)]
    dirs = O.make_dirs(n, (0.0, 0.0, 1.5), bcs)
    f = _rhs(n, dirs, (0.0, 1.0), 53)
    got, info, _ = _solve(n, dirs, bcs, (0.0, 1.0), prec, (tpt.FFT, tpt.FFT), f)
    r = O.residual(f, got, dirs, 0.0, 1.0, np.longdouble)
    rel = float(np.sqrt(np.sum(r ** 2) / np.sum(f ** 2)))
    ref, _ = O.solve_tensor(f, dirs, 0.0, 1.0)
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    print("fft-mixed lengths", n, prec, info["iters"], rel, err)
    assert info["rel_residual"] <= 1e-10 and rel <= RES_BAR and err <= ERR_BAR, (info, rel, err)
