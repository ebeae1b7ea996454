"""Float64-accurate transforms by the Ozaki scheme on GB300 (TPT_PREC_FP64_OZAKI):
each transform (x and y, forward and inverse) against the float64 DGEMM of a
plain float64 plan of the same grid, within 2e-12 of the result's max norm
(the scheme keeps ~1e-13 of sum |a||b|; a level whose float32 sums were not
exact would leave ~1e-7); whole solves against the oracle at the float64
parity bar 1e-12 after the plan's float64 refinement step; directions beyond
the scheme's contraction length are refused."""
import numpy as np
import pytest
import torch

import oracle as O
import seeded_inputs as S
from _tpt import load

pytestmark = pytest.mark.gpu
tpt, L = load()

OZ = L.TPT_PREC_FP64_OZAKI
NNN = [(1, 1)] * 3
DND = [(2, 1), (1, 2), (2, 2)]
PNN = [(0, 0), (1, 1), (1, 1)]


def _plan(dirs, prec, alpha=0.0, beta=1.0, bcs=NNN, xform=(tpt.GEMM, tpt.GEMM)):
    n = tuple(d.n for d in dirs)
    return tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs, xform=xform, alpha=alpha, beta=beta,
                    precision=prec, max_refine=1)


@pytest.mark.parametrize("n", [(64, 48, 40), (70, 45, 33), (512, 96, 8), (24, 512, 6)])
def test_ozaki_transforms_match_the_float64_gemm(n):
    dirs = O.make_dirs(n, (1.5, 2.0, 2.5), NNN)
    p64, poz = _plan(dirs, L.TPT_PREC_FP64), _plan(dirs, OZ)
    f = tpt.field_to_device(S.uniform_rhs(n, 3) * 1e3)
    for ax in (0, 1):
        for inverse in (False, True):
            ref = p64.transform(f, ax, inverse)
            got = poz.transform(f, ax, inverse)
            torch.cuda.synchronize()
            err = (got - ref).abs().max().item() / ref.abs().max().item()
            assert err <= 2e-12, (n, ax, inverse, err)


CASES = [
    ((48, 40, 32), (1.5, 2.0, 2.5), NNN, (0.0, 1.0)),
    ((70, 45, 33), (1.5, 2.0, 2.5), NNN, (1.0, -5e-4)),
    ((64, 48, 40), (3.0, 1.0, 2.0), DND, (1.0, -0.5 * 1e-2)),
    ((40, 36, 28), (1.2, 2.0, 2.5), PNN, (0.0, 1.0)),
    ((128, 128, 128), (2.0, 2.0, 2.0), NNN, (0.0, 1.0)),
]


@pytest.mark.parametrize("case", CASES)
def test_ozaki_solves_match_the_oracle(case):
    n, stretch, bcs, coef = case
    dirs = O.make_dirs(n, stretch, bcs)
    f = S.uniform_rhs(n, 5)
    if O.is_singular(dirs, coef[0]):
        f = S.remove_weighted_mean(f, [d.dxf for d in dirs])
    plan = _plan(dirs, OZ, *coef, bcs=bcs)
    phi, info = plan.solve(tpt.field_to_device(f))
    got = tpt.field_to_host(phi, n)
    ref, _ = O.solve_tensor(f, dirs, *coef)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print("ozaki", n, bcs[0], coef, "err", err, "rel residual", info["rel_residual"])
    assert err <= 1e-12, err


def test_ozaki_refuses_directions_beyond_its_contraction_length():
    dirs = O.make_dirs((600, 16, 8), (1.5, 1.5, 1.5), NNN)
    with pytest.raises(L.TptError) as e:
        _plan(dirs, OZ)
    assert e.value.status == L.TPT_ERR_UNSUPPORTED
