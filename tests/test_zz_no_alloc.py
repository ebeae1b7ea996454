"""tpt_thomas_noalloc: the Thomas step for callers that cannot allocate device
memory when they call the solver.  Its scratch is a fixed device array inside
the library; this test checks, through the C ABI, that two calls in a row give
the same result as the allocating entry point tpt_thomas, and that a plan too
large for the fixed array is rejected.  Kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
import seeded_inputs as S
from _tpt import load

pytestmark = pytest.mark.gpu
tpt, L = load()


def _plan(n, coef, bcs):
    dirs = O.make_dirs(n, (1.5, 2.0, 2.5), bcs)
    return tpt.Plan(n, [d.dxf for d in dirs], [d.dxc for d in dirs], bcs,
                    xform=(tpt.GEMM, tpt.GEMM), alpha=coef[0], beta=coef[1])


@pytest.mark.parametrize("coef,bcs", [((0.0, 1.0), [(1, 1)] * 3), ((1.0, -5e-4), [(2, 1), (1, 1), (1, 2)])])
def test_noalloc_matches_allocating_thomas_twice(coef, bcs):
    n = (70, 45, 33)
    plan = _plan(n, coef, bcs)
    stream = torch.cuda.current_stream()
    fh = tpt.field_to_device(S.uniform_rhs(n, 12))
    ref = plan.thomas(fh)                       # allocating entry point, own scratch
    torch.cuda.synchronize()
    ref_h = tpt.field_to_host(ref, n)
    for call in range(2):
        out = plan.new_field()
        out.fill_(float("nan"))
        st = L.lib.tpt_thomas_noalloc(plan._h, C.c_void_p(fh.data_ptr()), C.c_void_p(out.data_ptr()),
                                      C.c_void_p(stream.cuda_stream))
        assert st == L.TPT_OK, L.lib.tpt_status_string(st)
        torch.cuda.synchronize()
        got = tpt.field_to_host(out, n)
        err = np.abs(got - ref_h).max() / np.abs(ref_h).max()
        assert err <= 1e-13, (call, err)


def test_noalloc_rejects_plans_beyond_the_fixed_scratch():
    n = (256, 128, 129)                          # 4,227,072 points > 4,194,304
    plan = _plan(n, (1.0, -5e-4), [(1, 1)] * 3)
    x = plan.new_field()
    st = L.lib.tpt_thomas_noalloc(plan._h, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), None)
    assert st == L.TPT_ERR_UNSUPPORTED
