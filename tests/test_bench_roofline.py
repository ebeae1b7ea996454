"""The bench's per-stage roofline arithmetic on CPU: algorithmic bytes and
flops per launch of each stage of a split-bf16 correction, the x inverse
averaged over a solve's corrections (the first one writes phi without reading
it), and the measured DRAM traffic scaled to the workload's points with the
same weights."""
import sys

import pytest

from _tpt import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _stages(iters, n=(512, 512, 512)):
    ms = [0.0] * 8
    for i in range(1, 7):
        ms[i] = 0.5 * iters          # 0.5 ms per launch of every stage
    return {d["kernel"]: d for d in bench.stage_rooflines(ms, iters, n, 2)["per_stage"]}


@pytest.mark.parametrize("iters", [1, 3, 4])
def test_algorithmic_bytes_and_flops_per_launch(iters):
    n = (512, 512, 512)
    npts = float(n[0] * n[1] * n[2])
    st = _stages(iters, n)
    # split bf16: three products of 2 N_alpha flops per point; 4-byte intermediates
    for nm in ("x_forward", "y_forward", "y_inverse", "x_inverse"):
        assert st[nm]["flops_per_launch"] == 3 * 2.0 * 512 * npts
    assert st["thomas"]["bytes_per_launch"] == 8 * npts
    assert st["residual"]["bytes_per_launch"] == 20 * npts
    # x inverse: 4 in + 16 (phi pair read and written), 4 in + 8 in the first correction
    expect = npts * ((4 + 8) + (iters - 1) * (4 + 16)) / iters
    assert st["x_inverse"]["bytes_per_launch"] == pytest.approx(expect, rel=1e-12)
    assert st["x_inverse"]["bound"] == "hbm"
    assert st["x_inverse"]["achieved"] == pytest.approx(expect / 0.5e-3 / 1e9, rel=1e-12)


def test_traffic_scaled_by_points_and_averaged_over_corrections():
    n = (256, 256, 256)
    npts = float(n[0] * n[1] * n[2])
    iters = 3
    st = _stages(iters, n)
    T = bench.MEASURED_TRAFFIC_PER_POINT
    fmt = "mixed_bf16x3"
    assert st["residual"]["traffic"] == pytest.approx(T[("residual", fmt)] * npts, rel=1e-12)
    assert st["thomas"]["traffic"] == pytest.approx(T[("thomas", fmt)] * npts, rel=1e-12)
    want = npts * (T[("x_inverse_first", fmt)] + (iters - 1) * T[("x_inverse", fmt)]) / iters
    assert st["x_inverse"]["traffic"] == pytest.approx(want, rel=1e-12)
    # measured bytes close to the algorithmic ones (no re-reads): within 15 %
    for nm in ("residual", "thomas", "x_inverse"):
        assert 0.85 <= st[nm]["traffic"] / st[nm]["bytes_per_launch"] <= 1.05, nm
