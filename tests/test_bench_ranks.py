"""The bench is a one-GPU program.  Its own arm refuses more than one GPU
(and a launch under torchrun with WORLD_SIZE > 1) before it touches CUDA, so
no multi-GPU run can reach the paired-CTA GEMMs that share operand tiles by
TMA multicast; the reference arm (the CPU oracle) runs on rank 0 only and
the other ranks exit 0 without output."""
import os
import subprocess
import sys

import pytest

from _tpt import ROOT


def _bench(args, **env):
    e = dict(os.environ)
    e.update(env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True,
                          text=True, timeout=300, env=e, cwd=ROOT)


@pytest.mark.parametrize("args,env", [(["--gpus", "2"], {}), (["--gpus", "8"], {}),
                                      (["--gpus", "1"], {"WORLD_SIZE": "2", "RANK": "0"})])
def test_our_arm_refuses_more_than_one_gpu(args, env):
    out = _bench(args + ["--steps", "1", "--warmup", "1"], **env)
    assert out.returncode == 2, (out.returncode, out.stderr)
    assert out.stdout.strip() == ""
    assert "one GPU only" in out.stderr and "multicast" in out.stderr


def test_reference_arm_runs_on_rank_zero_only():
    out = _bench(["--impl", "reference", "--gpus", "2", "--size", "32", "--cpu-slabs", "4", "--steps", "1",
                  "--warmup", "1"], RANK="1", WORLD_SIZE="2")
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""


def test_refusal_helper_accepts_one_gpu():
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    old = os.environ.pop("WORLD_SIZE", None)
    try:
        assert bench.one_gpu_only(argparse.Namespace(gpus=1)) is None
        assert "one GPU only" in bench.one_gpu_only(argparse.Namespace(gpus=2))
    finally:
        if old is not None:
            os.environ["WORLD_SIZE"] = old
