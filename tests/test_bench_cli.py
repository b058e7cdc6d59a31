"""bench.py's options and its child-process leg, on the host (no GPU)."""
import sys

import pytest

import bench


def parse(*argv):
    old = sys.argv
    sys.argv = ["bench.py", *argv]
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_defaults_keep_the_measured_path():
    a = parse()
    assert a.build == "threads" and a.refine == "once" and a.build_legs and a.serve
    assert a.gpus == 1 and a.steps >= 1 and a.warmup >= 3


def test_refine_needs_a_batched_build():
    with pytest.raises(SystemExit):
        parse("--refine", "once_nt")
    assert parse("--refine", "once_nt", "--build", "batched").refine == "once_nt"


def test_child_leg_failure_is_reported_not_raised():
    """Without a GPU the child bench fails; the leg reports that as an error
    entry instead of raising, so the parent's numbers stand."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the child would run for real")
    r = bench.build_leg(parse("--cpu-seconds", "0"), "batched", "digest")
    assert r["build"] == "batched" and "error" in r
