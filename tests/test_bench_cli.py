"""bench.py's options and its host-side helpers (no GPU)."""
import pytest

import bench


def parse(*argv):
    return bench.parse(list(argv))


def test_defaults_keep_the_measured_path():
    a = parse()
    assert a.build == "batched-all" and a.refine == "once" and a.legs and a.serve
    assert a.per_size == 200 and a.limit == 1 << 22
    assert a.gpus == 1 and a.steps >= 1 and a.warmup >= 3


def test_refine_needs_a_batched_build():
    with pytest.raises(SystemExit):
        parse("--refine", "once_nt", "--build", "threads")
    assert parse("--refine", "once_nt", "--build", "batched").refine == "once_nt"


def test_oracle_sample_order_is_round_robin_over_sizes():
    """Both CPU baselines (cpu_baseline and --impl reference) take the queries
    in one fixed order: a permutation of the workload in which every prefix of
    5 j entries holds j queries of each size class."""
    per = 200
    order = bench.sample_order(5 * per, per)
    assert sorted(order) == list(range(5 * per))
    for j in range(1, 50):
        classes = [i // per for i in order[:5 * j]]
        assert all(classes.count(c) == j for c in range(5))
    assert order[:6] == [0, 200, 400, 600, 800, 1]


def test_percentiles():
    xs = list(range(1, 101))
    assert bench.pct(xs, 0.5) == 51 and bench.pct(xs, 0.99) == 99 and bench.pct(xs, 1.0) == 100
    assert bench.pct([], 0.5) is None
