"""The bench's byte model on the host (no GPU): the plan the benchmark workload gets
(gp_plan_params, the same host function gp_plan uses) and, for each of our kernels on
it, the algorithmic bytes per launch against the DRAM bytes ncu measured (the
`traffic` figures the bench reports).  Traffic well above the algorithmic bytes
would mean wasted re-reads; well below, a byte model that counts work not done."""
import numpy as np
import pytest

import bench
import gpinputs


@pytest.fixture(scope="module")
def bench_plan():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03608_gb300 import abi
    w = gpinputs.config_2d(1_000_000, 1.5)
    o = abi.default_opts(precision=abi.GP_FP32)
    info = abi.gp_plan_params(2, w.N, w.nu, w.eps, float(w.l.min()), float(w.l.max()),
                              [float(v) for v in w.points.min(0)], [float(v) for v in w.points.max(0)], o)
    return w, info


def test_the_benchmark_plan(bench_plan):
    _, i = bench_plan
    # the plan the profiles and the bench figures were taken on
    assert (i["nf"], i["M"], i["n_sigma"] + 1, i["kernel_width"], i["tile"], i["transform"]) == (8192, 2818, 9, 9, 24, 3)


def test_algorithmic_bytes_match_the_measured_traffic(bench_plan):
    w, info = bench_plan
    ab = bench.algorithmic_bytes(info, w.N, 1, 4)
    traffic = bench.MEASURED_TRAFFIC[(w.name, "f32", w.eps)]
    assert set(traffic) <= set(ab)
    for kernel, measured in traffic.items():
        ratio = measured / ab[kernel]
        assert 0.9 <= ratio <= 1.1, (kernel, ratio)

