"""Host-side arithmetic of the benchmark line (no GPU): the roofline entry of
the dominant inner kernel, its DRAM traffic from the stored ncu ratios, and
the kernel table."""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(os.path.dirname(HERE), "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def stats_of(**kw):
    """(ms, algorithmic bytes, flops, launches) per kernel slot."""
    base = {k: (0.0, 0.0, 0.0, 0) for k in ("arnoldi_spmv", "cgs_pass2", "cgs_pass3", "restart_update",
                                            "restart_residual")}
    base.update(kw)
    return base


def test_roofline_of_the_dominant_kernel(bench):
    # a: 400 launches of 95.5 MB in 20 ms in total -> 95.5 MB per 50 us = 1910 GB/s
    st = stats_of(arnoldi_spmv=(20.0, 400 * 95.5e6, 1.0e9, 400), cgs_pass2=(10.0, 400 * 70e6, 1.0e9, 400),
                  cgs_pass3=(15.0, 400 * 150e6, 1.0e9, 400))
    r = bench.roofline_of(st, bench.KNAMES["bicgstab"], 6788.3, "measured", "bicgstab", "batch64", "fp32")
    assert r["kernel"].startswith("k_bicg_a")
    assert r["achieved"] == pytest.approx(1910.0)
    assert r["frac"] == pytest.approx(1910.0 / 6788.3)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(95.5e6)
    # traffic: the stored DRAM / algorithmic ratio of k_bicg_a times the bytes per launch
    ratio = bench.NCU_TRAFFIC_RATIO[("batch64", "fp32", "bicgstab", "arnoldi_spmv")]
    assert r["traffic"] == pytest.approx(ratio * 95.5e6)
    # the step kernels together: all bytes over all time
    assert r["inner_kernels_GBps"] == pytest.approx(400 * (95.5e6 + 70e6 + 150e6) / 45e-3 / 1e9)


def test_traffic_only_for_the_captured_workload_and_precision(bench):
    st = stats_of(arnoldi_spmv=(20.0, 1e9, 1e9, 10), cgs_pass2=(1.0, 1e8, 1e8, 10), cgs_pass3=(1.0, 1e8, 1e8, 10))
    for wl, prec in (("mid3d", "fp32"), ("batch64", "fp64"), ("mid2d", "fp32")):
        r = bench.roofline_of(st, bench.KNAMES["bicgstab"], 6788.3, "measured", "bicgstab", wl, prec)
        assert r["traffic"] is None
    r = bench.roofline_of(st, bench.KNAMES["dcgs2"], 6788.3, "measured", "gmres", "batch64", "fp32")
    assert r["traffic"] is None and r["kernel"].startswith("k_dcgs_a")


def test_kernel_table_shares(bench):
    st = stats_of(arnoldi_spmv=(30.0, 3e9, 0.0, 100), cgs_pass2=(10.0, 1e9, 0.0, 100), restart_update=(0.0, 0.0,
                                                                                                        0.0, 0))
    t = bench.kernel_table(st, bench.KNAMES["bicgstab"])
    a = t["k_bicg_a (p update + product + rhat^* v)"]
    assert a["share"] == pytest.approx(0.75) and a["GBps"] == pytest.approx(100.0)
    assert len(t) == 2                      # kernels that never launched are left out
