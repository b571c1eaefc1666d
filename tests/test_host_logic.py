"""Host-side logic that needs no GPU: the clock sampler's parsing of
nvidia-smi samples, the serving latency percentiles, the traffic figure's
guard on the kernel source, and the workload description of the bench line."""
import importlib.util
import os
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


@pytest.fixture
def scratch():
    # inside the package's git-ignored build folder, so the test writes nothing outside the repository
    d = os.path.join(ROOT, "paper_1205_3830_gb300", "_build", "host_logic_tests")
    os.makedirs(d, exist_ok=True)
    return d


def _sampler_with(bench, scratch, lines):
    path = os.path.join(scratch, "clocks.csv")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s = bench.ClockSampler(0)
    s.path = path
    s.f = open(os.devnull, "w")
    s.proc = _FakeProc()
    return s


def test_clock_sampler_median_and_reasons(bench, scratch):
    # fields: index, clocks.sm, clocks.max.sm, power, active mask, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    lines = ["0, 2070, 2070, 1210.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 1950, 2070, 1398.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2010, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "garbage line",
             "0, [N/A], 2070, 1390.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    out = _sampler_with(bench, scratch, lines).stop()
    assert out == {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(os.path.join(scratch, "clocks.csv"))     # the sample file is removed


def test_clock_sampler_reports_thermal_slowdown(bench, scratch):
    lines = ["0, 1500, 2070, 900.0, 0x0000000000000040, Active, Active, Not Active, Not Active"]
    out = _sampler_with(bench, scratch, lines).stop()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_clock_sampler_without_samples(bench, scratch):
    assert _sampler_with(bench, scratch, ["only garbage"]).stop() is None
    s = bench.ClockSampler(0)                 # never started (no nvidia-smi)
    assert s.stop() is None


def test_latency_percentiles():
    from paper_1205_3830_gb300 import serve
    reqs = [types.SimpleNamespace(latency=i / 1e3) for i in range(100, 0, -1)]     # 1 .. 100 ms, unsorted
    reqs.append(types.SimpleNamespace(latency=None))                                   # still running: ignored
    st = serve.latency_stats(reqs)
    assert st["count"] == 100
    assert st["p50_ms"] == pytest.approx(51.0)       # index round(0.50 * 99) = 50
    assert st["p99_ms"] == pytest.approx(99.0)       # index round(0.99 * 99) = 98
    assert st["max_ms"] == pytest.approx(100.0)
    assert serve.latency_stats([]) == {}


def test_latency_stats_report_the_plans_share():
    from paper_1205_3830_gb300 import serve
    reqs = [types.SimpleNamespace(latency=0.01 * (i + 1),
                                  result={"plan_host_ms": 1.0 + i, "plan_dev_ms": 0.5 * i, "id_dev_ms": 10.0 + i})
            for i in range(5)]
    st = serve.latency_stats(reqs)
    assert st["plan_host_p50_ms"] == 3.0 and st["plan_dev_p50_ms"] == 1.0 and st["id_dev_p50_ms"] == 12.0


def test_traffic_figure_follows_the_kernel_source(bench, monkeypatch):
    """The ncu traffic of the product kernel is reported only for the source
    it was measured on: any other hash turns it off."""
    assert isinstance(bench.tc_source_unchanged(), bool)
    monkeypatch.setitem(bench.TC_TRAFFIC, "source_sha1", "0" * 40)
    assert bench.tc_source_unchanged() is False


def test_workload_config_names_the_workload(bench):
    import synth
    cfg = synth.CONFIGS["large_tall"]
    args = types.SimpleNamespace(nprobe=8, mode="fp64_emulated", estimator="rows", omega="gaussian", omega_bits=0)
    c = bench.workload_config(cfg, args)
    assert (c["m"], c["n"], c["k"], c["l"]) == (262144, 8192, 200, 208)
    assert c["workload"].startswith("large_tall: complex128")
    assert "32 GiB" in c["workload"] and "larger than L2" in c["l2"]
    args.omega, args.omega_bits = "srft", 24
    c = bench.workload_config(cfg, args)
    assert c["omega"].startswith("subsampled randomized Fourier transform") and "24 bits" in c["omega"]


def test_binding_argument_checks_raise_value_errors():
    """The binding's checks raise (they do not vanish under python -O like
    asserts would): host tensors, non-tensors and wrong perm types."""
    import torch
    import paper_1205_3830_gb300 as rid
    with pytest.raises(ValueError, match="CUDA tensor"):
        rid._check_matrix(torch.zeros((4, 3), dtype=torch.complex128).t(), "Y", 3, 4, torch.complex128)
    with pytest.raises(ValueError, match="CUDA tensor"):
        rid._check_matrix([[0j]], "A", 1, 1, torch.complex128)
    with pytest.raises(ValueError, match="int32 CUDA tensor"):
        rid._check_perm(torch.arange(5, dtype=torch.int32), 5)
    with pytest.raises(ValueError, match="omega"):
        rid._need(False, "omega must be 2 x 3")
    rid._need(True, "never raised")


# ---- the binding's layout checks (CPU tensors; the device check is separate) ----

def _layout(x, rows, cols, exact=False):
    import torch
    import paper_1205_3830_gb300 as rid
    rid._check_layout(x, "x", rows, cols, torch.complex128, exact)
    return rid._ld(x)


def test_layout_accepts_one_row_views_of_any_row_stride():
    import torch
    import paper_1205_3830_gb300 as rid
    # a k = 1 interpolation matrix: 1 x (n - k); torch treats the size-1 dim as
    # contiguous, so as_colmajor may leave stride(0) = n - k
    T = torch.zeros(1, 333 - 1, dtype=torch.complex128)
    assert T.stride() == (332, 1)
    assert _layout(T, 1, 332, exact=True) == 1
    assert _layout(rid.as_colmajor(T), 1, 332, exact=True) == 1
    Tc = torch.zeros(332, 1, dtype=torch.complex128).t()          # (1, 332) with strides (1, 1)
    assert _layout(Tc, 1, 332) == 1


def test_layout_accepts_one_column_views_of_any_column_stride():
    import torch
    x = torch.zeros(7, 1, dtype=torch.complex128)                   # strides (1, 1)
    assert _layout(x, 7, 1) == 7
    y = torch.zeros(5, 7, dtype=torch.complex128).t()[:, :1]        # (7, 1) with strides (1, 7)
    assert _layout(y, 7, 1) == 7


def test_layout_ld_is_the_column_stride_of_a_submatrix():
    import torch
    big = torch.zeros(10, 12, dtype=torch.complex128).t()           # 12 x 10, ld 12
    sub = big[:5, :4]
    assert _layout(sub, 5, 4) == 12


def test_layout_rejects_row_major_and_overlapping_views():
    import torch
    rowmajor = torch.zeros(4, 6, dtype=torch.complex128)
    with pytest.raises(ValueError, match="column-major"):
        _layout(rowmajor, 4, 6)
    col = torch.zeros(4, 1, dtype=torch.complex128)
    expanded = col.expand(4, 6)                                     # stride(1) = 0: every column the same memory
    assert expanded.stride() == (1, 0)
    with pytest.raises(ValueError, match="overlapping"):
        _layout(expanded, 4, 6)
    overlap = torch.zeros(20, dtype=torch.complex128).as_strided((4, 3), (1, 2))
    with pytest.raises(ValueError, match="overlapping"):
        _layout(overlap, 4, 3)


def test_layout_rejects_wrong_shape_and_dtype():
    import torch
    x = torch.zeros(3, 4, dtype=torch.complex128).t()
    with pytest.raises(ValueError, match="must be 3 x 4"):
        _layout(x, 3, 4, exact=True)
    with pytest.raises(ValueError, match="at least"):
        _layout(x, 5, 3)
    with pytest.raises(ValueError, match="complex128"):
        _layout(x.to(torch.complex64), 4, 3)


def test_tc_tuning_size_classes_and_candidates():
    """The autotuner's size classes (m to a power of two, column blocks, N-tiles
    at 128 rows) and its candidate list (K-splits only where the problem has
    twice the chunks)."""
    import paper_1205_3830_gb300 as rid
    T = rid.TcTuning
    assert T.size_class(64, 64, 12) == (256, 1, 1)
    assert T.size_class(257, 129, 64) == (512, 2, 1)
    assert T.size_class(1024, 1000, 65) == (1024, 8, 2)
    assert T.size_class(5000, 300, 40) == (8192, 4, 1)
    small = T.candidates((256, 1, 1))                       # 2 chunks: no K-split
    assert small == [(128, 1), (96, 1), (64, 1)]
    big = T.candidates((1024, 8, 1))                        # 8 chunks: 2 and 4 splits
    assert (64, 4) in big and len(big) == 9
    tun = T(None)
    assert tun.choice(300, 300, 20) == (0, 0)               # untuned class: the defaults
    tun.table[T.size_class(300, 300, 20)] = (96, 2)
    assert tun.choice(300, 300, 20) == (96, 2) and tun.choice(300, 300, 80) == (0, 0)
