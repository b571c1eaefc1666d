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
