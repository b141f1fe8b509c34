"""CPU checks of bench.py's host-side helpers: the roofline's DRAM traffic
and pipe activity are read from the committed ncu summaries, so those must
stay parseable and match the tables they summarise."""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_helpers", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_profile_figures_are_parsed():
    b = _bench()
    traffic = b.sweep_traffic_from_profiles()
    assert traffic is not None and 1e7 < traffic < 1e9
    fma = b.sweep_pipe_from_profiles()
    fp64 = b.sweep_pipe_from_profiles("sweep_fp64_riemann1024.md", "FP64")
    assert fma is not None and 0.3 < fma < 1.0
    assert fp64 is not None and 0.5 < fp64 < 1.0


def test_sweep_traffic_matches_the_launch_list():
    """The traffic figure of the sweep summary is the launch list's mean DRAM
    bytes per float32 sweep launch (within the rounding of the summaries)."""
    b = _bench()
    text = open(os.path.join(ROOT, "profiles", "launch_list_riemann1024.md")).read()
    m = re.search(r"mean ([0-9.]+) MB and [0-9.]+ ms per float32 sweep launch", text)
    assert m, "launch list lacks the mean per sweep launch"
    assert abs(b.sweep_traffic_from_profiles() / 1e6 - float(m.group(1))) <= 0.1


def test_host_info_reports_cores():
    b = _bench()
    info = b.host_info()
    cores = info[0] if isinstance(info, tuple) else info.get("cores")
    assert cores >= 1
