"""Host-side helpers of bench.py that shape the reported roofline (no GPU): the cell-build byte
count, the HBM peak it is measured against, and the tie between a traffic capture and the source
files of the kernel it measured."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_cell_build_bytes_and_fraction(bench):
    peak, src = bench.hbm_peak_gbs()
    assert peak > 0 and src
    r = bench.cell_build_roof(1000, 500, 3, 0.001)
    assert r["bytes_per_build"] == 1000 * (8 * 3 + 52) + 500 * 24
    assert r["achieved"] == pytest.approx(r["bytes_per_build"] / 1e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert bench.cell_build_roof(10, 0, 2, 1.0)["bytes_per_build"] == 10 * 68


def test_traffic_entries_resolve_to_their_kernel_sources(bench):
    # every recorded capture names an existing profile that records its digest, and a known kernel
    # family; while that family's sources are unchanged the line reports the capture's bytes
    for (workload, walk), (nbytes, profile, family, digest) in bench.TRAFFIC_PER_LAUNCH.items():
        assert os.path.exists(os.path.join(ROOT, profile)), profile
        assert family in bench.KERNEL_FILES
        with open(os.path.join(ROOT, profile)) as f:
            assert digest in f.read(), profile
        value, note = bench.traffic_entry(workload, walk)
        if digest == bench.kernel_digest(family):
            assert value == nbytes and digest in note, (workload, note)
        else:
            assert value is None and note.startswith("stale"), (workload, note)


def test_traffic_entry_goes_null_when_the_sources_change(bench, monkeypatch):
    key = next(iter(bench.TRAFFIC_PER_LAUNCH))
    nbytes, profile, family, digest = bench.TRAFFIC_PER_LAUNCH[key]
    monkeypatch.setitem(bench.TRAFFIC_PER_LAUNCH, key, (nbytes, profile, family, "0" * 16))
    value, note = bench.traffic_entry(*key)
    assert value is None and note.startswith("stale")
    assert bench.traffic_entry("no-such-workload", None)[0] is None
    # the digest depends on every file of the family and on nothing else
    assert bench.kernel_digest("field") != bench.kernel_digest("pair")
