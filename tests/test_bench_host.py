"""Host logic of bench.py that needs no GPU: the DRAM traffic it reports next
to a roofline comes from a committed ncu summary and must follow the kernel
sources it was taken on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_source_hash_is_stable_and_depends_on_the_files():
    a = bench.src_hash()
    assert a == bench.src_hash() and len(a) == 16
    assert bench.src_hash(bench.MLP_SOURCES) != a


def test_forward_traffic_scales_with_rows_and_follows_the_source(monkeypatch):
    t1 = bench.read_mlp_traffic(1 << 20)
    if t1 is None:
        pytest.skip("the committed forward profile is not of the current kernel source")
    assert t1 > 0
    # the features are read once: a launch over four times the rows moves four times the bytes
    assert bench.read_mlp_traffic(4 << 20) == pytest.approx(4 * t1, rel=1e-6)
    monkeypatch.setattr(bench, "src_hash", lambda files=None: "0" * 16)
    assert bench.read_mlp_traffic(1 << 20) is None


def test_search_traffic_follows_the_source(monkeypatch):
    t = bench.read_traffic()
    if t is None:
        pytest.skip("the committed search profile is not of the current kernel source")
    assert t > 0
    monkeypatch.setattr(bench, "src_hash", lambda files=None: "0" * 16)
    assert bench.read_traffic() is None
