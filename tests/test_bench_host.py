"""Host logic of bench.py that needs no GPU: the DRAM traffic it reports comes from an ncu summary
only when that summary was taken on the kernel sources built here."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_digest_is_stable_and_covers_the_stepping_kernels():
    d = bench.kernel_sources_digest()
    assert len(d) == 64 and int(d, 16) >= 0
    assert bench.kernel_sources_digest() == d


def test_traffic_is_reported_only_for_matching_sources(tmp_path):
    key = ("k_resid", "shell_331776_p3", "fp32")
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps({"sources_sha256": bench.kernel_sources_digest(), "k_resid:shell_331776_p3:fp32": 1.5e9}))
    assert bench.lookup_traffic(str(f), *key) == 1.5e9
    assert bench.lookup_traffic(str(f), "k_grad", "shell_331776_p3", "fp32") is None
    f.write_text(json.dumps({"sources_sha256": "0" * 64, "k_resid:shell_331776_p3:fp32": 1.5e9}))
    assert bench.lookup_traffic(str(f), *key) is None  # counters of other kernel sources
    f.write_text(json.dumps({"k_resid:shell_331776_p3:fp32": 1.5e9}))
    assert bench.lookup_traffic(str(f), *key) is None  # no digest recorded
    assert bench.lookup_traffic(str(tmp_path / "missing.json"), *key) is None
