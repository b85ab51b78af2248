"""Host logic of bench.py, without a GPU: the `bench-traffic:` lines of the
ncu summaries (traffic per row of the dominant kernel, valid only while the
kernel's source has the hash the line records), the spec list each workload
times, and the median of the end-to-end step timings."""
import hashlib
import os

import pytest

import bench


class _B:
    PAC_COUNT, PAC_SUM, PAC_AVG, PAC_MIN, PAC_MAX = 0, 1, 2, 3, 4
    PAC_EXACT, PAC_APPROX = 0, 1
    PAC_I64 = 0


def _write(root, name, text):
    path = os.path.join(root, name)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        f.write(text)
    return path


@pytest.fixture()
def fake_root(tmp_path, monkeypatch):
    root = str(tmp_path)
    src = _write(root, "csrc/k.cu", "__global__ void k() {}\n")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:12]
    monkeypatch.setattr(bench, "ROOT", root)
    return root, sha


def test_traffic_line_scales_to_the_rows_and_names_the_kernel(fake_root):
    root, sha = fake_root
    _write(root, "profiles/a.md",
           f"text\nbench-traffic: workload=w1 path=5 kernel=k_x kernel_source=csrc/k.cu sha={sha} bytes_per_row=17.5\n")
    assert bench._traffic_kernel("w1", 1000, 5) == (17500.0, "k_x")
    assert bench._traffic("w1", 2000, 5) == 35000.0


def test_traffic_line_without_a_path_is_the_tensor_core_path(fake_root):
    root, sha = fake_root
    _write(root, "profiles/a.md", f"bench-traffic: workload=w2 kernel_source=csrc/k.cu sha={sha} bytes_per_row=4\n")
    assert bench._traffic_kernel("w2", 10, 2) == (40.0, None)
    assert bench._traffic_kernel("w2", 10, 3) == (None, None)


def test_traffic_is_null_once_the_kernel_source_changes(fake_root):
    root, sha = fake_root
    _write(root, "profiles/a.md",
           f"bench-traffic: workload=w3 path=3 kernel=k_y kernel_source=csrc/k.cu sha={sha} bytes_per_row=8\n")
    assert bench._traffic("w3", 10, 3) == 80.0
    _write(root, "csrc/k.cu", "__global__ void k() { /* changed */ }\n")
    assert bench._traffic_kernel("w3", 10, 3) == (None, None)


def test_traffic_is_null_for_a_missing_source_or_workload(fake_root):
    root, sha = fake_root
    _write(root, "profiles/a.md",
           f"bench-traffic: workload=w4 path=3 kernel=k_z kernel_source=csrc/gone.cu sha={sha} bytes_per_row=8\n")
    assert bench._traffic_kernel("w4", 10, 3) == (None, None)
    assert bench._traffic_kernel("other", 10, 3) == (None, None)


def test_committed_traffic_lines_parse():
    # every line in profiles/ names a workload, a source and a positive figure
    import glob
    import re
    pat = re.compile(r"bench-traffic:\s*workload=(\S+)\s+(?:path=(\d+)\s+)?(?:kernel=(\S+)\s+)?kernel_source=(\S+)"
                     r"\s+sha=([0-9a-f]{12})\s+bytes_per_row=([0-9.]+)")
    n = 0
    for f in glob.glob(os.path.join(os.path.dirname(bench.__file__), "profiles", "*.md")):
        for line in open(f):
            if "bench-traffic:" in line:
                m = pat.search(line)
                assert m, line
                assert m.group(1) in bench.WORKLOADS, f
                assert float(m.group(6)) > 0
                assert os.path.exists(os.path.join(os.path.dirname(bench.__file__), m.group(4)))
                n += 1
    assert n >= 1


@pytest.mark.parametrize("xs,want", [([3.0], 3.0), ([5.0, 1.0, 3.0], 3.0), ([4.0, 1.0, 3.0, 2.0], 2.5),
                                     ([21.4, 35.1, 21.3, 21.5], 21.45)])
def test_median_of_step_timings(xs, want):
    assert bench._median(xs) == pytest.approx(want)


def test_spec_lists_of_the_workloads():
    kinds = lambda w: [(k, v) for k, v, *_ in bench._spec_list(_B, bench.WORKLOADS[w], [10, 11, 12, 13],
                                                                 list(range(100, 109)))]
    assert kinds("lowcard_60m") == [(0, 0)] + [(1, 0)] * 4 + [(2, 0)] * 4
    assert kinds("lowcard_60m_approx") == [(0, 0)] + [(1, 1)] * 4 + [(2, 1)] * 4
    assert kinds("ungrouped_1m") == [(0, 0), (1, 0)]
    assert kinds("max_1g") == [(0, 0), (4, 0)]
    for w, cfg in bench.WORKLOADS.items():
        if "aggs" in cfg:
            assert len(bench._spec_list(_B, cfg, [10, 11, 12, 13], list(range(100, 109)))) == bench._n_specs(cfg), w
