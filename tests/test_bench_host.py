"""Host logic of the benchmark (no GPU): the DRAM-traffic lookup in the ncu
summaries and the spec list each workload times."""
import os

import bench


class _B:
    PAC_COUNT, PAC_SUM, PAC_AVG, PAC_MIN, PAC_MAX = 0, 1, 2, 3, 4
    PAC_EXACT, PAC_APPROX = 0, 1
    PAC_I64 = 0


def _write_profile(root, line):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", "k_test.md"), "w") as f:
        f.write("# a summary\n\n" + line + "\n")


def test_traffic_follows_source_hash_and_path(tmp_path, monkeypatch):
    root = str(tmp_path)
    src = os.path.join(root, "k.cu")
    with open(src, "w") as f:
        f.write("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", root)
    sha = bench._source_sha("k.cu")
    _write_profile(root, f"bench-traffic: workload=w1 path=4 kernel_source=k.cu sha={sha} bytes_per_row=16.5")
    assert bench._traffic("w1", 1000, 4) == 16500.0
    assert bench._traffic("w1", 1000, 2) is None        # another aggregation path
    assert bench._traffic("w2", 1000, 4) is None        # another workload
    # a line without a path is the tensor-core path's
    _write_profile(root, f"bench-traffic: workload=w1 kernel_source=k.cu sha={sha} bytes_per_row=41.0")
    assert bench._traffic("w1", 10, 2) == 410.0
    # the kernel source changed since the counters were taken: no traffic
    with open(src, "a") as f:
        f.write("// edited\n")
    assert bench._traffic("w1", 10, 2) is None


def test_committed_traffic_lines_parse():
    """Every committed bench-traffic line names an existing source file."""
    import glob
    import re
    pat = re.compile(r"bench-traffic:\s*workload=(\S+)\s+(?:path=(\d+)\s+)?kernel_source=(\S+)\s+sha=(\S+)")
    found = 0
    for f in glob.glob(os.path.join(bench.ROOT, "profiles", "*.md")):
        for line in open(f):
            m = pat.search(line)
            if m:
                found += 1
                assert m.group(1) in bench.WORKLOADS, f
                assert os.path.exists(os.path.join(bench.ROOT, m.group(3))), f
    assert found >= 2


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
