"""The benchmark's contract pieces that run without a GPU: the reference arm
(the FP64 oracle on the host cores) prints one JSON line with the contract's
keys, and the committed profiles are found for the kernel sources they were
taken on."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload", ["uneven", "uneven-c64"])
def test_reference_arm_prints_the_contract_line(workload):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          workload, "--instances", "2000", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "gpu_launches"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert workload.split("-")[0] in line["config"]["workload"]


def test_profiles_name_their_sources_and_command():
    """Every committed kernel profile names the hash of the kernel sources it
    was captured on (the bench reports its traffic only while that hash is
    the current one, null after any kernel change) and the ncu command."""
    sys.path.insert(0, ROOT)
    import bench
    for name in ("grouped_3xbf16_uneven200k.md", "grouped_ffma_uneven200k.md",
                 "grouped_zgemm_uneven-c64100k.md", "grouped_3xbf16-r32d_uneven200k.md"):
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        ncu = [ln for ln in txt.splitlines() if ln.startswith("ncu ")]
        assert "kernel_source_hash: " in txt and ncu, name
        assert all("--clock-control none" in ln and "--set full" in ln for ln in ncu), name
        args = {"grouped_3xbf16_uneven200k.md": ("3xbf16",), "grouped_ffma_uneven200k.md": ("ffma",),
                "grouped_zgemm_uneven-c64100k.md": ("zgemm", "uneven-c64", 100_000),
                "grouped_3xbf16-r32d_uneven200k.md": ("3xbf16-r32d",)}[name]
        current = f"kernel_source_hash: {bench.kernel_source_hash(args[0])}" in txt
        traffic = bench.profile_traffic(*args)
        assert (traffic is not None and traffic > 0) == current, name


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_split_bookkeeping(world):
    """bench.py --split shard: the ranks' instance ranges cover the batch once,
    in order; their flops add up to the batch's; each rank's pool spans hold
    exactly the elements of its instances (what it copies end to end); and
    no rank gets much more than its share of the estimated cost."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    from paper_2208_09822_gb300 import workloads as W
    from paper_2208_09822_gb300.shard import instance_cost
    b = W.uneven(count=5000, seed=2)
    ranges = bench.shard_ranges(b, world)
    assert len(ranges) == world
    assert ranges[0]["i0"] == 0 and ranges[-1]["i1"] == b.count
    for r, s in zip(ranges, ranges[1:]):
        assert r["i1"] == s["i0"]
    assert sum(r["flops"] for r in ranges) == b.flops()
    cost = instance_cost(b.M, b.N, b.K, b.beta != 0, b.esize)
    for r in ranges:
        for name, pool in (("A", b.A), ("B", b.B), ("C", b.C)):
            lo, hi = r[name]
            rows, cols, ld, off = b.storage(name)
            idx = np.arange(r["i0"], r["i1"])
            if len(idx):
                first = off[idx]
                last = off[idx] + np.maximum(cols[idx] - 1, 0) * ld[idx] + rows[idx]
                assert lo <= first.min() and last.max() <= hi
            assert 0 <= lo <= hi <= pool.size
        assert cost[r["i0"]:r["i1"]].sum() <= cost.sum() / world + cost.max()


def test_bench_paths_resolve():
    """Every bench path names a precision the planner takes, a kernel family
    its precision allows (warp-tile for the tensor cores only, warp-direct
    for the CUDA cores only), a CUDA-core family for a routed part, and
    translation units that exist (so its profile hash covers real sources)."""
    sys.path.insert(0, ROOT)
    import bench
    csrc = os.path.join(ROOT, "paper_2208_09822_gb300", "csrc")
    for name, prec in bench.PRECISIONS.items():
        assert prec in (0, 1, 2, 3, 4), name
        k = bench.KERNEL[name]
        assert k in (0, 1, 2, 3, 4), name
        assert not (k == 3 and prec == 0) and not (k == 4 and prec != 0), name
        base = bench.ROUTE_BASE(name)
        if base in bench.ROUTE:
            rk, rm, rf = bench.ROUTE[base]
            assert prec != 0 and rk >= 0 and rm >= 0 and rf in (0, 1, 2, 4), name
        assert os.path.exists(os.path.join(csrc, bench.kernel_unit(name))), name
        assert len(bench.kernel_source_hash(name)) == 16, name
    # the headline is a routed tensor-core path with its small part on the
    # warp-direct kernel; its hash covers both kernels' sources
    assert bench.ROUTE["3xbf16-r32d"] == (8, 32 ** 3, 4)
    assert bench.kernel_source_hash("3xbf16-r32d") != bench.kernel_source_hash("3xbf16")
