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
    h = bench.kernel_source_hash()
    for name in ("grouped_3xbf16_uneven200k.md", "grouped_ffma_uneven200k.md",
                 "grouped_zgemm_uneven-c64100k.md"):
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        assert "kernel_source_hash: " in txt and "ncu --set full --clock-control none" in txt, name
        current = f"kernel_source_hash: {h}" in txt
        traffic = bench.profile_traffic(*{"grouped_3xbf16_uneven200k.md": ("3xbf16",),
                                         "grouped_ffma_uneven200k.md": ("ffma",),
                                         "grouped_zgemm_uneven-c64100k.md": ("zgemm", "uneven-c64", 100_000)}[name])
        assert (traffic is not None and traffic > 0) == current, name
