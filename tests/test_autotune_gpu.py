"""The autotuner (the GPU counterpart of the paper's install-time tuning):
it times the register-tile variants, the stage size and the kernel family of
default FP32 plans on this GPU, writes a JSON cache, and plans made with the
tuned model stay correct."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2208_09822_gb300 import iaat
from paper_2208_09822_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_09822_gb300 import build
    build.build()
    return torch


def autotune(path, *precisions):
    """Tune in a child process: iaat_autotune also applies the result to the
    process that calls it, which would change the default plans of every
    later test in this one."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2208_09822_gb300 import iaat\n"
            "for p in %r:\n"
            "    iaat.iaat_autotune(iaat.IAAT_F32, p, %r)\n" % (ROOT, list(precisions), path))
    env = dict(os.environ)
    env.pop("IAAT_TUNE_CACHE", None)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr


def test_autotune_writes_cache_and_tuned_plans_stay_correct(tmp_path):
    path = str(tmp_path / "tune.json")
    autotune(path, iaat.IAAT_PREC_DEFAULT, iaat.IAAT_PREC_3XBF16, iaat.IAAT_PREC_FP16)
    cache = json.load(open(path))
    assert len(cache["variant_scale_f32"]) == 5
    assert all(v > 0 for v in cache["variant_scale_f32"])
    assert cache["group_tasks_ffma"] in (8, 16, 24, 32)
    assert cache["group_tasks_3xbf16"] in (8, 16, 24, 32)
    # the kernel family each default plan runs: stage programs, stream or
    # warp-direct for FP32 on the CUDA cores, stage programs, stream or
    # warp-tile for the tensor-core paths
    assert cache["kernel_ffma"] in (1, 2, 4)
    assert cache["kernel_3xbf16"] in (1, 2, 3) and cache["kernel_fp16"] in (1, 2, 3)
    # a fresh process reads the cache through IAAT_TUNE_CACHE and still
    # matches the oracle
    code = (
        "import sys; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
        "from paper_2208_09822_gb300 import workloads as W\n"
        "from tests.gpu_util import run_grouped, compare\n"
        "b = W.random_small(1500, seed=91, max_dim=60, pad_max=3)\n"
        "import numpy as np\n"
        "b = b.select(np.nonzero(W.in_domain(b.M, b.N, b.K, b.transA, b.transB))[0])\n"
        "fam = %r\n"
        "for prec, tol in ((0, 1e-5), (1, 1e-5), (3, 1e-3)):\n"
        "    C, info = run_grouped(b, prec)\n"
        "    assert info['kernel_family'] == fam[prec], (prec, info)\n"
        "    e = compare(b, C)\n"
        "    assert e['eps_batch'] <= tol, e\n"
        "print('ok')\n" % (ROOT, ROOT, {0: cache["kernel_ffma"], 1: cache["kernel_3xbf16"], 3: cache["kernel_fp16"]}))
    env = dict(os.environ, IAAT_TUNE_CACHE=path)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


def test_cache_applies_only_on_the_gpu_it_was_measured_on(tmp_path):
    """The cache names the GPU, its SM count and compute capability, the
    driver and the CUDA runtime; a process applies it only when all match.
    A cache forcing 8 tasks per stage changes the plan's stage count; the
    same cache with another device name is ignored."""
    path = str(tmp_path / "tune.json")
    autotune(path, iaat.IAAT_PREC_DEFAULT)
    cache = json.load(open(path))
    for key in ("device", "sm_count", "compute_capability", "driver_version", "runtime_version"):
        assert key in cache, key
    forced = dict(cache, group_tasks_ffma=8, kernel_ffma=1)
    other = dict(forced, device=cache["device"] + " (another GPU)")
    paths = {}
    for name, c in (("forced", forced), ("other", other)):
        paths[name] = str(tmp_path / f"{name}.json")
        json.dump(c, open(paths[name], "w"))
    code = (
        "import sys; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
        "from paper_2208_09822_gb300 import workloads as W, iaat\n"
        "from tests.gpu_util import to_device\n"
        "b = W.uneven(count=3000, seed=5)\n"
        "tA, tB, tC, d = to_device(b)\n"
        "print(iaat.iaat_plan_info(iaat.iaat_plan_create(d, iaat.IAAT_F32))['groups'])\n" % (ROOT, ROOT))
    groups = {}
    for name in ("forced", "other", None):
        env = dict(os.environ)
        env.pop("IAAT_TUNE_CACHE", None)
        if name:
            env["IAAT_TUNE_CACHE"] = paths[name]
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stdout + r.stderr
        groups[name] = int(r.stdout.strip().splitlines()[-1])
    assert groups["other"] == groups[None]
    assert groups["forced"] > groups[None]
