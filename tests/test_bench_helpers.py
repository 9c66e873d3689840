"""Host-side pieces of bench.py (no GPU): the committed traffic capture is
used only while the traversal sources hash to the recorded value and the
chain count matches; the input byte counts of flat and instanced uploads;
the workload table's scene sizes; the reference arm's line (the FP64 oracle
on the host cores) and the bounded CPU-baseline sample."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2605_08916_gb300 import scenes as S  # noqa: E402


def test_traffic_capture_is_tied_to_the_sources_and_the_chain_count():
    kv = {}
    with open(os.path.join(ROOT, "profiles", "wf_traverse_traffic_procedural-1m-720p.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#") and ":" in line:
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    import hashlib
    h = hashlib.sha256()
    for f in bench.TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2605_08916_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    t = bench.traversal_traffic("procedural-1m-720p", int(kv["chains"]))
    if h.hexdigest() == kv["source_sha256"]:
        assert t == int(kv["dram_read_bytes_per_step"]) + int(kv["dram_write_bytes_per_step"])
    else:  # sources changed since the capture: no traffic figure
        assert t is None
    assert bench.traversal_traffic("procedural-1m-720p", int(kv["chains"]) // 2) is None
    assert bench.traversal_traffic("no-such-workload", 1) is None


def test_input_bytes_of_flat_and_instanced_uploads():
    isc = S.procedural_scene_instanced(1, 32, 18, target_tris=6000, n_objects=6, terrain_chunks=2)
    flat = isc.flatten()
    nb_flat = bench.input_bytes(flat)
    assert nb_flat == sum(a.nbytes for a in (flat.verts, flat.tris, flat.tri_mat, flat.materials, flat.camera,
                                              flat.normals))
    nb_inst = bench.input_bytes(isc)
    assert 0 < nb_inst < nb_flat  # the unit sphere and box are shared by their instances
    assert bench.flat_of(isc).n_tris == isc.n_tris == flat.n_tris


def test_workload_table():
    assert bench.DEFAULT in bench.WORKLOADS
    wl = bench.WORKLOADS["cornell-64-fd"]
    sc = wl["scene"]()
    assert (sc.width, sc.height, sc.n_tris) == (64, 64, 34) and wl["drift"] == "fd" and wl["L"] == 4
    for name, w in bench.WORKLOADS.items():
        assert w["chains"] > 0 and 1 <= w["L"] <= 16 and w["spp"] >= 1, name


def _run_bench(args, env_extra=None):
    import json
    import subprocess
    env = dict(os.environ)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_line():
    """The reference arm (the FP64 oracle on the host cores) prints one line
    with the contract's keys, on the workload and metric of the GPU arm."""
    (line,) = _run_bench(["--impl", "reference", "--workload", "cornell-64-fd", "--steps", "3", "--warmup", "3"])
    for k in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"]:
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 3 and line["warmup"] == 3 and line["value"] > 0 and line["higher_is_better"]
    assert line["config"]["workload"] == "cornell-64-fd"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm; the others exit 0
    without work and print no line."""
    env = {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2", "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": "29999"}
    assert _run_bench(["--impl", "reference", "--workload", "cornell-64-fd", "--steps", "3", "--warmup", "3"],
                      env) == []


def test_cpu_baseline_reports_a_bounded_sample():
    wl = bench.WORKLOADS["cornell-64-fd"]
    cb = bench.cpu_baseline(wl, wl["scene"](), steps=2, target_s=0.2)
    assert cb["kind"] == "oracle" and cb["unit"] == bench.UNIT and cb["value"] > 0 and cb["cores"] >= 1
    assert cb["seconds"] < 30 and "chains x 3 steps" in cb["sample"]


def test_measured_peaks_reads_the_file_or_falls_back(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")            # absent
    (tmp_path / "MEASURED_PEAKS.json").write_text("{not json")
    assert bench.measured_peaks() == (6800.0, "fallback")            # malformed
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"bf16_tflops": 1800}')
    assert bench.measured_peaks() == (6800.0, "fallback")            # no HBM figure
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6785.9}')
    assert bench.measured_peaks() == (6785.9, "measured")


def test_relmse_split_into_bias_and_variance():
    """Images I_s = R + b + noise_s (noise of variance v per pixel): the
    split returns bias2 = mean b^2 w and variance = v mean w (w = 1 / (R^2 +
    1e-2)), and they add up to the mean relMSE over seeds."""
    rng = np.random.default_rng(4)
    ref = rng.uniform(0.1, 2.0, (8, 12, 3))
    w = 1.0 / (ref ** 2 + 1e-2)
    bias = 0.05 * ref
    v = 0.01
    imgs = [ref + bias + rng.normal(size=ref.shape) * np.sqrt(v) for _ in range(400)]
    rm, sd, b2, var = bench.bias_variance(imgs, ref)
    assert abs(var / (v * w.mean()) - 1) < 0.05
    assert abs(b2 / np.mean(bias ** 2 * w) - 1) < 0.05
    assert abs(rm - (b2 + var)) < 0.02 * rm
    # no bias: the squared bias is (up to noise) zero, all of it variance
    rm, sd, b2, var = bench.bias_variance([ref + rng.normal(size=ref.shape) * 0.1 for _ in range(400)], ref)
    assert b2 < 0.01 * var
