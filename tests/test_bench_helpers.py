"""Host-side pieces of bench.py (no GPU): the committed traffic capture is
used only while the traversal sources hash to the recorded value and the
chain count matches; the input byte counts of flat and instanced uploads;
the workload table's scene sizes."""
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
