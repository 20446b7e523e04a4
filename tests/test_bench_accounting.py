"""bench.py's roofline accounting, without a GPU.

The algorithmic bytes of a solve (initial X read, five window arrays per
iteration, the final L write) and the way the committed ncu DRAM traffic is
matched to the device code and scaled to a launch's windows.
"""
import json
import os
import shutil

import bench


def test_solve_bytes_follow_the_iteration():
    m, T = 262144, 20
    unit = m * T * 4
    # initial pass reads X, every iteration reads X, S, Y and writes S', Y', the final step writes L (plus a mask byte
    # per pixel)
    got = bench._solve_bytes(m, T, 32)
    assert got in ((1 + 5 * 32 + 1) * unit, (1 + 5 * 32 + 1) * unit + m)


def test_traffic_entries_count_only_for_their_kernel_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash()
    (prof / "ncu_traffic.json").write_text(json.dumps({
        "batch_kernel": {"kernel_source_sha256": h, "iters_per_window": 32, "dram_bytes_per_window_solve": 1620},
        "fused_pass": {"kernel_source_sha256": "0" * 16, "dram_bytes_per_launch": 5},
        "batch_kernel_tc_tf32x3": {"kernel_source_sha256": h, "iters_per_window": 32,
                                   "dram_bytes_per_window_solve": 3240},
    }))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # one window at the captured iteration count gets the captured bytes; more iterations scale them by the
    # window arrays moved: (1 + 5 it + 5) / (1 + 5 it0 + 5)
    assert bench.ncu_batch_traffic(h, [32]) == 1620
    assert abs(bench.ncu_batch_traffic(h, [32, 38]) - (1620 + 1620 * (1 + 5 * 38 + 5) / (1 + 5 * 32 + 5))) < 1e-9
    assert bench.ncu_batch_traffic(h, [32], "batch_kernel_tc_tf32x3") == 3240
    # another device-code hash, or an entry taken on other code, gives no traffic
    assert bench.ncu_batch_traffic("f" * 16, [32]) is None
    assert bench.ncu_traffic(h) is None
    assert bench.ncu_batch_traffic(h, [32], "missing") is None


def test_kernel_source_hash_covers_the_narrow_headers(tmp_path, monkeypatch):
    csrc = os.path.join(os.path.dirname(bench.__file__), "paper_2506_10257_gb300", "csrc")
    heads = [f for f in os.listdir(csrc) if f.endswith(".cuh")]
    assert "rpca_kernels.cuh" in heads and "rpca_batch.cuh" in heads
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    # on a copy of the headers: editing a tiled header keeps the hash, editing
    # a narrow one (or adding a header) changes it
    dst = tmp_path / "paper_2506_10257_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in heads:
        shutil.copy(os.path.join(csrc, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_source_hash() == h
    for f in bench.TILED_HEADERS:
        with open(dst / f, "a") as fh:
            fh.write("// edited\n")
    assert bench.kernel_source_hash() == h
    with open(dst / "rpca_kernels.cuh", "a") as fh:
        fh.write("// edited\n")
    h2 = bench.kernel_source_hash()
    assert h2 != h
    (dst / "rpca_new.cuh").write_text("// a new narrow header\n")
    assert bench.kernel_source_hash() not in (h, h2)
