"""Host logic of bench.py that needs no GPU: the algorithmic byte model of
the CG kernels and the gate that keeps a captured DRAM traffic figure only
while the kernel sources are unchanged."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_byte_model_of_a_cg_iteration():
    # 243^3, FP32 fields: 6 components (small strain), 9 (finite strain)
    b = bench.bytes_per_voxel(243)
    it = sum(b[k] for k in ("p1_cg_f32", "p2_f32", "p3_f32", "p4_f32", "p5_dot_f32", "cg_update_f32"))
    assert abs(it - 460.8) < 0.1
    f = bench.fs_bytes_per_voxel(243)
    it = sum(f[k] for k in ("fs_p1_cg_f32", "fs_p2_f32", "fs_p3_f32", "fs_p4_f32", "fs_p5_dot_f32",
                            "fs_cg_update_f32"))
    assert abs(it - 686.1) < 0.2


def test_traffic_gate_ignores_comments_but_not_code():
    src = b"// header\nint a = 1; /* note */\n\n  // more\nint b = 2;\n"
    same = b"int a = 1;\n// another comment\nint b = 2;   \n"
    other = b"int a = 1;\nint b = 3;\n"
    assert bench._strip_comments(src) == bench._strip_comments(same)
    assert bench._strip_comments(src) != bench._strip_comments(other)


def test_captured_traffic_is_kept_only_for_its_sources(monkeypatch):
    for kind, tr in bench.TRAFFIC.items():
        # no re-reads: at most the algorithmic bytes (L2 may hold a little)
        alg = bench.bytes_per_voxel(tr["N"]).get(kind) or bench.fs_bytes_per_voxel(tr["N"]).get(kind)
        assert 0.9 * alg * tr["N"] ** 3 <= tr["bytes"] <= alg * tr["N"] ** 3
        assert bench.measured_traffic(kind, 135) is None            # other grid
        if tr["digest"] == bench.kernel_digest(tr["files"]):
            assert bench.measured_traffic(kind, tr["N"]) == tr["bytes"]
        changed = dict(bench.TRAFFIC)
        changed[kind] = dict(tr, digest="0" * 16)                   # sources changed since
        monkeypatch.setattr(bench, "TRAFFIC", changed)
        assert bench.measured_traffic(kind, tr["N"]) is None
        monkeypatch.undo()
