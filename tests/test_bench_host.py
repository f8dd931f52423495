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


def test_fft_flop_model_counts_the_pencil_plans():
    # radix-3 and radix-5 butterflies (16 and 48 real flops), complex
    # twiddle products (6): a 15-point pencil is 5 radix-3 butterflies,
    # (3-1)(5-1) twiddles and 3 radix-5 butterflies; a 243 = 27 x 9 pencil
    # has 405 radix-3 butterflies and 568 twiddle products
    assert bench.fft_flops(3) == 16 and bench.fft_flops(5) == 48
    assert bench.fft_flops(15) == 5 * 16 + 8 * 6 + 3 * 48
    assert bench.fft_flops(243) == 405 * 16 + 568 * 6
    f = bench.flops_per_voxel(243)
    assert 850 < sum(f.values()) < 950


def test_cg_roofline_from_kernel_times():
    # 243^3: 100 CG field-iterations, 5 Newton projections, one tangent
    # (12 extra field launches of P2-P4 in FP32); every kernel at 1 ms per
    # field launch gives its algorithmic bytes per millisecond
    V = 243 ** 3
    eff = {"p1_cg": 100, "p5_dot": 100, "cg_update": 100, "p2": 117, "p3": 117, "p4": 117}
    prof = {k + "_f32": (float(n), n + 3) for k, n in eff.items()}
    rf = bench.cg_roofline(prof, 243, 100, 5, 1, "_f32", hbm=1000.0)
    b = bench.bytes_per_voxel(243)
    for k in eff:
        assert rf["kernels"][k]["ms"] == 1.0
        assert abs(rf["kernels"][k]["GB/s"] - b[k + "_f32"] * V / 1e-3 / 1e9) < 0.1
    assert rf["matvec"]["ms_per_field_iter"] == 5.0 and rf["iteration"]["ms_per_field_iter"] == 6.0
    assert abs(rf["iteration"]["bytes_per_voxel"] - 460.8) < 0.2


def test_cg_roofline_of_the_fused_iteration():
    # the mixed path: P1 (with <p, C:p>), P2-P4, P5 (r update), cg_rr; the
    # iteration moves 388.8 B/voxel at 243^3 and the matvec is P1-P5
    eff = {"p1_cgf": 100, "p5_cgf": 100, "cg_rr": 100, "p2": 117, "p3": 117, "p4": 117}
    prof = {k + "_f32": (float(n), n) for k, n in eff.items()}
    rf = bench.cg_roofline(prof, 243, 100, 5, 1, "_f32", hbm=1000.0)
    assert set(rf["kernels"]) == set(eff)
    assert rf["matvec"]["ms_per_field_iter"] == 5.0 and rf["iteration"]["ms_per_field_iter"] == 6.0
    assert abs(rf["iteration"]["bytes_per_voxel"] - 388.8) < 0.2
    assert rf["matvec"]["bytes_per_voxel"] == rf["iteration"]["bytes_per_voxel"]
