"""Host logic of the benchmark: the algorithmic byte models behind the
roofline fraction, checked against counts worked out by hand from the data
layout (float32 SoA m of 12 B per cell, complex64 half spectra holding only
the valid rows, the real kernel on its symmetric octant), and the rule that
the measured DRAM traffic is reported only for the sources it was taken on."""

import json
import os

import bench

N2 = 1024 * 1024


def test_film_pass_bytes_by_hand():
    ab = bench.algorithmic_bytes(1024, 1024)
    m = 12 * N2
    spec = 3 * 1025 * 1024 * 8        # [c][kx][y], Hx = 2048/2 + 1, the 1024 valid rows
    kern = 4 * 1025 * 1025 * 4        # xx, yy, zz, xy on kx, ky >= 0
    assert ab["k_colconv_y"] == 2 * spec + kern
    assert ab["k_xfwd"] == spec + 3 * m              # reads m_n, k1; writes m_2 and its spectrum
    assert ab["k_xinv_h"] == spec + m                # spectrum in, H_demag out
    assert ab["k_xfwd_next"] == m + spec
    # stage s = 2..6 of the fused x pass: spectrum in, m_s with halo, m_n and
    # k_1..k_{s-1} (k_2 has weight 0 from stage 6 on), k_s and m_{s+1} out,
    # next spectrum out; stage 7: m_7, k_1, k_3..k_6 in, k_7 out
    reads = [2, 3, 4, 5, 5]
    assert ab["k_xinv_local_fused"] == sum(2 * spec + m * (1 + r + 2) for r in reads) / 5
    assert ab["k_xinv_local"] == spec + m + 5 * m + m
    # a Dormand-Prince step: one x forward, six column passes, five fused and one final x pass
    assert ab["step"] == ab["k_xfwd"] + 6 * ab["k_colconv_y"] + 5 * ab["k_xinv_local_fused"] + ab["k_xinv_local"]
    assert 199.0 < ab["step"] / (6 * N2) < 201.0     # about 200 B per cell-evaluation


def test_cube_pass_bytes_by_hand():
    # 256 x 256 x 64, periodic in x and y (no padding there), open z padded to 128
    ab = bench.algorithmic_bytes_3d((256, 256, 64), 128, (True, True, False), axes=True)
    N = 256 * 256 * 64
    m = 12 * N
    s1 = 3 * 129 * 64 * 256 * 8       # x spectrum [c][kx][z][y]: 50.7 MB
    s2 = 3 * 129 * 256 * 64 * 8       # y spectrum [c][kx][ky][z]
    kern = 6 * 129 * 129 * 65 * 4     # six components on the kx, ky, kz >= 0 octant
    assert s1 == 50724864
    assert ab["k_yfwd"] == s1 + s2 and ab["k_yinv"] == s2 + s1
    assert ab["k_colconv_z"] == 2 * s2 + kern
    heun1 = s1 + m + 2 * m + s1 + m   # spectrum, m_n + halo, k1 and predictor out, next spectrum, axes
    heun2 = s1 + m + 3 * m + s1 + m   # as heun1 plus m_{n+1} out
    assert ab["k_xinv_local_fused"] == (heun1 + heun2) / 2
    assert ab["step"] == 2 * (2 * (s1 + s2) + 2 * s2 + kern) + heun1 + heun2


def test_rk_3d_step_bytes_reduce_to_the_passes():
    # the ensemble's 3-D samples: open in all three axes; up to 8 z cells the
    # y and z stages are one pass over the x spectrum, beyond they go through
    # the z-padded spectrum s2
    for nz, pz in ((3, 8), (12, 32)):
        nx, ny = 40, 30
        N = nx * ny * nz
        m = 12 * N
        hx = nx + 1
        s1 = 3 * hx * nz * ny * 8
        s2 = 3 * hx * 2 * ny * nz * 8
        kern = 6 * hx * (ny + 1) * (pz // 2 + 1) * 4
        col = 2 * s1 + kern if nz <= 8 else 2 * (s1 + s2) + 2 * s2 + kern
        reads = [2, 3, 4, 5, 5]
        fused = sum(2 * s1 + m * (1 + r + 2) for r in reads)
        final = s1 + 7 * m
        assert bench.algorithmic_bytes_rk_3d((nx, ny, nz))["step"] == (s1 + 3 * m) + 6 * col + fused + final


def test_traffic_is_reported_only_for_the_profiled_sources(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    kernel = next(iter(rec["kernels"]))
    monkeypatch.setattr(bench, "_source_hash", lambda: "not-these-sources")
    assert bench._traffic_for(kernel) is None
    monkeypatch.setattr(bench, "_source_hash", lambda: rec["source_hash"])
    v = bench._traffic_for(kernel)
    assert v is not None and v > 0
