"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Sizes span several tiles and ragged edges; kernels cover disks at every workload radius
that fits the oracle's time, the workload hexagon and ellipse, asymmetric and even-n span
kernels, and the degenerate cases (1x1, one row, one column, radius 0, constant images,
the adversarial checkerboard). The tolerance is 0: the output is a selected input value.
"""
import numpy as np
import pytest

import datagen
import oracle
from helpers import assert_bit_exact, fim_kernel, gpu_filter, oracle_offsets

pytestmark = pytest.mark.gpu

NP = {"u8": np.uint8, "u16": np.uint16, "f32": np.float32}


def run_case(img, kind, *args, pitch_elems=None, percentile=None):
    k = fim_kernel(kind, *args)
    off = oracle_offsets(kind, *args)
    assert k.info["ntaps"] == len(off)
    rank = None if percentile is None else oracle.percentile_rank(len(off), percentile)
    got = gpu_filter(img, k, pitch_elems=pitch_elems, percentile=percentile)
    exp = oracle.median_filter(img, off, rank=rank)
    assert_bit_exact(got, exp, f"{kind}{args} {img.dtype} {img.shape}")


def test_config1_full():
    """u8 256x256 uniform, disk r=4 (49 taps), whole image."""
    run_case(datagen.config1_image(), "circle", 4)


@pytest.mark.parametrize("r", [1, 2, 3, 8, 16, 32, 48])
def test_u16_photo_crops(r):
    img = datagen.config2_image(4096, 4096)[1000:1000 + 203, 2000:2000 + 217]
    run_case(np.ascontiguousarray(img), "circle", r)


@pytest.mark.parametrize("tile", ["64,64,8,2", "32,32,2,1", "32,16,2,2", "64,32,4,2"])
@pytest.mark.parametrize("r", [3, 8, 20])
def test_u16_sort_paths(tile, r, monkeypatch):
    """16-bit data sorts by the 65536-bin counting sort in 1024-thread CTAs and by two radix
    passes in smaller CTAs; both must give the oracle's result on the same crop."""
    monkeypatch.setenv("FIM_TILE", tile)
    img = datagen.config2_image(4096, 4096)[1500:1500 + 131, 700:700 + 149]
    run_case(np.ascontiguousarray(img), "circle", r)


@pytest.mark.parametrize("tile", ["32,32,2,1", "32,64,4,1"])
@pytest.mark.parametrize("dtype", ["u16", "f32"])
def test_radix_small_cta_wide_box(tile, dtype, monkeypatch):
    """Radix sort in a small CTA with a footprint box wider than 255 (32-bit entries and
    positions, lists in the CTA's global slice)."""
    monkeypatch.setenv("FIM_TILE", tile)
    img = datagen.image_for(dtype, datagen.seed_for(3, 11), 97, 83)
    run_case(img, "circle", 115)


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
@pytest.mark.parametrize("r", [5, 21])
def test_dtypes_ragged(dtype, r):
    img = datagen.image_for(dtype, 100 + r, 141, 167)
    run_case(img, "circle", r)


@pytest.mark.parametrize("r", [24, 40, 64])
def test_f32_disks(r):
    img = datagen.image_for("f32", 300 + r, 120, 133)
    run_case(img, "circle", r)


def test_f32_hexagon64():
    img = datagen.image_for("f32", 401, 96, 101)
    run_case(img, "polygon", oracle.regular_polygon_vertices(6, 64.0))


def test_f32_ellipse80x40():
    img = datagen.image_for("f32", 402, 90, 77)
    run_case(img, "ellipse", 80, 40)


@pytest.mark.parametrize("spec", [
    ("spans", [0, -1, -2], [2, 1, 0], -2),            # asymmetric
    ("spans", [0, 0], [1, 1], 0),                     # even n = 4, lower median
    ("spans", [-3], [2], 0),                          # one row
    ("spans", [0] * 7, [0] * 7, -3),                  # one column
    ("spans", [-1] * 3, [1] * 3, -1),                 # 3x3 square
    ("ellipse", 9, 3),
    ("disk_limit", 48 * 48 + 48),                     # the fuller disk of Fig. 10
])
def test_kernel_shapes(spec):
    img = datagen.image_for("u16", 77, 97, 131)
    run_case(img, *spec)


@pytest.mark.parametrize("sides,R,phase", [(4, 12.0, 45.0), (8, 15.5, 10.0), (12, 30.0, 0.0), (3, 20.0, 90.0)])
def test_polygons(sides, R, phase):
    img = datagen.image_for("u8", 88, 90, 111)
    run_case(img, "polygon", oracle.regular_polygon_vertices(sides, R, phase))


@pytest.mark.parametrize("shape", [(1, 1), (1, 75), (66, 1), (2, 3), (31, 33), (64, 64), (65, 129)])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_degenerate_sizes(shape, dtype):
    img = datagen.image_for(dtype, 55, *shape)
    run_case(img, "circle", 6)


def test_radius0_identity_and_constant():
    img = datagen.image_for("u16", 9, 70, 90)
    run_case(img, "circle", 0)
    run_case(np.full((70, 90), 1234, np.uint16), "circle", 20)
    run_case(np.full((50, 40), -2.5, np.float32), "ellipse", 30, 10)


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_adversarial_checkerboard(dtype):
    img = datagen.adversarial_tile(150, 170, dtype, border=24)
    run_case(img, "circle", 20)


def test_pitch_wider_than_row():
    img = datagen.image_for("u16", 12, 77, 101)
    run_case(img, "circle", 9, pitch_elems=128)
    img = datagen.image_for("f32", 13, 50, 61)
    run_case(img, "circle", 7, pitch_elems=64)


@pytest.mark.parametrize("pct", [0, 10, 30, 50, 70, 90, 100])
def test_percentiles(pct):
    img = datagen.image_for("u16", 61, 120, 99)
    run_case(img, "circle", 12, percentile=pct)


def test_float_signed_zero_and_denormals():
    rng = np.random.default_rng(5)
    vals = np.array([0.0, -0.0, 1e-45, -1e-45, 2e-40, -2e-40, 1.0, -1.0, 3e38, -3e38], np.float32)
    img = vals[rng.integers(0, len(vals), size=(60, 70))]
    run_case(img, "circle", 3)
    run_case(img, "circle", 11)


def test_full_size_config2_sampled():
    """4096x4096 u16 at r = 8, 32, 48 in the launch configuration the bench times: every
    tile-border row/column sample plus random pixels against the oracle, point by point."""
    import torch
    import paper_2505_22938_gb300 as fim
    from helpers import to_device, to_host
    img = datagen.config2_image()
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.integers(0, 4096, 3000), np.array([0, 4095, 63, 64, 127, 128, 4032, 4031])])
    ys = np.concatenate([rng.integers(0, 4096, 3000), np.array([4095, 0, 64, 63, 128, 127, 4031, 4032])])
    store, _ = to_device(img)
    out = torch.empty_like(store)
    for r in (8, 32, 48):
        k = fim.fim_create_kernel_circle(r)
        fim.median(store, k, out=out)
        torch.cuda.synchronize()
        assert fim.fim_sync_status() == 0
        got = to_host(out)[ys, xs]
        exp = oracle.median_points(img, oracle.disk_offsets(r), xs, ys)
        assert np.array_equal(got, exp), f"r={r}: {np.sum(got != exp)} of {len(xs)} samples differ"


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
@pytest.mark.parametrize("r", [80, 96, 100, 113, 128])
def test_large_radius(dtype, r):
    """Kernels whose footprint needs global scratch (radix keys, 32-bit omnigram entries), or
    whose default tile is the smaller one that keeps the omnigram in shared memory (r = 80), or
    whose footprints exceed 65535 pixels on the larger tile (8-bit and float data keep it)."""
    img = datagen.image_for(dtype, 500 + r, 45, 71)
    run_case(img, "circle", r)


def test_f32_r100_multi_tile():
    img = datagen.image_for("f32", 601, 70, 99)
    run_case(img, "circle", 100)


@pytest.mark.parametrize("spec", [("ellipse", 128, 20), ("ellipse", 20, 128), ("disk_limit", 128 * 128 + 128)])
def test_large_extents(spec):
    img = datagen.image_for("u16", 602, 40, 44)
    run_case(img, *spec)


@pytest.mark.parametrize("spec", [("ellipse", 96, 20), ("ellipse", 20, 96), ("circle", 64)])
@pytest.mark.parametrize("dtype", ["u16", "f32"])
def test_box_side_256(spec, dtype):
    """Footprint boxes with one side exactly 256 (8-bit coordinates use the whole range on that
    axis, so the padding sentinel relies on the other axis) and 256 x 256 (32-bit entries)."""
    img = datagen.image_for(dtype, 613, 150, 170)
    run_case(img, *spec)


def test_full_size_config3_sampled():
    """8192x8192 f32 (fields + Cauchy outliers) at disk r=64 and 100, the hexagon (R=64) and
    the 80x40 ellipse, in the launch configuration of a full-image call: sampled pixels,
    including tile and image borders, against the oracle point by point."""
    import torch
    import paper_2505_22938_gb300 as fim
    img = datagen.config3_image()
    rng = np.random.default_rng(3)
    n = 600
    xs = np.concatenate([rng.integers(0, 8192, n), [0, 8191, 31, 32, 63, 64, 8160, 8191, 0]])
    ys = np.concatenate([rng.integers(0, 8192, n), [8191, 0, 32, 31, 64, 63, 8191, 8160, 4095]])
    dev = torch.from_numpy(img).cuda()
    out = torch.empty_like(dev)
    cases = [("circle", 64), ("circle", 100), ("polygon", oracle.regular_polygon_vertices(6, 64.0)),
             ("ellipse", 80, 40)]
    for spec in cases:
        k = fim_kernel(*spec)
        fim.median(dev, k, out=out)
        torch.cuda.synchronize()
        assert fim.fim_sync_status() == 0
        got = out.cpu().numpy()[ys, xs]
        exp = oracle.median_points(img, oracle_offsets(*spec), xs, ys)
        assert np.array_equal(got.view(np.uint32), exp.view(np.uint32)), \
            f"{spec[0]}: {np.sum(got.view(np.uint32) != exp.view(np.uint32))} of {len(xs)} samples differ"


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_tile_shapes_by_image_size(dtype):
    """The default tile shape depends on the image size: small images take smaller tiles that
    fill the GPU in one wave, 1024^2 keeps the large-image shapes. Both are checked against the
    oracle (whole small images; sampled pixels, tile borders included, at 1024^2)."""
    import torch
    import paper_2505_22938_gb300 as fim
    from helpers import to_device, to_host
    code = {"u8": fim.FIM_U8, "u16": fim.FIM_U16, "f32": fim.FIM_F32}[dtype]
    for r in (4, 16, 24, 32):
        k = fim.fim_create_kernel_circle(r)
        small = fim.fim_plan_info(k, code, 256, 256)
        big = fim.fim_plan_info(k, code, 1024, 1024)
        assert (small["tile_w"], small["tile_h"]) in ((32, 8), (32, 16)), (r, small)
        assert big["tile_w"] * big["tile_h"] >= 1024, (r, big)
    for r in (48, 96):
        k = fim.fim_create_kernel_circle(r)
        small = fim.fim_plan_info(k, code, 256, 256)
        assert (small["tile_w"], small["tile_h"]) in ((32, 16), (64, 32)), (r, small)
    img = datagen.image_for(dtype, 811, 256, 256)
    for r in (4, 24):
        run_case(img, "circle", r)
    img = datagen.image_for(dtype, 813, 200, 184)
    run_case(img, "circle", 48)
    img = datagen.image_for(dtype, 812, 1024, 1024)
    store, _ = to_device(img)
    out = torch.empty_like(store)
    rng = np.random.default_rng(5)
    edges = np.array([0, 31, 32, 63, 64, 127, 128, 1023])
    xs = np.concatenate([rng.integers(0, 1024, 600), edges, rng.integers(0, 1024, 8)])
    ys = np.concatenate([rng.integers(0, 1024, 600), rng.integers(0, 1024, 8), edges])
    for r in (4, 16, 32):
        fim.median(store, fim.fim_create_kernel_circle(r), out=out)
        torch.cuda.synchronize()
        assert fim.fim_sync_status() == 0
        got = to_host(out)[ys, xs]
        exp = oracle.median_points(img, oracle.disk_offsets(r), xs.astype(np.int32), ys.astype(np.int32))
        assert np.array_equal(np.ascontiguousarray(got).view(np.uint8), np.ascontiguousarray(exp).view(np.uint8)), r


def test_f32_footprints_beyond_65535():
    """Float keys whose tile footprint exceeds 65535 pixels (1024^2, disk r = 100 on 64x128 tiles,
    r = 128 on 64x64): the 16-bit pass of the radix sort counts in two rounds. Sampled pixels,
    tile borders included, against the oracle."""
    import torch
    import paper_2505_22938_gb300 as fim
    from helpers import to_device, to_host
    img = datagen.image_for("f32", 814, 1024, 1024)
    store, _ = to_device(img)
    out = torch.empty_like(store)
    rng = np.random.default_rng(8)
    edges = np.array([0, 63, 64, 127, 128, 511, 512, 1023])
    xs = np.concatenate([rng.integers(0, 1024, 300), edges, rng.integers(0, 1024, 8)])
    ys = np.concatenate([rng.integers(0, 1024, 300), rng.integers(0, 1024, 8), edges])
    for r in (100, 128):
        k = fim.fim_create_kernel_circle(r)
        assert fim.fim_plan_info(k, fim.FIM_F32, 1024, 1024)["footprint"] > 65535
        fim.median(store, k, out=out)
        torch.cuda.synchronize()
        assert fim.fim_sync_status() == 0
        got = to_host(out)[ys, xs]
        exp = oracle.median_points(img, oracle.disk_offsets(r), xs.astype(np.int32), ys.astype(np.int32))
        assert np.array_equal(np.ascontiguousarray(got).view(np.uint32), np.ascontiguousarray(exp).view(np.uint32)), r
