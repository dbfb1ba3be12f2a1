"""Spatially varying percentile (Fig. 14): fim_percentile_map against the oracle's rank-order
filter with a rank per pixel, bit for bit. The oracle's ranks come from its own percentile
rounding (fp64, clamped, NaN as 0), which the kernel must reproduce exactly."""
import numpy as np
import pytest

import datagen
import oracle
from helpers import assert_bit_exact, fim_kernel, oracle_offsets, to_device, to_host

pytestmark = pytest.mark.gpu


def run_map(img, kind, args, pct, pitch_elems=None):
    import torch
    import paper_2505_22938_gb300 as fim
    k = fim_kernel(kind, *args)
    off = oracle_offsets(kind, *args)
    store_in, _ = to_device(img, pitch_elems)
    out = torch.zeros_like(store_in)
    pmap = torch.from_numpy(np.ascontiguousarray(pct, dtype=np.float32)).cuda()
    h, w = img.shape
    pitch = store_in.stride(0) * store_in.element_size()
    code = {np.dtype(np.uint8): fim.FIM_U8, np.dtype(np.uint16): fim.FIM_U16,
            np.dtype(np.float32): fim.FIM_F32}[img.dtype]
    stream = torch.cuda.current_stream().cuda_stream
    fim.fim_percentile_map(store_in.data_ptr(), out.data_ptr(), pmap.data_ptr(), pmap.stride(0) * 4, w, h, pitch,
                           code, k, stream)
    torch.cuda.synchronize()
    st = fim.fim_sync_status(stream)
    assert st == 0, fim.STATUS.get(st, st)
    got = to_host(out)
    if pitch_elems is not None and pitch_elems > w:
        assert not np.any(got[:, w:] != 0), "wrote outside the image"
    exp = oracle.rank_map_filter(img, off, oracle.percentile_rank_map(len(off), pct))
    assert_bit_exact(got[:, :w], exp, f"{kind}{args} map {img.dtype} {img.shape}")


def ramp(h, w):
    """0 % at the left edge to 100 % at the right (the Fig. 14 setting)."""
    return np.broadcast_to(np.linspace(0.0, 100.0, w, dtype=np.float32), (h, w)).copy()


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
@pytest.mark.parametrize("r", [3, 12, 32])
def test_horizontal_ramp(dtype, r):
    img = datagen.image_for(dtype, 30 + r, 133, 157)
    run_map(img, "circle", (r,), ramp(133, 157))


@pytest.mark.parametrize("r", [5, 20])
def test_random_map_with_jumps(r):
    """Independent random percentiles at every pixel: neighbouring targets differ by up to n - 1."""
    rng = np.random.default_rng(r)
    img = datagen.image_for("u16", 40 + r, 120, 101)
    run_map(img, "circle", (r,), rng.uniform(0, 100, (120, 101)).astype(np.float32))


def test_vertical_ramp_and_blocks_pitched():
    """A top-to-bottom ramp plus constant blocks, on a pitched input."""
    h, w = 140, 97
    pct = np.broadcast_to(np.linspace(100.0, 0.0, h, dtype=np.float32)[:, None], (h, w)).copy()
    pct[20:60, 10:50] = 50.0
    pct[70:90, 60:90] = 0.0
    img = datagen.image_for("f32", 9, h, w)
    run_map(img, "circle", (7,), pct, pitch_elems=128)


def test_out_of_range_and_nan_values_clamp():
    rng = np.random.default_rng(2)
    h, w = 64, 70
    pct = rng.uniform(-50, 150, (h, w)).astype(np.float32)
    pct[rng.random((h, w)) < 0.05] = np.nan
    pct[0, :5] = [np.inf, -np.inf, 100.0, 0.0, 50.0]
    img = datagen.image_for("u8", 3, h, w)
    run_map(img, "circle", (4,), pct)


def test_constant_map_equals_fim_percentile():
    from helpers import gpu_filter
    img = datagen.image_for("u16", 8, 90, 90)
    for p in (12.5, 50.0, 87.0):
        k = fim_kernel("circle", 9)
        run_map(img, "circle", (9,), np.full((90, 90), p, np.float32))
        off = oracle.disk_offsets(9)
        assert_bit_exact(gpu_filter(img, k, percentile=p),
                         oracle.median_filter(img, off, rank=oracle.percentile_rank(len(off), p)), f"p{p}")


def test_convex_kernels():
    h, w = 100, 120
    img = datagen.image_for("u16", 13, h, w)
    run_map(img, "polygon", (oracle.regular_polygon_vertices(6, 8.0),), ramp(h, w))
    run_map(img, "ellipse", (9, 4), ramp(h, w)[:, ::-1].copy())


def test_python_helper():
    import torch
    import paper_2505_22938_gb300 as fim
    img = datagen.image_for("u16", 5, 60, 80)
    _, view = to_device(img)
    pct = ramp(60, 80)
    k = fim.fim_create_kernel_circle(6)
    out = fim.percentile_map(view, k, torch.from_numpy(pct).cuda())
    torch.cuda.synchronize()
    off = oracle.disk_offsets(6)
    assert_bit_exact(to_host(out), oracle.rank_map_filter(img, off, oracle.percentile_rank_map(len(off), pct)),
                     "helper")
