"""Several percentiles from one ordinal transform (fim_percentiles, the extension Sec. 6.2
proposes): every output must equal the oracle's rank-order filter at its own rank, bit for
bit, and the single-percentile entry point on the same image."""
import numpy as np
import pytest

import datagen
import oracle
from helpers import assert_bit_exact, fim_kernel, gpu_filter, oracle_offsets, to_device, to_host

pytestmark = pytest.mark.gpu


def run_multi(img, kind, args, pcts, pitch_elems=None):
    import torch
    import paper_2505_22938_gb300 as fim
    k = fim_kernel(kind, *args)
    off = oracle_offsets(kind, *args)
    store_in, _ = to_device(img, pitch_elems)
    outs = [torch.zeros_like(store_in) for _ in pcts]
    h, w = img.shape
    pitch = store_in.stride(0) * store_in.element_size()
    code = {np.dtype(np.uint8): fim.FIM_U8, np.dtype(np.uint16): fim.FIM_U16,
            np.dtype(np.float32): fim.FIM_F32}[img.dtype]
    stream = torch.cuda.current_stream().cuda_stream
    fim.fim_percentiles(store_in.data_ptr(), [o.data_ptr() for o in outs], pcts, w, h, pitch, code, k, stream)
    torch.cuda.synchronize()
    st = fim.fim_sync_status(stream)
    assert st == 0, fim.STATUS.get(st, st)
    for pct, o in zip(pcts, outs):
        got = to_host(o)
        if pitch_elems is not None and pitch_elems > w:
            assert not np.any(got[:, w:] != 0), "wrote outside the image"
        got = got[:, :w]
        exp = oracle.median_filter(img, off, rank=oracle.percentile_rank(len(off), pct))
        assert_bit_exact(got, exp, f"{kind}{args} p{pct} {img.dtype} {img.shape}")
        assert_bit_exact(got, gpu_filter(img, k, percentile=pct), f"single-percentile p{pct}")


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
@pytest.mark.parametrize("r", [4, 12, 30])
def test_quartiles(dtype, r):
    """25th/50th/75th percentiles (small-CTA and 1024-thread tiles, every dtype)."""
    img = datagen.image_for(dtype, 7 + r, 141, 123)
    run_multi(img, "circle", (r,), [25, 50, 75])


def test_eight_ranks_with_extremes_and_repeats():
    """The most outputs one launch takes, including ranks 0 and n - 1 and a repeated percentile,
    on a pitched input."""
    img = datagen.image_for("u16", 3, 150, 97)
    run_multi(img, "circle", (9,), [0, 10, 50, 50, 90, 100, 37.5, 62.5], pitch_elems=160)


def test_convex_kernel_percentiles():
    img = datagen.image_for("f32", 11, 90, 133)
    run_multi(img, "polygon", (oracle.regular_polygon_vertices(6, 10.0, 0.3),), [10, 30, 70, 90])


def test_one_percentile_equals_fim_percentile():
    img = datagen.image_for("u8", 5, 70, 64)
    run_multi(img, "circle", (6,), [40])


def test_python_helper_returns_one_image_per_percentile():
    import torch
    import paper_2505_22938_gb300 as fim
    img = datagen.image_for("u16", 2, 64, 80)
    _, view = to_device(img)
    k = fim.fim_create_kernel_circle(5)
    outs = fim.percentiles(view, k, [20, 80])
    torch.cuda.synchronize()
    off = oracle.disk_offsets(5)
    for pct, o in zip([20, 80], outs):
        exp = oracle.median_filter(img, off, rank=oracle.percentile_rank(len(off), pct))
        assert_bit_exact(to_host(o), exp, f"helper p{pct}")
