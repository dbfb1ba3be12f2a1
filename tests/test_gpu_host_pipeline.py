"""fim_median_host: the banded host pipeline (copy in, filter, copy out, band by band on three
streams) must give the oracle's result, for images of one band and of many, for every dtype,
with pageable and with pinned host buffers, and with a row pitch wider than the row."""
import numpy as np
import pytest

import datagen
import oracle
from helpers import assert_bit_exact, fim_kernel, oracle_offsets

pytestmark = pytest.mark.gpu


def run_host(img, r, pinned=False, pitch_elems=None):
    import torch
    import paper_2505_22938_gb300 as fim
    k = fim_kernel("circle", r)
    h, w = img.shape
    pe = w if pitch_elems is None else pitch_elems
    src = np.zeros((h, pe), img.dtype)
    src[:, :w] = img
    dst = np.zeros_like(src)
    if pinned:  # the same bytes in page-locked host memory
        tsrc = torch.from_numpy(src.view(np.uint8)).pin_memory()
        tdst = torch.zeros_like(tsrc).pin_memory()
        fim.fim_median_host(tsrc.data_ptr(), tdst.data_ptr(), w, h, src.strides[0], fim_code(img.dtype), k, 0)
        dst = tdst.numpy().view(img.dtype).reshape(h, pe)
    else:
        fim.fim_median_host(src.ctypes.data, dst.ctypes.data, w, h, src.strides[0], fim_code(img.dtype), k, 0)
    exp = oracle.median_filter(img, oracle_offsets("circle", r))
    assert_bit_exact(dst[:, :w], exp, f"host r={r} {img.dtype} {img.shape} pinned={pinned}")


def fim_code(dt):
    import paper_2505_22938_gb300 as fim
    return {np.dtype(np.uint8): fim.FIM_U8, np.dtype(np.uint16): fim.FIM_U16, np.dtype(np.float32): fim.FIM_F32}[np.dtype(dt)]


@pytest.mark.parametrize("r", [3, 8, 30])
@pytest.mark.parametrize("pinned", [False, True])
def test_u16_many_bands(r, pinned):
    img = np.ascontiguousarray(datagen.config2_image(4096, 4096)[300:300 + 611, 900:900 + 197])
    run_host(img, r, pinned=pinned)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_dtypes_and_pitch(dtype):
    img = datagen.image_for(dtype, datagen.seed_for(1, 7), 263, 141)
    run_host(img, 6, pitch_elems=160)


def test_single_band():
    img = np.ascontiguousarray(datagen.config2_image(4096, 4096)[0:30, 0:333])  # one tile row
    run_host(img, 5)
