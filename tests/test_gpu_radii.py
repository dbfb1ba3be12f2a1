"""Several disk radii from one ordinal transform (fim_median_radii, the multi-radius half of the
extension Sec. 6.2 proposes): every output must equal the oracle's median with its own disk, bit
for bit, and the single-kernel entry point on the same image."""
import numpy as np
import pytest

import datagen
import oracle
from helpers import assert_bit_exact, gpu_filter, to_device, to_host

pytestmark = pytest.mark.gpu


def run_radii(img, kernels_spec, pitch_elems=None):
    """kernels_spec: list of ("circle", r) or ("disk_limit", limit)."""
    import torch
    import paper_2505_22938_gb300 as fim
    ks, offs = [], []
    for kind, a in kernels_spec:
        if kind == "circle":
            ks.append(fim.fim_create_kernel_circle(a))
            offs.append(oracle.disk_offsets(a))
        else:
            r = int(np.sqrt(a))
            ks.append(fim.fim_create_kernel_disk_limit(a))
            offs.append(oracle.disk_limit_offsets(r, a))
    store_in, _ = to_device(img, pitch_elems)
    outs = [torch.zeros_like(store_in) for _ in ks]
    h, w = img.shape
    pitch = store_in.stride(0) * store_in.element_size()
    code = {np.dtype(np.uint8): fim.FIM_U8, np.dtype(np.uint16): fim.FIM_U16,
            np.dtype(np.float32): fim.FIM_F32}[img.dtype]
    stream = torch.cuda.current_stream().cuda_stream
    fim.fim_median_radii(store_in.data_ptr(), [o.data_ptr() for o in outs], ks, w, h, pitch, code, stream)
    torch.cuda.synchronize()
    st = fim.fim_sync_status(stream)
    assert st == 0, fim.STATUS.get(st, st)
    for (kind, a), k, off, o in zip(kernels_spec, ks, offs, outs):
        got = to_host(o)
        if pitch_elems is not None and pitch_elems > w:
            assert not np.any(got[:, w:] != 0), "wrote outside the image"
        got = got[:, :w]
        assert_bit_exact(got, oracle.median_filter(img, off), f"{kind}{a} {img.dtype} {img.shape}")
        assert_bit_exact(got, gpu_filter(img, k), f"single-kernel {kind}{a}")


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_radii_8_16_32(dtype):
    """Sec. 6.2's example radii; the tile is the r = 32 one (1024-thread CTAs, every dtype)."""
    img = datagen.image_for(dtype, 40, 170, 150)
    run_radii(img, [("circle", 8), ("circle", 16), ("circle", 32)])


def test_radii_small_ctas_and_order():
    """Radii up to 12 (small-CTA tiles), given out of order with a repeat and radius 0."""
    img = datagen.image_for("u16", 41, 131, 77)
    run_radii(img, [("circle", 5), ("circle", 12), ("circle", 0), ("circle", 5), ("circle", 2)])


def test_radii_large_and_fuller_disk():
    """The largest disk needs global scratch (r = 100 float); a r^2 + r disk among them."""
    img = datagen.image_for("f32", 42, 90, 110)
    run_radii(img, [("circle", 100), ("circle", 64), ("disk_limit", 48 * 48 + 48)])


def test_eight_radii_pitched():
    img = datagen.image_for("u8", 43, 120, 99)
    run_radii(img, [("circle", r) for r in (1, 3, 6, 10, 15, 21, 28, 36)], pitch_elems=128)


def test_radii_rejects_non_disks_and_counts():
    import torch
    import paper_2505_22938_gb300 as fim
    img = torch.zeros((32, 32), dtype=torch.uint8, device="cuda")
    outs = [torch.zeros_like(img) for _ in range(9)]
    ks = [fim.fim_create_kernel_circle(3)] * 9
    with pytest.raises(fim.FimError):
        fim.fim_median_radii(img.data_ptr(), [o.data_ptr() for o in outs], ks, 32, 32, 32, fim.FIM_U8)
    ell = fim.fim_create_kernel_ellipse(4, 2)
    with pytest.raises(fim.FimError):
        fim.fim_median_radii(img.data_ptr(), [outs[0].data_ptr(), outs[1].data_ptr()], [ks[0], ell], 32, 32, 32,
                             fim.FIM_U8)
