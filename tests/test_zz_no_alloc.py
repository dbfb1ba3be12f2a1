"""fim_median_noalloc: the allocation-free entry point gives the same bytes as fim_median.

Callers that must not allocate device memory (stream capture, externally owned memory pools,
real-time services) use this entry point; it works out of a fixed device array inside the
library. This file is collected last so that a failure here cannot hide any other test.
"""
import numpy as np
import pytest

import datagen
from helpers import assert_bit_exact, to_device, to_host

pytestmark = pytest.mark.gpu

CODES = {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1, np.dtype(np.float32): 2}


def _run_both(img, kernel):
    import torch
    import paper_2505_22938_gb300 as fim
    store, _ = to_device(img)
    h, w = img.shape
    pitch = store.stride(0) * store.element_size()
    code = CODES[img.dtype]
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.zeros_like(store)
    fim.fim_median(store.data_ptr(), ref.data_ptr(), w, h, pitch, code, kernel, stream)
    outs = []
    for _ in range(2):  # two calls in a row share (and reuse) the fixed workspace
        out = torch.full_like(store, 0)
        fim.fim_median_noalloc(store.data_ptr(), out.data_ptr(), w, h, pitch, code, kernel, stream)
        outs.append(out)
    torch.cuda.synchronize()
    assert fim.fim_sync_status(stream) == 0
    exp = to_host(ref)
    for out in outs:
        assert_bit_exact(to_host(out), exp, f"noalloc vs fim_median {img.dtype} {img.shape}")


@pytest.mark.parametrize("dtype,r,shape", [
    ("u16", 32, (300, 277)),     # everything in shared memory: the workspace holds the tile queue
    ("f32", 100, (70, 99)),      # radix keys in the per-CTA workspace buffers
    ("u8", 128, (45, 71)),       # 32-bit omnigram in the per-CTA workspace buffers
])
def test_noalloc_matches_fim_median(dtype, r, shape):
    import paper_2505_22938_gb300 as fim
    img = datagen.image_for(dtype, 900 + r, *shape)
    _run_both(img, fim.fim_create_kernel_circle(r))


def test_noalloc_rejects_oversize_workspace():
    """A request whose per-CTA buffers exceed the fixed array is refused, not truncated."""
    import torch
    import paper_2505_22938_gb300 as fim
    h = w = 4096
    src = torch.zeros((h, w), dtype=torch.float32, device="cuda")
    out = torch.zeros_like(src)
    k = fim.fim_create_kernel_circle(100)
    with pytest.raises(fim.FimError) as e:
        fim.fim_median_noalloc(src.data_ptr(), out.data_ptr(), w, h, w * 4, fim.FIM_F32, k,
                               torch.cuda.current_stream().cuda_stream)
    assert e.value.code == 2  # FIM_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert not torch.any(out != 0)  # nothing was launched
