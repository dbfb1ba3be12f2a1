"""Shared helpers for the GPU parity tests: run the CUDA path and the oracle on the same
seeded input and compare bit for bit."""
import numpy as np

import oracle

def torch_dtype(np_dtype):
    import torch
    return {np.dtype(np.uint8): torch.uint8, np.dtype(np.uint16): torch.uint16,
            np.dtype(np.float32): torch.float32}[np.dtype(np_dtype)]


def to_device(img, pitch_elems=None):
    """Copies a 2-D numpy image to the GPU, optionally with a row pitch wider than its width.
    Returns (storage tensor, view of the image)."""
    import torch
    h, w = img.shape
    pe = w if pitch_elems is None else pitch_elems
    store = torch.zeros((h, pe), dtype=torch_dtype(img.dtype), device="cuda")
    src = torch.from_numpy(np.ascontiguousarray(img).view(np.int16) if img.dtype == np.uint16
                           else np.ascontiguousarray(img))
    if img.dtype == np.uint16:
        store.view(torch.int16)[:, :w].copy_(src)
    else:
        store[:, :w].copy_(src)
    return store, store[:, :w]


def to_host(t):
    import torch
    if t.dtype == torch.uint16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def gpu_filter(img, kernel, pitch_elems=None, percentile=None):
    """Runs fim_median (or fim_percentile) through the C ABI on a device copy of img."""
    import torch
    import paper_2505_22938_gb300 as fim
    store_in, vin = to_device(img, pitch_elems)
    store_out = torch.full_like(store_in, 0)
    h, w = img.shape
    pitch = store_in.stride(0) * store_in.element_size()
    code = {np.dtype(np.uint8): fim.FIM_U8, np.dtype(np.uint16): fim.FIM_U16,
            np.dtype(np.float32): fim.FIM_F32}[img.dtype]
    stream = torch.cuda.current_stream().cuda_stream
    if percentile is None:
        fim.fim_median(store_in.data_ptr(), store_out.data_ptr(), w, h, pitch, code, kernel, stream)
    else:
        fim.fim_percentile(store_in.data_ptr(), store_out.data_ptr(), w, h, pitch, code, kernel, percentile,
                           stream)
    torch.cuda.synchronize()
    st = fim.fim_sync_status(stream)
    assert st == 0, fim.STATUS.get(st, st)
    out = to_host(store_out)
    if pitch_elems is not None and pitch_elems > w:
        assert not np.any(out[:, w:] != 0), "wrote outside the image"
    return out[:, :w]


def assert_bit_exact(got, exp, what=""):
    """Equality of the bit patterns (so -0.0 and +0.0 differ), with the first mismatch reported."""
    g = np.ascontiguousarray(got)
    e = np.ascontiguousarray(exp)
    assert g.shape == e.shape and g.dtype == e.dtype, (g.shape, e.shape, g.dtype, e.dtype)
    ui = {1: np.uint8, 2: np.uint16, 4: np.uint32}[g.itemsize]
    gu, eu = g.view(ui), e.view(ui)
    if not np.array_equal(gu, eu):
        bad = np.argwhere(gu != eu)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} of {g.size} pixels differ; first at (y={y}, x={x}): "
                             f"gpu={g[y, x]!r} oracle={e[y, x]!r}")


def oracle_offsets(kind, *args):
    if kind == "circle":
        return oracle.disk_offsets(*args)
    if kind == "disk_limit":
        r = int(np.sqrt(args[0]))
        return oracle.disk_limit_offsets(r, args[0])
    if kind == "ellipse":
        return oracle.ellipse_offsets(*args)
    if kind == "polygon":
        return oracle.polygon_offsets(args[0])
    if kind == "spans":
        return oracle.spans_offsets(*args)
    raise ValueError(kind)


def fim_kernel(kind, *args):
    import paper_2505_22938_gb300 as fim
    if kind == "circle":
        return fim.fim_create_kernel_circle(*args)
    if kind == "disk_limit":
        return fim.fim_create_kernel_disk_limit(*args)
    if kind == "ellipse":
        return fim.fim_create_kernel_ellipse(*args)
    if kind == "polygon":
        return fim.fim_create_kernel_polygon(args[0])
    if kind == "spans":
        return fim.fim_create_kernel_spans(*args)
    raise ValueError(kind)
