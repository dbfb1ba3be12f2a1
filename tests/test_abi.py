"""C-ABI checks that need no GPU: the library loads, exports every declared symbol, and its
host-side kernel geometry and argument checks behave as documented in include/fim.h."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2505_22938_gb300 as fim

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fim.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fim_[a-z0-9_]+)\s*\(", text)))


def test_library_loads_and_exports_every_symbol():
    lib = fim.lib()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert name in fim.SIGNATURES, f"binding lacks {name}"
    assert fim.fim_version().count(".") == 2
    for code, name in fim.STATUS.items():
        assert fim.fim_status_string(code) == name


@pytest.mark.parametrize("r", [0, 1, 2, 4, 8, 17, 32, 48, 64, 100, 128])
def test_circle_geometry_matches_oracle(r):
    k = fim.fim_create_kernel_circle(r)
    info = k.info
    off = oracle.disk_offsets(r)
    assert info["ntaps"] == len(off)
    assert (info["xmin"], info["xmax"], info["ymin"], info["ymax"]) == (-r, r, -r, r)


def test_disk_limit_geometry():
    k = fim.fim_create_kernel_disk_limit(48 * 48 + 48)
    assert k.info["ntaps"] == len(oracle.disk_limit_offsets(48, 48 * 48 + 48)) == 7393
    assert fim.fim_create_kernel_disk_limit(6).info["ntaps"] == 21  # Fig. 3b


@pytest.mark.parametrize("a,b", [(80, 40), (3, 1), (0, 5), (5, 0), (0, 0), (7, 7), (128, 1)])
def test_ellipse_geometry(a, b):
    k = fim.fim_create_kernel_ellipse(a, b)
    off = oracle.ellipse_offsets(a, b)
    assert k.info["ntaps"] == len(off)
    assert (k.info["xmin"], k.info["xmax"]) == (off[:, 0].min(), off[:, 0].max())
    assert (k.info["ymin"], k.info["ymax"]) == (off[:, 1].min(), off[:, 1].max())


@pytest.mark.parametrize("sides,R,phase", [(6, 64.0, 0.0), (6, 3.0, 0.0), (4, 10.0, 45.0), (8, 20.5, 11.0),
                                           (12, 40.0, 0.0), (3, 9.0, 90.0)])
def test_polygon_geometry(sides, R, phase):
    v = oracle.regular_polygon_vertices(sides, R, phase)
    k = fim.fim_create_kernel_polygon(v)
    off = oracle.polygon_offsets(v)
    assert k.info["ntaps"] == len(off)
    assert (k.info["ymin"], k.info["ymax"]) == (off[:, 1].min(), off[:, 1].max())


def test_invalid_kernels_rejected():
    with pytest.raises(fim.FimError):
        fim.fim_create_kernel_circle(-1)
    with pytest.raises(fim.FimError):
        fim.fim_create_kernel_circle(129)
    with pytest.raises(fim.FimError):  # clockwise
        fim.fim_create_kernel_polygon(oracle.regular_polygon_vertices(6, 5.0)[::-1])
    with pytest.raises(fim.FimError):  # not convex (arrow head)
        fim.fim_create_kernel_polygon([(0, 0), (4, -4), (2, 0), (4, 4)][::-1])
    with pytest.raises(fim.FimError):  # empty row span
        fim.fim_create_kernel_spans([0, 2], [1, 1], 0)
    with pytest.raises(fim.FimError):  # a column with two runs (U shape)
        fim.fim_create_kernel_spans([-1, -1, -1], [1, -1, 1], -1)
    with pytest.raises(fim.FimError):  # too wide
        fim.fim_create_kernel_spans([-200], [200], 0)
    k = fim.fim_create_kernel_spans([0, -1, -2], [2, 1, 0], -2)
    assert k.info == dict(ntaps=9, xmin=-2, xmax=2, ymin=-2, ymax=0)


def test_argument_checks_need_no_gpu():
    lib = fim.lib()
    k = fim.fim_create_kernel_circle(3)
    buf = ctypes.create_string_buffer(4096)
    a = ctypes.addressof(buf)
    INVALID = 1
    # null pointers, bad sizes, bad dtype, bad border
    assert lib.fim_median(None, a, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    assert lib.fim_median(a, a + 2048, 0, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    assert lib.fim_median(a, a + 2048, 4, 4, 8, 7, k.handle, 0, None) == INVALID
    assert lib.fim_median(a, a + 2048, 4, 4, 8, fim.FIM_U16, k.handle, 3, None) == INVALID
    assert lib.fim_median(a, a + 2048, 4, 4, 8, fim.FIM_U16, None, 0, None) == INVALID
    # pitch below w * elem, pitch not a multiple of the element size
    assert lib.fim_median(a, a + 2048, 4, 4, 6, fim.FIM_U16, k.handle, 0, None) == INVALID
    assert lib.fim_median(a, a + 2048, 4, 4, 9, fim.FIM_U16, k.handle, 0, None) == INVALID
    # overlapping input and output
    assert lib.fim_median(a, a + 16, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    # percentile outside [0, 100]
    assert lib.fim_percentile(a, a + 2048, 4, 4, 8, fim.FIM_U16, k.handle, 101.0, 0, None) == INVALID
    assert lib.fim_percentile(a, a + 2048, 4, 4, 8, fim.FIM_U16, k.handle, float("nan"), 0, None) == INVALID
    # several percentiles: count outside 1..8, a null output, an output overlapping the input,
    # a percentile outside [0, 100]
    outs = (ctypes.c_void_p * 9)(*([a + 2048] * 9))
    pcts = (ctypes.c_double * 9)(*([50.0] * 9))
    for count in (0, 9):
        assert lib.fim_percentiles(a, outs, pcts, count, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    assert lib.fim_percentiles(a, None, pcts, 2, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    assert lib.fim_percentiles(a, outs, None, 2, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    bad = (ctypes.c_void_p * 2)(a + 2048, None)
    assert lib.fim_percentiles(a, bad, pcts, 2, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    bad = (ctypes.c_void_p * 2)(a + 2048, a + 16)
    assert lib.fim_percentiles(a, bad, pcts, 2, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    badp = (ctypes.c_double * 2)(50.0, -1.0)
    assert lib.fim_percentiles(a, outs, badp, 2, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    # several radii: count outside 1..8, null arrays, a kernel that is not a disk, an output
    # overlapping the input
    kk = (ctypes.c_void_p * 9)(*([k.handle] * 9))
    for count in (0, 9):
        assert lib.fim_median_radii(a, outs, kk, count, 4, 4, 8, fim.FIM_U16, 0, None) == INVALID
    assert lib.fim_median_radii(a, None, kk, 2, 4, 4, 8, fim.FIM_U16, 0, None) == INVALID
    assert lib.fim_median_radii(a, outs, None, 2, 4, 4, 8, fim.FIM_U16, 0, None) == INVALID
    sq = fim.fim_create_kernel_spans([-1, -1, -1], [1, 1, 1], -1)
    mixed = (ctypes.c_void_p * 2)(k.handle, sq.handle)
    assert lib.fim_median_radii(a, outs, mixed, 2, 4, 4, 8, fim.FIM_U16, 0, None) == INVALID
    assert lib.fim_median_radii(a, bad, kk, 2, 4, 4, 8, fim.FIM_U16, 0, None) == INVALID
    # percentile map: null, pitch below 4 * w or not a multiple of 4, overlapping the output
    m = a + 3072
    assert lib.fim_percentile_map(a, a + 2048, None, 16, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    assert lib.fim_percentile_map(a, a + 2048, m, 12, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    assert lib.fim_percentile_map(a, a + 2048, m, 18, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    assert lib.fim_percentile_map(a, a + 2048, a + 2040, 16, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID
    assert lib.fim_percentile_map(a, a + 2048, a + 2060, 16, 4, 4, 8, fim.FIM_U16, k.handle, 0, None) == INVALID


def test_batch_rejects_aliased_images():
    """One batch runs every job in one launch: an output overlapping its own input, another
    job's input or another output is refused before any device work; a shared input is not."""
    lib = fim.lib()
    k = fim.fim_create_kernel_circle(2)
    buf = ctypes.create_string_buffer(1 << 16)
    a = ctypes.addressof(buf)

    def create(jobs):
        arr = (fim.fim_job * len(jobs))(*jobs)
        h = ctypes.c_void_p()
        return lib.fim_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(jobs), ctypes.byref(h))

    def job(i, o):  # 8x8 u16 images, pitch 16 bytes: each spans 128 bytes
        return fim.make_job(a + i, a + o, 8, 8, 16, fim.FIM_U16, k)

    INVALID = 1
    assert create([job(0, 64)]) == INVALID                      # own input and output overlap
    assert create([job(0, 1024), job(2048, 1100)]) == INVALID   # two outputs overlap
    assert create([job(0, 1024), job(1024 + 64, 3000)]) == INVALID  # an input under another output
    assert create([job(0, 1024), job(3000, 1024 + 127)]) == INVALID  # last byte of an output
    # disjoint outputs, one shared input: passes the checks (fails later without a GPU)
    assert create([job(0, 1024), job(0, 2048)]) != INVALID
    assert create([job(0, 1024), job(512, 1152)]) != INVALID    # outputs back to back
