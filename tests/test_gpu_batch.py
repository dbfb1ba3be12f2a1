"""Batched persistent launch and autotuner: identical bytes to sequential single-image calls
and to the oracle, including under CUDA-graph replay."""
import numpy as np
import pytest

import datagen
import oracle
from helpers import assert_bit_exact, to_device, to_host

pytestmark = pytest.mark.gpu

CODES = {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1, np.dtype(np.float32): 2}


def small_mixed_jobs(seed=7, count=12):
    """A miniature of the mixed batch: uneven sides, all dtypes, radii log-uniform in [2, 128]."""
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(count):
        r = int(round(np.exp(rng.uniform(np.log(2), np.log(128)))))
        side_hi = 200 if r < 40 else 90
        w, h = int(rng.integers(20, side_hi)), int(rng.integers(20, side_hi))
        dtype = ("u8", "u16", "f32")[i % 3]
        jobs.append(dict(img=datagen.image_for(dtype, 1000 + i, h, w), r=r))
    jobs.append(dict(img=datagen.image_for("u16", 2000, 37, 45), r=128))
    jobs.append(dict(img=datagen.image_for("f32", 2001, 30, 33), r=100))
    return jobs


def build_batch(specs, percentiles=None):
    import torch
    import paper_2505_22938_gb300 as fim
    stores, outs, kernels, cjobs = [], [], [], []
    for i, sp in enumerate(specs):
        store, _ = to_device(sp["img"])
        out = torch.zeros_like(store)
        k = fim.fim_create_kernel_circle(sp["r"])
        h, w = sp["img"].shape
        pct = -1.0 if percentiles is None else percentiles[i]
        cjobs.append(fim.make_job(store.data_ptr(), out.data_ptr(), w, h, store.stride(0) * store.element_size(),
                                  CODES[sp["img"].dtype], k, pct))
        stores.append(store)
        outs.append(out)
        kernels.append(k)
    return fim.fim_batch_create(cjobs, kernels), stores, outs, kernels


def test_batch_matches_oracle_and_sequential():
    import torch
    import paper_2505_22938_gb300 as fim
    specs = small_mixed_jobs()
    batch, stores, outs, kernels = build_batch(specs)
    batch.run(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert fim.fim_sync_status() == 0
    assert batch.info["total_tiles"] > 0
    for sp, store, out, k in zip(specs, stores, outs, kernels):
        exp = oracle.median_filter(sp["img"], oracle.disk_offsets(sp["r"]))
        assert_bit_exact(to_host(out), exp, f"batch r={sp['r']} {sp['img'].dtype} {sp['img'].shape}")
        seq = fim.median(store, k)
        torch.cuda.synchronize()
        assert_bit_exact(to_host(seq), to_host(out), "batch vs sequential")


def test_batch_graph_replay():
    import torch
    import paper_2505_22938_gb300 as fim
    specs = small_mixed_jobs(seed=11, count=6)
    batch, stores, outs, kernels = build_batch(specs)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    batch.run(int(s.cuda_stream))  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.run(int(s.cuda_stream))
    for _ in range(2):
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert fim.fim_sync_status() == 0
        for sp, out in zip(specs, outs):
            exp = oracle.median_filter(sp["img"], oracle.disk_offsets(sp["r"]))
            assert_bit_exact(to_host(out), exp, "graph replay")


def test_batch_percentiles():
    import torch
    specs = small_mixed_jobs(seed=13, count=5)
    pcts = [0.0, 10.0, 50.0, 90.0, 100.0, 25.0, 75.0]
    batch, stores, outs, kernels = build_batch(specs, percentiles=pcts)
    batch.run(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for sp, out, pct in zip(specs, outs, pcts):
        off = oracle.disk_offsets(sp["r"])
        exp = oracle.median_filter(sp["img"], off, rank=oracle.percentile_rank(len(off), pct))
        assert_bit_exact(to_host(out), exp, f"batch percentile {pct}")


def test_one_shot_batch():
    import torch
    import paper_2505_22938_gb300 as fim
    specs = small_mixed_jobs(seed=17, count=4)
    stores, outs, jobs, ks = [], [], [], []
    for sp in specs:
        store, _ = to_device(sp["img"])
        out = torch.zeros_like(store)
        k = fim.fim_create_kernel_circle(sp["r"])
        h, w = sp["img"].shape
        jobs.append(fim.make_job(store.data_ptr(), out.data_ptr(), w, h, store.stride(0) * store.element_size(),
                                 CODES[sp["img"].dtype], k))
        stores.append(store), outs.append(out), ks.append(k)
    fim.fim_median_batch(jobs, torch.cuda.current_stream().cuda_stream)
    for sp, out in zip(specs, outs):
        assert_bit_exact(to_host(out), oracle.median_filter(sp["img"], oracle.disk_offsets(sp["r"])), "one-shot")


def test_autotune_then_filter():
    import torch
    import paper_2505_22938_gb300 as fim
    img = datagen.config2_image(512, 512)
    store, _ = to_device(img)
    out = torch.empty_like(store)
    k = fim.fim_create_kernel_circle(20)
    try:
        tw, th = fim.fim_autotune(store.data_ptr(), out.data_ptr(), 512, 512, 1024, fim.FIM_U16, k,
                                  torch.cuda.current_stream().cuda_stream)
        plan = fim.fim_plan_info(k, fim.FIM_U16, 512, 512)
        assert (plan["tile_w"], plan["tile_h"]) == (tw, th)
        got = to_host(fim.median(store, k))
        exp = oracle.median_filter(img, oracle.disk_offsets(20))
        assert_bit_exact(got, exp, "after autotune")
        assert_bit_exact(to_host(out), exp, "autotune output")
    finally:
        fim.fim_autotune_clear()


@pytest.mark.parametrize("dtype,r", [("u8", 16), ("u16", 48), ("f32", 64)])
def test_one_job_batch_and_two_job_class(dtype, r):
    """A class of one job runs the single-image kernel over the class's workspace; two jobs of
    the same class run the class kernel. Both match fim_median byte for byte and the oracle on
    sampled pixels (images wide enough for interior tiles, whose footprints the kernels stage)."""
    import torch
    import paper_2505_22938_gb300 as fim
    img = datagen.image_for(dtype, 700 + r, 300, 260)
    store, view = to_device(img, pitch_elems=272)  # rows of a multiple of 16 bytes: staged copies
    k = fim.fim_create_kernel_circle(r)
    ref = fim.median(view, k, out=torch.empty_like(store)[:, :260])
    torch.cuda.synchronize()
    code = {"u8": fim.FIM_U8, "u16": fim.FIM_U16, "f32": fim.FIM_F32}[dtype]
    pitch = store.stride(0) * store.element_size()
    for njobs in (1, 2):
        outs = [torch.empty_like(store) for _ in range(njobs)]
        jobs = [fim.make_job(store.data_ptr(), o.data_ptr(), 260, 300, pitch, code, k) for o in outs]
        batch = fim.fim_batch_create(jobs, [k])
        batch.run(torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert fim.fim_sync_status() == 0
        for o in outs:
            assert_bit_exact(to_host(o[:, :260]), to_host(ref), f"{njobs}-job batch vs fim_median")
    rng = np.random.default_rng(r)
    ys, xs = rng.integers(0, 300, 200), rng.integers(0, 260, 200)
    exp = oracle.median_points(img, oracle.disk_offsets(r), xs.astype(np.int32), ys.astype(np.int32))
    got = to_host(ref)[ys, xs]
    assert np.array_equal(got.view(np.uint8), np.ascontiguousarray(exp).view(np.uint8))
