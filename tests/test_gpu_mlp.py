"""Rank-bracket network on the GPU: forward and gradient against the fp64 oracle on the same
bf16 weights, training, checkpoints, and bit-exact filtering with untrained and trained nets."""
import os
import tempfile

import numpy as np
import pytest

import datagen
import oracle
from oracle import mlp
from helpers import assert_bit_exact, to_device, to_host

pytestmark = pytest.mark.gpu
ROW = 42


def _rows(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (n, 41)).astype(np.float32)
    y = rng.uniform(0, 1, n).astype(np.float32)
    return np.concatenate([x, y[:, None]], axis=1)


def test_forward_matches_oracle():
    import torch
    import paper_2505_22938_gb300 as fim
    m = fim.Model.create(seed=5)
    rows = _rows(300, 1)
    d = torch.from_numpy(rows).cuda()
    out = torch.empty((300, 2), dtype=torch.float32, device="cuda")
    m.forward(d.data_ptr(), 300, ROW, out.data_ptr())
    _, bits = m.params()
    exp, _ = mlp.forward(mlp.bf16_values(bits), rows[:, :41].astype(np.float64))
    got = out.cpu().numpy().astype(np.float64)
    assert np.allclose(got, exp, rtol=1e-4, atol=1e-5), np.abs(got - exp).max()


def test_gradient_matches_oracle():
    import torch
    import paper_2505_22938_gb300 as fim
    m = fim.Model.create(seed=7)
    rows = _rows(512, 2)
    d = torch.from_numpy(rows).cuda()
    g = torch.empty(fim.Model.param_count(), dtype=torch.float32, device="cuda")
    loss = m.loss_grad(d.data_ptr(), 512, ROW, d.data_ptr() + 41 * 4, ROW, g.data_ptr())
    _, bits = m.params()
    eloss, eg = mlp.loss_and_grad(mlp.bf16_values(bits), rows[:, :41].astype(np.float64),
                                  rows[:, 41].astype(np.float64))
    got = g.cpu().numpy().astype(np.float64)
    assert abs(loss - eloss) <= 1e-4 * abs(eloss) + 1e-6
    scale = np.abs(eg).max()
    assert np.abs(got - eg).max() <= 1e-3 * scale + 1e-7, (np.abs(got - eg).max(), scale)


def test_training_reduces_loss_and_checkpoint_round_trip():
    import torch
    import paper_2505_22938_gb300 as fim
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1, (8192, 41)).astype(np.float32)
    a = rng.normal(0, 0.5, 41)
    y = (1 / (1 + np.exp(-(x @ a)))).astype(np.float32)
    rows = np.concatenate([x, y[:, None]], axis=1)
    d = torch.from_numpy(rows).cuda()
    m = fim.Model.create(seed=11)
    first = m.train(d.data_ptr(), 8192, 1, 1024, 1e-3)
    last = m.train(d.data_ptr(), 8192, 20, 1024, 1e-3)
    assert last < first - 0.5, (first, last)
    z = m.calibrate(d.data_ptr(), 8192, 0.95)
    assert 0 < z < 10 and abs(m.bracket_z - z) < 1e-6
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "m.bin")
        m.save(path)
        m2 = fim.Model.load(path)
        f1, b1 = m.params()
        f2, b2 = m2.params()
        assert np.array_equal(f1, f2) and np.array_equal(b1, b2) and m2.bracket_z == m.bracket_z


def _learned(img, kernel, model):
    import torch
    import paper_2505_22938_gb300 as fim
    store, _ = to_device(img)
    out = torch.zeros_like(store)
    stats = torch.zeros(5, dtype=torch.int64, device="cuda")
    h, w = img.shape
    fim.fim_median_learned(store.data_ptr(), out.data_ptr(), w, h, store.stride(0) * store.element_size(),
                           {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1, np.dtype(np.float32): 2}[img.dtype],
                           kernel, model, torch.cuda.current_stream().cuda_stream, stats.data_ptr())
    torch.cuda.synchronize()
    assert fim.fim_sync_status() == 0
    return to_host(out), stats.cpu().numpy()


@pytest.mark.parametrize("r", [8, 24])  # small-CTA tiles (scan width read at run time) and 1024-thread tiles
@pytest.mark.parametrize("dtype", ["u16", "f32", "u8"])
def test_untrained_bracket_is_still_exact(dtype, r):
    import paper_2505_22938_gb300 as fim
    img = datagen.image_for(dtype, 71, 150, 170)
    k = fim.fim_create_kernel_circle(r)
    got, st = _learned(img, k, fim.Model.create(seed=3))
    assert_bit_exact(got, oracle.median_filter(img, oracle.disk_offsets(r)), "untrained bracket")
    assert st[0] > 0 and st[1] + st[2] + st[3] == st[0]


def _train_on_photos(k, r, images=6, side=512):
    """Training rows from the plain path's seed windows on photo-like images (labels: exact
    medians), checked against the oracle on the first image; returns (rows tensor, count)."""
    import torch
    import paper_2505_22938_gb300 as fim
    cap = 1 << 16
    rows = torch.zeros((cap, ROW), dtype=torch.float32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    for i in range(images):
        img = datagen.config2_image(side, side, image_index=50 + i)
        store, _ = to_device(img)
        out = torch.empty_like(store)
        fim.fim_collect_seed_samples(store.data_ptr(), out.data_ptr(), side, side, side * 2, fim.FIM_U16, k,
                                     rows.data_ptr(), cap, count.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        if i == 0:
            ys, xs = np.mgrid[0:side:37, 0:side:41]
            assert np.array_equal(to_host(out)[ys, xs].ravel(),
                                  oracle.median_points(img, oracle.disk_offsets(r), xs.ravel(), ys.ravel()))
    n = int(count.item())
    return rows[:n], n


def test_trained_network_shortens_the_walk():
    """What the trained network gains over the same exact seed solve without it: a constant
    predictor (every seed's median guessed at the middle of the tile's feasible ranks, its bracket
    calibrated on the same rows) against the network trained on photo-like seeds. Both give the
    oracle's bytes; the network walks fewer omnigram ranks per seed."""
    import paper_2505_22938_gb300 as fim
    r = 48
    k = fim.fim_create_kernel_circle(r)
    data, n = _train_on_photos(k, r, images=8)
    assert n > 500
    trained = fim.Model.create(seed=1)
    trained.train(data.data_ptr(), n, 40, 512, 2e-3)
    trained.calibrate(data.data_ptr(), n, 0.9)
    const = fim.Model.create(seed=1)
    w = np.zeros(fim.Model.param_count(), np.float32)
    w[-2:] = [0.5, np.log(0.25)]  # output bias: mu = middle of the feasible ranks, log sigma
    const.set_params(w)
    const.calibrate(data.data_ptr(), n, 0.9)
    img = datagen.config2_image(384, 320, image_index=98)
    exp = oracle.median_filter(img, oracle.disk_offsets(r))
    got_t, st_t = _learned(img, k, trained)
    got_c, st_c = _learned(img, k, const)
    assert_bit_exact(got_t, exp, "trained network")
    assert_bit_exact(got_c, exp, "constant predictor")
    walk_t = st_t[4] / st_t[0]
    walk_c = st_c[4] / st_c[0]
    assert walk_t < 0.8 * walk_c, (walk_t, walk_c)


def test_trained_bracket_exact_and_hits():
    """Train on seeds of a few photo-like images, then filter a new one: same bytes as the plain
    path, and most seed windows land inside the predicted bracket."""
    import torch
    import paper_2505_22938_gb300 as fim
    k = fim.fim_create_kernel_circle(32)
    cap = 1 << 16
    rows = torch.zeros((cap, ROW), dtype=torch.float32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    for i in range(6):
        img = datagen.config2_image(512, 512, image_index=50 + i)
        store, _ = to_device(img)
        out = torch.empty_like(store)
        fim.fim_collect_seed_samples(store.data_ptr(), out.data_ptr(), 512, 512, 1024, fim.FIM_U16, k,
                                     rows.data_ptr(), cap, count.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        if i == 0:  # the plain filter still produced the exact image
            ys, xs = np.mgrid[0:512:37, 0:512:41]
            assert np.array_equal(to_host(out)[ys, xs].ravel(),
                                  oracle.median_points(img, oracle.disk_offsets(32), xs.ravel(), ys.ravel()))
    n = int(count.item())
    assert n > 1000
    data = rows[:n]
    assert float(data[:, 41].min()) >= 0.0 and float(data[:, 41].max()) <= 1.0
    m = fim.Model.create(seed=1)
    m.train(data.data_ptr(), n, 40, 512, 2e-3)
    m.calibrate(data.data_ptr(), n, 0.9)
    img = datagen.config2_image(300, 280, image_index=99)
    got, st = _learned(img, k, m)
    assert_bit_exact(got, oracle.median_filter(img, oracle.disk_offsets(32)), "trained bracket")
    assert st[1] >= 0.5 * st[0], st
