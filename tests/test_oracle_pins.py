"""Pins of the CPU oracle to facts fixed outside itself (no GPU needed).

Each test checks the oracle against something it does not compute itself: brute-force
sorting on tiny inputs, scipy's median/rank filters (a special case that reduces to a
library routine), closed forms of the kernel geometry, values the paper prints
(tests/golden/), and invariants of the median. The last group plants mistakes in the
oracle's inputs and shows that these pins catch them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import datagen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                vals[k] = int(v)
    return vals


def brute_force(img, offsets, rank):
    """Gather each window by fancy indexing and take a full np.sort (tiny images only)."""
    h, w = img.shape
    yy, xx = np.mgrid[0:h, 0:w]
    wins = []
    for dx, dy in offsets:
        wins.append(img[np.clip(yy + dy, 0, h - 1), np.clip(xx + dx, 0, w - 1)])
    stack = np.stack(wins, axis=-1)
    return np.sort(stack, axis=-1, kind="stable")[..., rank]


def random_image(rng, dtype, h, w):
    if dtype == "u8":
        return rng.integers(0, 256, (h, w), dtype=np.uint8)
    if dtype == "u16":
        return rng.integers(0, 65536, (h, w), dtype=np.uint16)
    a = rng.standard_normal((h, w)).astype(np.float32)
    a[rng.random((h, w)) < 0.05] = np.float32(1e30)
    return a + np.float32(0.0)


def kernel_zoo():
    """Kernels spanning symmetric, asymmetric, even-n and one-row/one-column shapes."""
    return {
        "disk1": oracle.disk_offsets(1),
        "disk2": oracle.disk_offsets(2),
        "disk3": oracle.disk_offsets(3),
        "square3": oracle.spans_offsets([-1] * 3, [1] * 3, -1),
        "ellipse3x1": oracle.ellipse_offsets(3, 1),
        "hexagon3": oracle.polygon_offsets(oracle.regular_polygon_vertices(6, 3.0)),
        "asym": oracle.spans_offsets([0, -1, -2], [2, 1, 0], -2),   # sheared, not symmetric
        "even": oracle.spans_offsets([0, 0], [1, 1], 0),             # 2x2, n = 4
        "row": oracle.spans_offsets([-3], [2], 0),
        "col": oracle.spans_offsets([0] * 4, [0] * 4, -1),
    }


# ----------------------------------------------------------------------------------------
# 1. brute force on tiny inputs
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_brute_force_tiny(dtype):
    rng = np.random.default_rng(7)
    for name, off in kernel_zoo().items():
        for (h, w) in [(1, 1), (1, 7), (6, 1), (9, 13), (16, 16)]:
            img = random_image(rng, dtype, h, w)
            k = oracle.median_rank(len(off))
            got = oracle.median_filter(img, off)
            exp = brute_force(img, off, k)
            assert np.array_equal(np.ascontiguousarray(got).view(np.uint8), np.ascontiguousarray(exp).view(np.uint8)), (name, h, w)
            # every rank, not only the median
            for rank in {0, len(off) - 1, k // 2}:
                got = oracle.median_filter(img, off, rank=rank)
                assert np.array_equal(got, brute_force(img, off, rank)), (name, rank)


def test_exhaustive_binary_3x3():
    """All 512 binary 3x3 images under the 3x3 square and the 5-tap disk."""
    for off in (oracle.spans_offsets([-1] * 3, [1] * 3, -1), oracle.disk_offsets(1)):
        k = oracle.median_rank(len(off))
        for bits in range(512):
            img = np.array([(bits >> i) & 1 for i in range(9)], dtype=np.uint8).reshape(3, 3)
            assert np.array_equal(oracle.median_filter(img, off), brute_force(img, off, k))


def test_points_match_full():
    rng = np.random.default_rng(3)
    img = random_image(rng, "u16", 40, 37)
    off = oracle.disk_offsets(4)
    full = oracle.median_filter(img, off)
    ys, xs = np.mgrid[0:40, 0:37]
    vals = oracle.median_points(img, off, xs.ravel(), ys.ravel())
    assert np.array_equal(vals, full.ravel())


# ----------------------------------------------------------------------------------------
# 1b. spatially varying percentile (Fig. 14): a rank of its own at every pixel
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_rank_map_brute_force_tiny(dtype):
    """Per-pixel ranks against a full sort of every window, pixel by pixel."""
    rng = np.random.default_rng(17)
    for name, off in kernel_zoo().items():
        n = len(off)
        for (h, w) in [(1, 1), (1, 7), (6, 1), (9, 13)]:
            img = random_image(rng, dtype, h, w)
            ranks = rng.integers(0, n, (h, w)).astype(np.int32)
            got = oracle.rank_map_filter(img, off, ranks)
            sorted_wins = {k: brute_force(img, off, k) for k in np.unique(ranks)}
            for y in range(h):
                for x in range(w):
                    assert got[y, x] == sorted_wins[ranks[y, x]][y, x], (name, y, x)


def test_rank_map_scipy_ramp():
    """A left-to-right ramp from the 0th to the 100th percentile (the Fig. 14 setting) on an
    asymmetric kernel: each pixel equals scipy's rank filter at that pixel's rank."""
    nd = pytest.importorskip("scipy.ndimage")
    img = datagen.image_for("u16", 21, 37, 45)
    off = oracle.spans_offsets([0, -1, -2, -2, -1], [3, 2, 2, 1, 0], -2)
    n = len(off)
    pct = np.broadcast_to(np.linspace(0.0, 100.0, 45, dtype=np.float32), (37, 45))
    ranks = oracle.percentile_rank_map(n, pct)
    assert ranks[0, 0] == 0 and ranks[0, -1] == n - 1 and np.all(np.diff(ranks[0]) >= 0)
    got = oracle.rank_map_filter(img, off, ranks)
    for k in np.unique(ranks):
        ref = nd.rank_filter(img, int(k), footprint=_footprint_mask(off), mode="nearest")
        sel = ranks == k
        assert np.array_equal(got[sel], ref[sel]), k
    # a mirrored map (a plausible slip: x read right to left) disagrees
    bad = oracle.rank_map_filter(img, off, ranks[:, ::-1].copy())
    assert not np.array_equal(bad, got)


def test_percentile_rank_map_closed_form():
    """Ranks for n = 81 (n - 1 = 80, so rank = floor(0.8 p + 0.5)), clamping, NaN and infinities."""
    pct = np.array([0.0, 50.0, 100.0, 12.5, 0.625, 0.6249, 99.375, 99.3749, -5.0, 150.0,
                    np.nan, np.inf, -np.inf], dtype=np.float32)
    exp = np.array([0, 40, 80, 10, 1, 0, 80, 79, 0, 80, 0, 80, 0], dtype=np.int32)
    assert np.array_equal(oracle.percentile_rank_map(81, pct), exp)
    # a constant map gives the single-percentile rank
    for p in (0.0, 10.0, 33.3, 50.0, 90.0, 100.0):
        for n in (1, 2, 49, 7845):
            assert oracle.percentile_rank_map(n, np.float32([p]))[0] == oracle.percentile_rank(n, float(np.float32(p)))


def test_constant_rank_map_is_the_percentile_filter():
    rng = np.random.default_rng(4)
    img = random_image(rng, "f32", 23, 29)
    off = oracle.disk_offsets(3)
    for k in (0, 7, len(off) - 1):
        ranks = np.full(img.shape, k, np.int32)
        assert np.array_equal(oracle.rank_map_filter(img, off, ranks), oracle.median_filter(img, off, rank=k))


def test_rank_map_rejects_out_of_range_ranks():
    img = np.zeros((4, 4), np.uint8)
    off = oracle.disk_offsets(1)
    for bad in (-1, len(off)):
        ranks = np.zeros((4, 4), np.int32)
        ranks[2, 3] = bad
        with pytest.raises(ValueError):
            oracle.rank_map_filter(img, off, ranks)


# ----------------------------------------------------------------------------------------
# 10. special case that reduces to a library routine: scipy.ndimage
# ----------------------------------------------------------------------------------------

def _footprint_mask(off):
    rx = int(np.abs(off[:, 0]).max())
    ry = int(np.abs(off[:, 1]).max())
    m = np.zeros((2 * ry + 1, 2 * rx + 1), dtype=bool)
    m[off[:, 1] + ry, off[:, 0] + rx] = True
    return m


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_scipy_median_filter(dtype):
    nd = pytest.importorskip("scipy.ndimage")
    img = datagen.image_for(dtype, 11, 48, 53)
    for off in (oracle.disk_offsets(4), oracle.disk_offsets(7), oracle.ellipse_offsets(5, 2),
                oracle.polygon_offsets(oracle.regular_polygon_vertices(6, 5.0))):
        assert len(off) % 2 == 1
        exp = nd.median_filter(img, footprint=_footprint_mask(off), mode="nearest")
        assert np.array_equal(oracle.median_filter(img, off), exp)


@pytest.mark.parametrize("pct", [0, 10, 25, 50, 75, 90, 100])
def test_scipy_rank_filter(pct):
    nd = pytest.importorskip("scipy.ndimage")
    img = datagen.image_for("u16", 12, 40, 41)
    off = oracle.disk_offsets(5)
    rank = oracle.percentile_rank(len(off), pct)
    exp = nd.rank_filter(img, rank, footprint=_footprint_mask(off), mode="nearest")
    assert np.array_equal(oracle.median_filter(img, off, rank=rank), exp)


# ----------------------------------------------------------------------------------------
# 2-6, 9. invariants of the median
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_radius0_identity(dtype):
    img = datagen.image_for(dtype, 5, 33, 29)
    assert np.array_equal(oracle.median_filter(img, oracle.disk_offsets(0)), img)


@pytest.mark.parametrize("dtype,val", [("u8", 200), ("u16", 4242), ("f32", -3.25)])
def test_constant_fixed_point(dtype, val):
    img = np.full((21, 17), val, dtype=oracle.NP_DTYPE[dtype])
    assert np.array_equal(oracle.median_filter(img, oracle.disk_offsets(5)), img)


def test_monotone_map_invariance():
    """median(f(I)) = f(median(I)) for strictly increasing f (abstract; Sec. 3.2)."""
    img8 = datagen.image_for("u8", 21, 40, 40)
    off = oracle.disk_offsets(4)
    m8 = oracle.median_filter(img8, off)
    # u8 -> u16 by v * 257
    m16 = oracle.median_filter(img8.astype(np.uint16) * 257, off)
    assert np.array_equal(m16, m8.astype(np.uint16) * 257)
    # gamma through a strictly increasing lookup table
    lut = (np.round(65000.0 * (np.arange(256) / 255.0) ** 2.2) + np.arange(256)).astype(np.uint16)
    assert np.all(np.diff(lut.astype(np.int64)) > 0)
    assert np.array_equal(oracle.median_filter(lut[img8], off), lut[m8])
    # float affine map a*v + b, a > 0, exactly representable
    imgf = img8.astype(np.float32)
    mf = oracle.median_filter(imgf * np.float32(0.5) - np.float32(3.0), off)
    assert np.array_equal(mf, m8.astype(np.float32) * np.float32(0.5) - np.float32(3.0))
    # a decreasing map turns rank k into rank n-1-k
    n = len(off)
    k = oracle.median_rank(n)
    assert np.array_equal(oracle.median_filter(255 - img8, off, rank=n - 1 - k), 255 - m8)


@pytest.mark.parametrize("dtype", ["u16", "f32"])
def test_membership_and_rank_counts(dtype):
    """out is a window member and #{w < m} <= k <= #{w <= m} - 1, checked per pixel."""
    img = datagen.image_for(dtype, 31, 30, 34)
    off = oracle.ellipse_offsets(4, 3)
    n = len(off)
    k = oracle.median_rank(n)
    out = oracle.median_filter(img, off)
    h, w = img.shape
    for y in range(h):
        for x in range(w):
            win = np.array([img[min(max(y + dy, 0), h - 1), min(max(x + dx, 0), w - 1)] for dx, dy in off])
            m = out[y, x]
            assert np.any(win == m)
            assert np.sum(win < m) <= k <= np.sum(win <= m) - 1


def test_odd_tap_count_for_centrally_symmetric():
    for r in range(0, 40):
        assert len(oracle.disk_offsets(r)) % 2 == 1
    hexagon = oracle.polygon_offsets(oracle.regular_polygon_vertices(6, 64.0))
    ell = oracle.ellipse_offsets(80, 40)
    for off in (hexagon, ell):
        assert len(off) % 2 == 1
        s = set(map(tuple, off))
        assert all((-a, -b) in s for a, b in s)


def test_transpose_and_flip_symmetry():
    img = datagen.image_for("u16", 41, 37, 45)
    off = oracle.spans_offsets([0, -1, -2], [3, 1, 0], -1)  # asymmetric
    out = oracle.median_filter(img, off)
    t_off = off[:, ::-1].copy()
    assert np.array_equal(oracle.median_filter(np.ascontiguousarray(img.T), t_off), out.T)
    f_off = off * np.array([-1, 1], dtype=np.int32)
    assert np.array_equal(oracle.median_filter(np.ascontiguousarray(img[:, ::-1]), f_off), out[:, ::-1])


def test_float_total_order_signed_zero():
    """-0 < +0 under the float ordering (Sec. 4.1 float key); values otherwise numeric."""
    img = np.array([[-0.0, 0.0, -0.0]], dtype=np.float32)
    off = oracle.spans_offsets([-1], [1], 0)
    lo = oracle.median_filter(img, off, rank=0)
    hi = oracle.median_filter(img, off, rank=2)
    assert np.signbit(lo[0, 1]) and not np.signbit(hi[0, 1])
    sub = np.array([[1e-45, -1e-45, 0.0, 2e-45, -3e-45]], dtype=np.float32)  # denormals
    exp = brute_force(sub, off, 1)
    assert np.array_equal(oracle.median_filter(sub, off), exp)


# ----------------------------------------------------------------------------------------
# 7-8. geometry closed forms and the paper's printed counts
# ----------------------------------------------------------------------------------------

def disk_count_closed_form(r, limit):
    """Sum over rows of 2*floor(sqrt(limit - dy^2)) + 1 (integer square root)."""
    return sum(2 * math.isqrt(limit - dy * dy) + 1 for dy in range(-r, r + 1) if dy * dy <= limit)


def test_disk_counts_closed_form():
    for r in list(range(0, 20)) + [32, 48, 64, 100, 128]:
        assert len(oracle.disk_offsets(r)) == disk_count_closed_form(r, r * r)
        assert len(oracle.disk_limit_offsets(r, r * r + r)) == disk_count_closed_form(r, r * r + r)
    # Gauss circle problem values: N(10) = 317, N(100) = 31417
    assert len(oracle.disk_offsets(10)) == 317
    assert len(oracle.disk_offsets(100)) == 31417


def test_paper_geometry_counts():
    g = read_golden("paper_geometry.txt")
    # Fig. 3b: 5x5 square without corners
    sq5 = oracle.spans_offsets([-2] * 5, [2] * 5, -2)
    no_corners = np.array([p for p in sq5 if not (abs(p[0]) == 2 and abs(p[1]) == 2)], dtype=np.int32)
    assert len(no_corners) == g["fig3b_taps_5x5_circle"]
    assert len(oracle.disk_limit_offsets(2, 2 * 2 + 2)) == g["fig3b_taps_5x5_circle"]
    # Fig. 10 under the fuller disk reading dx^2 + dy^2 <= r^2 + r
    k48 = oracle.disk_limit_offsets(48, 48 * 48 + 48)
    N = oracle.tile_footprint_size(k48, 64, 64)
    assert N == g["fig10_footprint_r48_t64"]
    assert oracle.candidate_median_ranks(len(k48), N) == g["fig10_candidate_ranks_r48_t64"]
    assert 64 + 2 * 48 == g["fig10_footprint_side_r48_t64"]
    # the workload disk dx^2 + dy^2 <= r^2 leaves the candidate range unchanged
    k48b = oracle.disk_offsets(48)
    Nb = oracle.tile_footprint_size(k48b, 64, 64)
    assert (len(k48b), Nb) == (7213, 23404)
    assert oracle.candidate_median_ranks(len(k48b), Nb) == g["fig10_candidate_ranks_r48_t64"]
    # Sec. 3.1: 7x7 square, median is the 25th value
    sq7 = oracle.spans_offsets([-3] * 7, [3] * 7, -3)
    assert len(sq7) == g["sec31_square7_taps"]
    assert oracle.median_rank(len(sq7)) + 1 == g["sec31_square7_median_1based"]
    # Fig. 6: a 13-wide circle is the radius-6 disk
    d6 = oracle.disk_offsets(6)
    assert d6[:, 0].max() - d6[:, 0].min() + 1 == g["fig6_circle_width"]
    # Sec. 4.1: 128x128 input tile, pivots at multiples of 64 -> at most 256 pivot values
    side = g["sec41_pivot8_max_tile_side"]
    assert side * side // g["sec41_pivot_quantum"] == 256
    assert g["sec41_max_input_tile_side"] ** 2 == 1 << 16


def test_config_kernel_counts():
    """Tap counts of the workload kernels (all centrally symmetric, so all odd)."""
    assert len(oracle.disk_offsets(4)) == 49
    hexagon = oracle.polygon_offsets(oracle.regular_polygon_vertices(6, 64.0))
    assert len(hexagon) == 10651
    assert hexagon[:, 0].min() == -64 and hexagon[:, 0].max() == 64
    assert hexagon[:, 1].min() == -55 and hexagon[:, 1].max() == 55
    assert len(oracle.ellipse_offsets(80, 40)) == 10041


def test_ellipse_rows_closed_form_and_orientation():
    """Row dy of the ellipse with semi-axis a along x and b along y holds the dx with
    dx^2 b^2 <= a^2 (b^2 - dy^2), i.e. |dx| <= isqrt(a^2 (b^2 - dy^2)) // b: 2 * that + 1
    taps. The x extent is +-a and the y extent +-b, so a swapped (a, b) fails."""
    for a, b in ((80, 40), (5, 2), (2, 5), (7, 7), (13, 4), (1, 9)):
        off = oracle.ellipse_offsets(a, b)
        assert off[:, 0].min() == -a and off[:, 0].max() == a, (a, b)
        assert off[:, 1].min() == -b and off[:, 1].max() == b, (a, b)
        for dy in range(-b, b + 1):
            half = math.isqrt(a * a * (b * b - dy * dy)) // b
            row = np.sort(off[off[:, 1] == dy, 0])
            assert np.array_equal(row, np.arange(-half, half + 1)), (a, b, dy)
        if a != b:
            assert not np.array_equal(np.sort(off, axis=0), np.sort(oracle.ellipse_offsets(b, a), axis=0))


def _pick_count(verts):
    """Lattice points inside or on a polygon with integer vertices by Pick's theorem:
    A = I + B/2 - 1, so I + B = A + B/2 + 1 (A by the shoelace formula, B = sum over the edges
    of gcd(|dx|, |dy|))."""
    m = len(verts)
    twice_area = 0
    boundary = 0
    for i in range(m):
        (x0, y0), (x1, y1) = verts[i], verts[(i + 1) % m]
        twice_area += x0 * y1 - x1 * y0
        boundary += math.gcd(abs(x1 - x0), abs(y1 - y0))
    assert twice_area > 0, "counter-clockwise"
    return (twice_area + boundary) // 2 + 1


def test_polygon_counts_pick_theorem():
    """Convex polygons with lattice vertices (triangles, a skew quadrilateral, an irregular
    hexagon, a thin sliver): the rasteriser's point count equals Pick's theorem, every vertex
    is included, and mirroring the polygon mirrors the point set."""
    polys = [
        [(0, 0), (7, 0), (0, 5)],
        [(-3, -2), (4, -1), (1, 6)],
        [(-5, -1), (2, -4), (6, 3), (-1, 5)],
        [(-6, 0), (-3, -5), (3, -5), (6, 0), (3, 5), (-3, 5)],
        [(-9, -1), (9, 0), (-9, 1)],
        [(0, 0), (11, 3), (4, 8)],
    ]
    for verts in polys:
        off = oracle.polygon_offsets(np.asarray(verts, dtype=np.float64))
        assert len(off) == _pick_count(verts), verts
        pts = {tuple(p) for p in off.tolist()}
        assert all(tuple(v) in pts for v in verts)
        mirrored = [(-x, y) for x, y in reversed(verts)]  # mirrored in x, still counter-clockwise
        moff = oracle.polygon_offsets(np.asarray(mirrored, dtype=np.float64))
        assert {(-x, y) for x, y in moff.tolist()} == pts


def test_fig4_ordinal_example():
    """Fig. 4: ties get consecutive ordinals, and a window's median value and median ordinal
    correspond through the reverse map."""
    rows = np.loadtxt(os.path.join(GOLDEN, "fig4_ordinal.txt"), dtype=np.int64)
    card = rows[:, 1]
    # ordinal transform by a stable argsort: equal values receive consecutive ordinals
    order = np.argsort(card, kind="stable")
    ordinal = np.empty_like(order)
    ordinal[order] = np.arange(len(card))
    assert list(ordinal) == list(rows[:, 0])
    tied = ordinal[card == 29]
    assert sorted(tied) == [3, 4]
    # a 4x4 image holding these values (rest larger), its ordinal image, and the median of
    # each 3x3 window both ways: cardinal median == reverse_map[ordinal median]
    rng = np.random.default_rng(4)
    vals = np.concatenate([card, 42 + rng.permutation(10)]).astype(np.uint16)
    img = rng.permutation(vals).reshape(4, 4)
    flat = img.ravel()
    o = np.empty(16, dtype=np.int64)
    o[np.argsort(flat, kind="stable")] = np.arange(16)
    ordimg = o.reshape(4, 4).astype(np.uint16)
    reverse = np.sort(flat)
    off = oracle.spans_offsets([-1] * 3, [1] * 3, -1)
    assert np.array_equal(oracle.median_filter(img, off), reverse[oracle.median_filter(ordimg, off)])


# ----------------------------------------------------------------------------------------
# 11. planted mistakes: each plausible slip in the oracle's inputs is caught by a pin
# ----------------------------------------------------------------------------------------

def test_planted_mistakes_are_caught():
    nd = pytest.importorskip("scipy.ndimage")
    img = datagen.image_for("u16", 51, 32, 35)
    off = oracle.spans_offsets([0, -1, -2, -2], [3, 2, 1, 0], -1)  # asymmetric, n = 15
    n = len(off)
    k = oracle.median_rank(n)
    exp = brute_force(img, off, k)
    assert np.array_equal(oracle.median_filter(img, off), exp)
    assert np.array_equal(exp, nd.median_filter(img, footprint=_footprint_mask(off), mode="nearest"))
    mistakes = {
        "rank off by one": dict(offsets=off, rank=k + 1),
        "transposed offsets": dict(offsets=off[:, ::-1].copy(), rank=k),
        "dy sign flipped": dict(offsets=off * np.array([1, -1], dtype=np.int32), rank=k),
        "dropped tap": dict(offsets=off[1:].copy(), rank=oracle.median_rank(n - 1)),
    }
    for name, kw in mistakes.items():
        bad = oracle.median_filter(img, kw["offsets"], rank=kw["rank"])
        assert not np.array_equal(bad, exp), name
    # a wrong border mode (wrap instead of clamp) also disagrees with the brute force
    wrapped = nd.median_filter(img, footprint=_footprint_mask(off), mode="wrap")
    assert not np.array_equal(wrapped, exp)
