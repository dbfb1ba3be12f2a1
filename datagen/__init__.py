"""Seeded synthetic inputs shaped like the median filter's workloads.

This module only draws images. It holds no part of the median filter's
arithmetic, so both the CPU oracle (``oracle/``) and the CUDA path can take
their inputs from it without sharing any of the method's code.

The paper benchmarks on photographs (a 37-megapixel greyscale photo, Sec. 5),
which are not available here. The recipes below stand in for them with the same
structure: smooth low-frequency content, sharp step edges, impulse noise for
16-bit data, and heavy-tailed outliers for float data.

Every generator is a pure function of its arguments. Seeds follow
``seed = 20250522 + config_index * 1000 + image_index``.
"""
from __future__ import annotations

import math

import numpy as np

try:  # multithreaded FFT when scipy is present; numpy's FFT otherwise
    import scipy.fft as _fft

    def _rfft2(a):
        return _fft.rfft2(a, workers=-1)

    def _irfft2(a, s):
        return _fft.irfft2(a, s=s, workers=-1)
except Exception:  # pragma: no cover - scipy is optional
    def _rfft2(a):
        return np.fft.rfft2(a)

    def _irfft2(a, s):
        return np.fft.irfft2(a, s=s)

SEED_BASE = 20250522


def seed_for(config_index: int, image_index: int = 0) -> int:
    """Seed of image ``image_index`` of workload ``config_index`` (1-based)."""
    return SEED_BASE + config_index * 1000 + image_index


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def smooth_field(rng: np.random.Generator, h: int, w: int, sigma: float) -> np.ndarray:
    """White noise smoothed by a periodic Gaussian of std ``sigma`` px, scaled to unit variance."""
    noise = rng.standard_normal((h, w), dtype=np.float32)
    fy = np.fft.fftfreq(h).astype(np.float32)[:, None]
    fx = np.fft.rfftfreq(w).astype(np.float32)[None, :]
    # Fourier transform of a unit-area Gaussian of std sigma (frequencies in cycles/px).
    g = np.exp(np.float32(-2.0 * math.pi ** 2 * sigma ** 2) * (fy * fy + fx * fx))
    out = _irfft2(_rfft2(noise) * g, s=(h, w)).astype(np.float32)
    # Per-pixel variance of filtered unit white noise is the mean of |G|^2 over the full
    # frequency grid; dividing by it (not by the sample std) keeps small images sane.
    fxf = np.fft.fftfreq(w).astype(np.float64)[None, :]
    gfull = np.exp(-2.0 * math.pi ** 2 * sigma ** 2 * (fy.astype(np.float64) ** 2 + fxf * fxf))
    sd = math.sqrt(float(np.mean(gfull * gfull)))
    return out / np.float32(sd)


def _convex_polygon_mask(rng: np.random.Generator, h: int, w: int,
                         rscale: float = 1.0) -> tuple[np.ndarray, tuple[int, int]]:
    """Random convex polygon (3-8 vertices, radius 64-1024 px times ``rscale``) as a boolean
    mask over its bounding box."""
    nv = int(rng.integers(3, 9))
    rad = float(rng.uniform(64, 1024)) * rscale
    cx, cy = float(rng.uniform(0, w)), float(rng.uniform(0, h))
    ang = np.sort(rng.uniform(0, 2 * math.pi, nv))
    vx = cx + rad * np.cos(ang)
    vy = cy + rad * np.sin(ang)
    x0, x1 = max(0, int(math.floor(vx.min()))), min(w - 1, int(math.ceil(vx.max())))
    y0, y1 = max(0, int(math.floor(vy.min()))), min(h - 1, int(math.ceil(vy.max())))
    if x1 < x0 or y1 < y0:
        return np.zeros((0, 0), bool), (0, 0)
    yy, xx = np.mgrid[y0:y1 + 1, x0:x1 + 1].astype(np.float32)
    inside = np.ones(xx.shape, bool)
    for i in range(nv):  # vertices sorted by angle are counter-clockwise
        ax, ay = vx[i], vy[i]
        bx, by = vx[(i + 1) % nv], vy[(i + 1) % nv]
        inside &= (bx - ax) * (yy - ay) - (by - ay) * (xx - ax) >= 0
    return inside, (y0, x0)


def photo_u16(seed: int, h: int, w: int, n_polygons: int = 32, impulse_frac: float = 0.05) -> np.ndarray:
    """16-bit photo-like image: Gaussian fields (sigma 2, 16, 64), polygon step edges, salt-and-pepper.

    The polygon radii are 64-1024 px for a 4096x4096 image and scale with sqrt(h*w)/4096
    otherwise, so the fraction of the image the edges cover does not depend on its size."""
    rng = _rng(seed)
    rscale = math.sqrt(h * w) / 4096.0
    f = (smooth_field(rng, h, w, 2.0) + smooth_field(rng, h, w, 16.0) + smooth_field(rng, h, w, 64.0))
    img = np.float32(32768.0) + np.float32(8192.0 / math.sqrt(3.0)) * f
    for _ in range(n_polygons):
        mask, (y0, x0) = _convex_polygon_mask(rng, h, w, rscale)
        if mask.size:
            step = np.float32(rng.uniform(-12000, 12000))
            img[y0:y0 + mask.shape[0], x0:x0 + mask.shape[1]] += np.where(mask, step, np.float32(0))
    out = np.clip(np.rint(img), 0, 65535).astype(np.uint16)
    n_imp = int(round(impulse_frac * h * w))
    if n_imp:
        idx = rng.choice(h * w, size=n_imp, replace=False)
        vals = np.where(rng.random(n_imp) < 0.5, 0, 65535).astype(np.uint16)
        out.reshape(-1)[idx] = vals
    return out


def uniform_u8(seed: int, h: int, w: int) -> np.ndarray:
    """i.i.d. uniform 8-bit noise."""
    return _rng(seed).integers(0, 256, size=(h, w), dtype=np.uint8)


def field_f32(seed: int, h: int, w: int, outlier_frac: float = 0.01, cauchy_scale: float = 10.0) -> np.ndarray:
    """Float image: unit-variance mix of Gaussian fields plus Cauchy outliers; no NaN/Inf, no -0.0."""
    rng = _rng(seed)
    f = smooth_field(rng, h, w, 2.0) + smooth_field(rng, h, w, 16.0) + smooth_field(rng, h, w, 64.0)
    f /= np.float32(max(float(f.std()), 1e-30))
    n_out = int(round(outlier_frac * h * w))
    if n_out:
        idx = rng.choice(h * w, size=n_out, replace=False)
        c = np.clip(cauchy_scale * rng.standard_cauchy(n_out), -1e30, 1e30).astype(np.float32)
        f.reshape(-1)[idx] += c
    f = f.astype(np.float32)
    f[~np.isfinite(f)] = 0.0
    f += np.float32(0.0)  # maps -0.0 to +0.0
    return f


# --------------------------------------------------------------------------------------
# The five workloads.
# --------------------------------------------------------------------------------------

CONFIG1 = dict(name="u8 256x256 uniform, disk r=4", dtype="u8", h=256, w=256, radii=(4,))
CONFIG2 = dict(name="u16 4096x4096 photo-like, disks r=8/32/48", dtype="u16", h=4096, w=4096, radii=(8, 32, 48))
CONFIG3 = dict(name="f32 8192x8192 fields+Cauchy, disks r=64/100, hexagon R=64, ellipse 80x40",
               dtype="f32", h=8192, w=8192, radii=(64, 100))
CONFIG4 = dict(name="u16 6000x4000x3 photo-like planes, disk r=48", dtype="u16", h=4000, w=6000, channels=3,
               radii=(48,))


def config1_image(h: int = 256, w: int = 256) -> np.ndarray:
    return uniform_u8(seed_for(1), h, w)


def config2_image(h: int = 4096, w: int = 4096, image_index: int = 0) -> np.ndarray:
    return photo_u16(seed_for(2, image_index), h, w)


def config3_image(h: int = 8192, w: int = 8192, image_index: int = 0) -> np.ndarray:
    return field_f32(seed_for(3, image_index), h, w)


def config4_planes(h: int = 4000, w: int = 6000) -> list[np.ndarray]:
    return [photo_u16(seed_for(4, c), h, w) for c in range(3)]


def config4_training_image(index: int, side: int = 1024) -> np.ndarray:
    """Training images for the rank-bracket predictor (disjoint seeds from the evaluation planes)."""
    return photo_u16(seed_for(4, 100 + index), side, side)


def config5_jobs(count: int = 64, lo: int = 512, hi: int = 4096, seed: int | None = None) -> list[dict]:
    """(w, h, dtype, r) for the mixed batch: sides uniform in [lo, hi], r log-uniform in [2, 128]."""
    rng = _rng(seed_for(5) if seed is None else seed)
    jobs = []
    for i in range(count):
        w = int(rng.integers(lo, hi + 1))
        h = int(rng.integers(lo, hi + 1))
        dtype = ("u8", "u16", "f32")[int(rng.integers(0, 3))]
        r = int(round(math.exp(rng.uniform(math.log(2.0), math.log(128.0)))))
        jobs.append(dict(index=i, w=w, h=h, dtype=dtype, r=r, seed=seed_for(5, 1 + i)))
    return jobs


def config5_image(job: dict) -> np.ndarray:
    if job["dtype"] == "u8":
        return uniform_u8(job["seed"], job["h"], job["w"])
    if job["dtype"] == "u16":
        return photo_u16(job["seed"], job["h"], job["w"])
    return field_f32(job["seed"], job["h"], job["w"])


def image_for(dtype: str, seed: int, h: int, w: int) -> np.ndarray:
    """Any-size image of the given dtype with that dtype's workload recipe."""
    if dtype == "u8":
        return uniform_u8(seed, h, w)
    if dtype == "u16":
        return photo_u16(seed, h, w)
    if dtype == "f32":
        return field_f32(seed, h, w)
    raise ValueError(dtype)


def adversarial_tile(h: int, w: int, dtype: str = "u16", border: int = 24) -> np.ndarray:
    """High-frequency black/white checkerboard inside a thick mid-grey frame (Sec. 6 stress case)."""
    hi = {"u8": 255, "u16": 65535, "f32": 1.0}[dtype]
    mid = {"u8": 128, "u16": 32768, "f32": 0.5}[dtype]
    npd = {"u8": np.uint8, "u16": np.uint16, "f32": np.float32}[dtype]
    yy, xx = np.mgrid[0:h, 0:w]
    img = np.where((xx + yy) % 2 == 0, 0, hi).astype(npd)
    frame = (xx < border) | (yy < border) | (xx >= w - border) | (yy >= h - border)
    img[frame] = mid
    return img


# --------------------------------------------------------------------------------------
# The same recipes drawn on a CUDA device with torch (fast inputs for large benchmarks).
# Same structure and parameters; the random streams differ from the numpy versions.
# --------------------------------------------------------------------------------------

def _torch_field(gen, h, w, sigma, device):
    import torch
    noise = torch.randn((h, w), generator=gen, device=device, dtype=torch.float32)
    fy = torch.fft.fftfreq(h, device=device)[:, None]
    fx = torch.fft.rfftfreq(w, device=device)[None, :]
    g = torch.exp(-2.0 * math.pi ** 2 * sigma ** 2 * (fy * fy + fx * fx))
    out = torch.fft.irfft2(torch.fft.rfft2(noise) * g, s=(h, w))
    fxf = torch.fft.fftfreq(w, device=device, dtype=torch.float64)[None, :]
    gfull = torch.exp(-2.0 * math.pi ** 2 * sigma ** 2 * (fy.double() ** 2 + fxf * fxf))
    return out / math.sqrt(float((gfull * gfull).mean()))


def torch_photo_u16(seed: int, h: int, w: int, device="cuda", n_polygons: int = 32, impulse_frac: float = 0.05):
    """photo_u16's recipe on the GPU (int16 storage view of uint16 data is returned as torch.uint16)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    f = sum(_torch_field(gen, h, w, s, device) for s in (2.0, 16.0, 64.0))
    img = 32768.0 + (8192.0 / math.sqrt(3.0)) * f
    rng = _rng(seed)
    rscale = math.sqrt(h * w) / 4096.0
    yy = torch.arange(h, device=device, dtype=torch.float32)[:, None]
    xx = torch.arange(w, device=device, dtype=torch.float32)[None, :]
    for _ in range(n_polygons):
        nv = int(rng.integers(3, 9))
        rad = float(rng.uniform(64, 1024)) * rscale
        cx, cy = float(rng.uniform(0, w)), float(rng.uniform(0, h))
        ang = np.sort(rng.uniform(0, 2 * math.pi, nv))
        vx, vy = cx + rad * np.cos(ang), cy + rad * np.sin(ang)
        inside = torch.ones((h, w), dtype=torch.bool, device=device)
        for i in range(nv):
            ax, ay, bx, by = vx[i], vy[i], vx[(i + 1) % nv], vy[(i + 1) % nv]
            inside &= (bx - ax) * (yy - ay) - (by - ay) * (xx - ax) >= 0
        img += inside.float() * float(rng.uniform(-12000, 12000))
    out = torch.clamp(torch.round(img), 0, 65535).to(torch.int32)
    imp = torch.rand((h, w), generator=gen, device=device) < impulse_frac
    hi = torch.rand((h, w), generator=gen, device=device) < 0.5
    out = torch.where(imp, torch.where(hi, 65535, 0), out)
    return out.to(torch.int32).to(torch.uint16) if hasattr(torch, "uint16") else out


def torch_field_f32(seed: int, h: int, w: int, device="cuda", outlier_frac: float = 0.01, cauchy_scale: float = 10.0):
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    f = sum(_torch_field(gen, h, w, s, device) for s in (2.0, 16.0, 64.0))
    f = f / max(float(f.std()), 1e-30)
    mask = torch.rand((h, w), generator=gen, device=device) < outlier_frac
    u = torch.rand((h, w), generator=gen, device=device, dtype=torch.float64)
    c = torch.clamp(cauchy_scale * torch.tan(math.pi * (u - 0.5)), -1e30, 1e30).float()
    f = torch.where(mask, f + c, f)
    f = torch.nan_to_num(f, nan=0.0, posinf=0.0, neginf=0.0)
    return f + 0.0


def torch_uniform_u8(seed: int, h: int, w: int, device="cuda"):
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    return torch.randint(0, 256, (h, w), generator=gen, device=device, dtype=torch.uint8)


def torch_config5_image(job: dict, device="cuda"):
    if job["dtype"] == "u8":
        return torch_uniform_u8(job["seed"], job["h"], job["w"], device)
    if job["dtype"] == "u16":
        return torch_photo_u16(job["seed"], job["h"], job["w"], device)
    return torch_field_f32(job["seed"], job["h"], job["w"], device)
