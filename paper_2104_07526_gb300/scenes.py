"""Seeded synthetic point clouds and cameras.

This module only makes inputs.  It holds none of the rendering method's
arithmetic: no projection, no depth keys, no Morton codes.  The CUDA path and
the CPU oracle both take the bytes it produces.

Point record: 16 bytes, ``float32 x, y, z`` then ``uint32 rgba``, with r in the
low byte.  The paper uses the same record size (12.7 GB for 796M points, §5,
Table "scenarios").  Clouds come back as ``torch.int32`` tensors of shape
``(n, 4)``.  Column 3 holds the rgba word and columns 0-2 hold float32 bit
patterns.

Randomness is counter based.  Each draw is the MurmurHash3 64-bit finaliser of
``(seed, stream, index)``, so a chunk can be generated on its own, on CPU or
GPU, with the same integer streams.  Transcendental functions (sin, cos, sqrt)
may differ by an ulp between devices.  Callers that compare two renderers
therefore generate a cloud once and hand the same bytes to both.

Recipes (the paper's datasets are not available; these stand in for them):

* ``sphere_plane``: the 1M-point case.  Half the points lie on the unit
  sphere, half on the plane z=-1 over [-2,2]^2.  Colours are uniform bytes.
* ``boxes``: the 50M-point case.  200 axis-aligned boxes (sides 0.1-5 m) on a
  100x100 m ground plane, 2 mm jitter, one hue per box.
* ``scan``: the 800M-point case.  40 facade walls sampled as vertical
  scanlines plus a 400x400 m sinusoid heightfield sampled in row scanlines.
  Generation order is scanline order, which is the "original" order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

POINT_BYTES = 16

# MurmurHash3 fmix64 constants, as signed int64 for torch arithmetic.
_C1 = 0xFF51AFD7ED558CCD - (1 << 64)
_C2 = 0xC4CEB9FE1A85EC53 - (1 << 64)
_GOLD = 0x9E3779B97F4A7C15 - (1 << 64)


def _lsr(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _fmix64(x: torch.Tensor) -> torch.Tensor:
    x = x ^ _lsr(x, 33)
    x = x * _C1
    x = x ^ _lsr(x, 33)
    x = x * _C2
    return x ^ _lsr(x, 33)


def _seed_word(seed: int, stream: int) -> int:
    v = (seed * 0x100000001B3 + stream * 0x2545F4914F6CDD1D + 0x632BE59BD9B4E019) & ((1 << 64) - 1)
    return v - (1 << 64) if v >= (1 << 63) else v


def hash_u24(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """24 uniform random bits per index, as int64."""
    x = idx * _GOLD + _seed_word(seed, stream)
    return _lsr(_fmix64(x), 40)


def uniform(seed: int, stream: int, idx: torch.Tensor, lo: float = 0.0, hi: float = 1.0) -> torch.Tensor:
    """float64 uniform in [lo, hi) with 24-bit resolution."""
    u = hash_u24(seed, stream, idx).to(torch.float64) * (1.0 / (1 << 24))
    return lo + (hi - lo) * u


def _pack(x, y, z, r, g, b, a=255) -> torch.Tensor:
    """Pack float64 coordinates and integer colour channels into 16-byte records."""
    n = x.shape[0]
    out = torch.empty((n, 4), dtype=torch.int32, device=x.device)
    out[:, 0] = x.to(torch.float32).view(torch.int32)
    out[:, 1] = y.to(torch.float32).view(torch.int32)
    out[:, 2] = z.to(torch.float32).view(torch.int32)
    rgba = (r.to(torch.int64) & 255) | ((g.to(torch.int64) & 255) << 8) | ((b.to(torch.int64) & 255) << 16)
    if isinstance(a, torch.Tensor):
        rgba = rgba | ((a.to(torch.int64) & 255) << 24)
    else:
        rgba = rgba | ((a & 255) << 24)
    rgba = torch.where(rgba >= (1 << 31), rgba - (1 << 32), rgba)
    out[:, 3] = rgba.to(torch.int32)
    return out


def _hsv_to_rgb(h, s, v):
    """HSV in [0,1) to byte channels (float64 tensors in, int64 out)."""
    i = torch.floor(h * 6.0)
    f = h * 6.0 - i
    p = v * (1 - s)
    q = v * (1 - s * f)
    t = v * (1 - s * (1 - f))
    i = i.to(torch.int64) % 6
    r = torch.stack([v, q, p, p, t, v], 0).gather(0, i[None])[0]
    g = torch.stack([t, v, v, q, p, p], 0).gather(0, i[None])[0]
    b = torch.stack([p, p, t, v, v, q], 0).gather(0, i[None])[0]
    to8 = lambda c: torch.clamp(torch.floor(c * 255.0 + 0.5), 0, 255).to(torch.int64)
    return to8(r), to8(g), to8(b)


# ---------------------------------------------------------------------------
# Recipes
# ---------------------------------------------------------------------------

def random_cloud(n: int, seed: int = 0, device="cpu", lo=-1.0, hi=1.0) -> torch.Tensor:
    """Uniform points in a cube with uniform colour bytes (small test clouds)."""
    idx = torch.arange(n, dtype=torch.int64, device=device)
    x = uniform(seed, 1, idx, lo, hi)
    y = uniform(seed, 2, idx, lo, hi)
    z = uniform(seed, 3, idx, lo, hi)
    c = hash_u24(seed, 4, idx)
    return _pack(x, y, z, c & 255, (c >> 8) & 255, (c >> 16) & 255)


def sphere_plane(n: int = 1_000_000, seed: int = 0, device="cpu") -> torch.Tensor:
    """Unit-sphere surface for the first half, plane z=-1 over [-2,2]^2 for the rest."""
    idx = torch.arange(n, dtype=torch.int64, device=device)
    half = n // 2
    zs = uniform(seed, 1, idx, -1.0, 1.0)
    phi = uniform(seed, 2, idx, 0.0, 2.0 * math.pi)
    r = torch.sqrt(torch.clamp(1.0 - zs * zs, min=0.0))
    px = uniform(seed, 3, idx, -2.0, 2.0)
    py = uniform(seed, 4, idx, -2.0, 2.0)
    on_sphere = idx < half
    x = torch.where(on_sphere, r * torch.cos(phi), px)
    y = torch.where(on_sphere, r * torch.sin(phi), py)
    z = torch.where(on_sphere, zs, torch.full_like(zs, -1.0))
    c = hash_u24(seed, 5, idx)
    return _pack(x, y, z, c & 255, (c >> 8) & 255, (c >> 16) & 255)


@dataclass
class BoxesLayout:
    centres: np.ndarray   # (B, 2)
    sides: np.ndarray     # (B, 3)
    hues: np.ndarray      # (B,)


def boxes_layout(seed: int = 0, nboxes: int = 200) -> BoxesLayout:
    rng = np.random.default_rng(seed + 7919)
    return BoxesLayout(centres=rng.uniform(-50.0, 50.0, size=(nboxes, 2)),
                       sides=rng.uniform(0.1, 5.0, size=(nboxes, 3)),
                       hues=rng.uniform(0.0, 1.0, size=nboxes))


def _box_faces(layout: BoxesLayout):
    """Faces as (origin, u, v, rgb, area); five per box (no bottom) plus the ground."""
    faces = []
    for (cx, cy), (sx, sy, sz), hue in zip(layout.centres, layout.sides, layout.hues):
        x0, y0 = cx - sx / 2, cy - sy / 2
        rgb = _hsv_scalar(hue, 0.8, 0.9)
        faces.append(((x0, y0, sz), (sx, 0, 0), (0, sy, 0), rgb))          # top
        faces.append(((x0, y0, 0), (sx, 0, 0), (0, 0, sz), rgb))           # y-min side
        faces.append(((x0, y0 + sy, 0), (sx, 0, 0), (0, 0, sz), rgb))      # y-max side
        faces.append(((x0, y0, 0), (0, sy, 0), (0, 0, sz), rgb))           # x-min side
        faces.append(((x0 + sx, y0, 0), (0, sy, 0), (0, 0, sz), rgb))      # x-max side
    faces.append(((-50.0, -50.0, 0.0), (100.0, 0, 0), (0, 100.0, 0), (128, 128, 128)))  # ground
    origin = np.array([f[0] for f in faces], dtype=np.float64)
    u = np.array([f[1] for f in faces], dtype=np.float64)
    v = np.array([f[2] for f in faces], dtype=np.float64)
    rgb = np.array([f[3] for f in faces], dtype=np.int64)
    area = np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1)
    return origin, u, v, rgb, area


def _hsv_scalar(h, s, v):
    r, g, b = _hsv_to_rgb(torch.tensor([h], dtype=torch.float64), torch.tensor([s], dtype=torch.float64),
                          torch.tensor([v], dtype=torch.float64))
    return (int(r[0]), int(g[0]), int(b[0]))


def _counts_by_area(n: int, area: np.ndarray) -> np.ndarray:
    counts = np.floor(area / area.sum() * n).astype(np.int64)
    counts[-1] += n - counts.sum()
    return counts


def boxes(n: int = 50_000_000, seed: int = 0, device="cpu", chunk: int = 1 << 25) -> torch.Tensor:
    """Points on 200 boxes over a ground plane; face by face in generation order."""
    layout = boxes_layout(seed)
    origin, u, v, rgb, area = _box_faces(layout)
    counts = _counts_by_area(n, area)
    starts = np.concatenate([[0], np.cumsum(counts)])
    t_origin = torch.tensor(origin, device=device)
    t_u = torch.tensor(u, device=device)
    t_v = torch.tensor(v, device=device)
    t_rgb = torch.tensor(rgb, device=device)
    t_bounds = torch.tensor(starts[1:], device=device)
    out = torch.empty((n, 4), dtype=torch.int32, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = torch.arange(s, e, dtype=torch.int64, device=device)
        face = torch.searchsorted(t_bounds, idx, right=True)
        a = uniform(seed, 11, idx)[:, None]
        b = uniform(seed, 12, idx)[:, None]
        jit = torch.stack([uniform(seed, 13 + k, idx, -1e-3, 1e-3) for k in range(3)], 1)
        p = t_origin[face] + a * t_u[face] + b * t_v[face] + jit
        c = t_rgb[face]
        out[s:e] = _pack(p[:, 0], p[:, 1], p[:, 2], c[:, 0], c[:, 1], c[:, 2])
    return out


@dataclass
class ScanLayout:
    walls: np.ndarray      # (W, 6): x0, y0, angle, width, height, hue
    wall_counts: np.ndarray
    terrain_rows: int
    terrain_cols: int


def _terrain_height(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Sum of four sinusoids over the 400x400 m terrain (metres)."""
    h = 6.0 * torch.sin(x * 0.011 + 0.3) * torch.cos(y * 0.013 + 1.1)
    h = h + 3.0 * torch.sin(x * 0.031 + 2.0) * torch.cos(y * 0.027 + 0.4)
    h = h + 1.0 * torch.sin(x * 0.093 + 0.7) * torch.cos(y * 0.101 + 2.9)
    h = h + 0.25 * torch.sin(x * 0.37 + 1.9) * torch.cos(y * 0.41 + 0.2)
    return h


def scan_layout(n: int, seed: int = 0, nwalls: int = 40, facade_share: float = 0.6) -> ScanLayout:
    rng = np.random.default_rng(seed + 104729)
    walls = np.zeros((nwalls, 6))
    walls[:, 0] = rng.uniform(-150.0, 150.0, nwalls)
    walls[:, 1] = rng.uniform(-150.0, 150.0, nwalls)
    walls[:, 2] = rng.uniform(0.0, math.pi, nwalls)
    walls[:, 3] = rng.uniform(10.0, 60.0, nwalls)
    walls[:, 4] = rng.uniform(5.0, 30.0, nwalls)
    walls[:, 5] = rng.uniform(0.0, 1.0, nwalls)
    nfac = int(n * facade_share)
    wall_counts = _counts_by_area(nfac, walls[:, 3] * walls[:, 4])
    nter = n - nfac
    cols = max(1, int(math.sqrt(max(nter, 1))))
    rows = (nter + cols - 1) // cols if nter > 0 else 0
    return ScanLayout(walls=walls, wall_counts=wall_counts, terrain_rows=rows, terrain_cols=cols)


def scan(n: int = 800_000_000, seed: int = 0, device="cpu", chunk: int = 1 << 25,
         out: torch.Tensor | None = None, indices: torch.Tensor | None = None) -> torch.Tensor:
    """Facade walls in vertical scanlines, then terrain in row scanlines.

    With ``indices``, only those points of the n-point cloud are made (in
    that order); each point depends on its index alone."""
    lay = scan_layout(n, seed)
    nfac = int(lay.wall_counts.sum())
    total = n if indices is None else int(indices.shape[0])
    if out is None:
        out = torch.empty((total, 4), dtype=torch.int32, device=device)
    wstart = np.concatenate([[0], np.cumsum(lay.wall_counts)])
    # per-wall scanline grid: columns along the wall, rows bottom to top
    wrows = np.maximum(1, np.round(np.sqrt(lay.wall_counts * lay.walls[:, 4] / lay.walls[:, 3]))).astype(np.int64)
    wcols = (lay.wall_counts + wrows - 1) // wrows
    t_wbounds = torch.tensor(wstart[1:], device=device)
    t_wstart = torch.tensor(wstart[:-1], device=device)
    t_walls = torch.tensor(lay.walls, device=device)
    t_wrows = torch.tensor(wrows, device=device)
    t_wcols = torch.tensor(np.maximum(wcols, 1), device=device)
    base_z = _terrain_height(t_walls[:, 0], t_walls[:, 1]) - 1.0
    wr, wg, wb = _hsv_to_rgb(t_walls[:, 5], torch.full_like(t_walls[:, 5], 0.6), torch.full_like(t_walls[:, 5], 0.85))
    for s in range(0, total, chunk):
        e = min(total, s + chunk)
        if indices is None:
            idx = torch.arange(s, e, dtype=torch.int64, device=device)
        else:
            idx = indices[s:e].to(device=device, dtype=torch.int64)
        is_fac = idx < nfac
        # facades
        w = torch.clamp(torch.searchsorted(t_wbounds, idx, right=True), max=len(lay.wall_counts) - 1)
        j = idx - t_wstart[w]
        rows = t_wrows[w]
        col = (j // rows).to(torch.float64)
        row = (j % rows).to(torch.float64)
        fa = (col + 0.5) / t_wcols[w].to(torch.float64)
        fb = (row + 0.5) / rows.to(torch.float64)
        ang = t_walls[w, 2]
        along = fa * t_walls[w, 3]
        jit = [uniform(seed, 21 + k, idx, -1e-3, 1e-3) for k in range(3)]
        fx = t_walls[w, 0] + along * torch.cos(ang) + jit[0]
        fy = t_walls[w, 1] + along * torch.sin(ang) + jit[1]
        fz = base_z[w] + fb * t_walls[w, 4] + jit[2]
        noise = hash_u24(seed, 25, idx) & 31
        fr = torch.clamp(wr[w] + noise - 16, 0, 255)
        fg = torch.clamp(wg[w] + noise - 16, 0, 255)
        fbl = torch.clamp(wb[w] + noise - 16, 0, 255)
        # terrain
        k = torch.clamp(idx - nfac, min=0)
        trow = (k // lay.terrain_cols).to(torch.float64)
        tcol = (k % lay.terrain_cols).to(torch.float64)
        tx = -200.0 + (tcol + 0.5) * (400.0 / lay.terrain_cols) + jit[0]
        ty = -200.0 + (trow + 0.5) * (400.0 / max(lay.terrain_rows, 1)) + jit[1]
        tz = _terrain_height(tx, ty)
        hn = torch.clamp((tz + 10.0) / 20.0, 0.0, 1.0)
        tr = (60 + 140 * hn).to(torch.int64) + (noise >> 1)
        tg = (110 + 60 * hn).to(torch.int64) + (noise >> 1)
        tb = (40 + 120 * hn * hn).to(torch.int64) + (noise >> 1)
        x = torch.where(is_fac, fx, tx)
        y = torch.where(is_fac, fy, ty)
        z = torch.where(is_fac, fz, tz)
        r = torch.where(is_fac, fr, tr)
        g = torch.where(is_fac, fg, tg)
        b = torch.where(is_fac, fbl, tb)
        out[s:e] = _pack(x, y, z, r, g, b)
    return out


# ---------------------------------------------------------------------------
# Cameras: standard look-at and OpenGL perspective, built in float64 and
# rounded to float32 once.  Row-major; clip = M @ (x, y, z, 1).
# ---------------------------------------------------------------------------

def look_at(eye, target, up) -> np.ndarray:
    eye, target, up = (np.asarray(a, dtype=np.float64) for a in (eye, target, up))
    f = target - eye
    f = f / np.linalg.norm(f)
    s = np.cross(f, up)
    s = s / np.linalg.norm(s)
    u = np.cross(s, f)
    v = np.eye(4)
    v[0, :3], v[1, :3], v[2, :3] = s, u, -f
    v[0, 3], v[1, 3], v[2, 3] = -s @ eye, -u @ eye, f @ eye
    return v


def perspective(fovy_deg: float, aspect: float, near: float = 0.1, far: float = 1e4) -> np.ndarray:
    t = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    p = np.zeros((4, 4))
    p[0, 0] = t / aspect
    p[1, 1] = t
    p[2, 2] = (far + near) / (near - far)
    p[2, 3] = 2.0 * far * near / (near - far)
    p[3, 2] = -1.0
    return p


def camera(eye, target, up, width: int, height: int, fovy_deg: float = 60.0) -> np.ndarray:
    """Row-major float32 4x4 view-projection matrix."""
    m = perspective(fovy_deg, width / height) @ look_at(eye, target, up)
    return m.astype(np.float32)


@dataclass
class View:
    name: str
    matrix: np.ndarray
    width: int
    height: int


def sphere_plane_views() -> list[View]:
    return [View("front", camera((0, 0, 4), (0, 0, 0), (0, 1, 0), 640, 480), 640, 480)]


def boxes_views(seed: int = 0) -> list[View]:
    lay = boxes_layout(seed)
    k = int(np.argmax(np.prod(lay.sides, axis=1)))
    cx, cy = lay.centres[k]
    cz = lay.sides[k, 2] / 2
    W, H = 1920, 1080
    return [
        View("overview", camera((0, -120, 90), (0, 0, 0), (0, 0, 1), W, H), W, H),
        View("mid", camera((25, -35, 12), (0, 0, 2), (0, 0, 1), W, H), W, H),
        View("inside", camera((cx, cy, cz), (cx + 1.0, cy, cz), (0, 0, 1), W, H), W, H),
    ]


def scan_views(n: int = 800_000_000, seed: int = 0) -> list[View]:
    lay = scan_layout(n, seed)
    x0, y0, ang, width, height, _ = lay.walls[0]
    mid = np.array([x0 + 0.5 * width * math.cos(ang), y0 + 0.5 * width * math.sin(ang)])
    normal = np.array([-math.sin(ang), math.cos(ang)])
    base = float(_terrain_height(torch.tensor([x0], dtype=torch.float64),
                                 torch.tensor([y0], dtype=torch.float64))[0])
    eye = np.array([*(mid + 15.0 * normal), base + height * 0.5])
    tgt = np.array([*mid, base + height * 0.5])
    W, H = 1920, 1080
    return [
        View("overview", camera((0, -450, 300), (0, 0, 0), (0, 0, 1), W, H), W, H),
        View("closeup", camera(tuple(eye), tuple(tgt), (0, 0, 1), W, H), W, H),
        View("empty", camera((0, -600, 50), (0, -1000, 50), (0, 0, 1), W, H), W, H),
    ]


def as_numpy_points(cloud: torch.Tensor) -> np.ndarray:
    """Contiguous (n, 4) int32 host copy of a cloud (bytes unchanged)."""
    return np.ascontiguousarray(cloud.cpu().numpy())


# ---------------------------------------------------------------------------
# Batched workload: 8 clouds of uneven size (the boxes recipe, seeds 0..7),
# 8 views each at 256^2 .. 2048^2, cameras on an orbit around the scene.
# ---------------------------------------------------------------------------

BATCH_CLOUD_SIZES = (1_000_000, 2_000_000, 5_000_000, 10_000_000, 20_000_000, 50_000_000, 100_000_000,
                     200_000_000)
BATCH_VIEW_SIZES = (256, 512, 768, 1024, 1280, 1536, 1792, 2048)


def batch_views(num_clouds: int = 8, sizes=BATCH_VIEW_SIZES) -> list[tuple[int, View]]:
    """(cloud index, view) pairs: each cloud seen from len(sizes) orbit
    cameras, one per square resolution, the orbit phase shifted per cloud."""
    out = []
    for c in range(num_clouds):
        for k, size in enumerate(sizes):
            a = 2.0 * math.pi * (k + 0.37 * c) / len(sizes)
            eye = (80.0 * math.cos(a), 80.0 * math.sin(a), 40.0 + 5.0 * (k % 3))
            out.append((c, View(f"cloud{c}/orbit{k}", camera(eye, (0, 0, 0), (0, 0, 1), size, size), size, size)))
    return out


# ---------------------------------------------------------------------------
# Served workload: 16 clouds (boxes recipe, 1M..300M points, log-spaced) and a
# Poisson stream of view requests over them.
# ---------------------------------------------------------------------------

SERVE_CLOUD_SIZES = tuple(int(round(1e6 * 300.0 ** (i / 15))) for i in range(16))
SERVE_RESOLUTIONS = ((512, 512), (1280, 720), (1920, 1080), (2560, 1440), (3840, 2160))


def serve_requests(count: int, rate_per_s: float = 2000.0, seed: int = 0, num_clouds: int = 16):
    """(arrival seconds, cloud, matrix, width, height, flags) tuples: Poisson
    arrivals at the given mean rate, a uniform cloud, a uniform resolution,
    basic or HQ with equal odds (flags 1 or 2), a random orbit camera."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
    out = []
    for i in range(count):
        c = int(rng.integers(0, num_clouds))
        W, H = SERVE_RESOLUTIONS[int(rng.integers(0, len(SERVE_RESOLUTIONS)))]
        flags = 1 if rng.random() < 0.5 else 2
        a = rng.uniform(0.0, 2.0 * math.pi)
        eye = (80.0 * math.cos(a), 80.0 * math.sin(a), 35.0 + 15.0 * rng.random())
        out.append((float(t[i]), c, camera(eye, (0, 0, 0), (0, 0, 1), W, H), W, H, flags))
    return out
