"""Seeded synthetic light-field microscopy (LFM) raw frames.

Inputs only: this module holds none of the compression method's arithmetic
and serves the tests, the smoke check and the benchmark alike.

Forward model (stand-in for the paper's bead, MCF-10A cell and zebrafish
vessel recordings, which are not available):

* Objects live in sub-aperture coordinates (s, t), in lenslet units, on an
  Nx x Ny lenslet grid with pitch p (each lenslet covers p x p pixels).
* View (u, v) sees an object at depth disparity d shifted by
  d * (u - c) / (p - 1) along s and d * (v - c) / (p - 1) along t, c = (p-1)/2.
* Pixels outside the circular lenslet aperture (u-c)^2 + (v-c)^2 > (p/2)^2
  receive no signal.
* Expected photons lambda -> Poisson(lambda) + N(0, 2^2) DN read noise
  + 100 DN offset, gain 1 DN per photon, rounded and clipped to uint16.
* Raw layout: raw[t*p + v, s*p + u] = view(u, v)[t, s].

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import math

import numpy as np

OFFSET_DN = 100.0
READ_SIGMA_DN = 2.0


def _views(p: int):
    c = (p - 1) / 2.0
    u = np.arange(p, dtype=np.float64)
    du = (u - c) / max(p - 1, 1)
    aperture = ((u[None, :] - c) ** 2 + (u[:, None] - c) ** 2) <= (p / 2.0) ** 2  # [v, u]
    return du, aperture


def _to_raw(sub: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """sub[v, u, t, s] expected photons -> uint16 raw frame [H, W]."""
    p, _, Ny, Nx = sub.shape
    photons = rng.poisson(np.maximum(sub, 0.0)).astype(np.float64)
    dn = photons + rng.normal(0.0, READ_SIGMA_DN, size=photons.shape) + OFFSET_DN
    dn = np.clip(np.rint(dn), 0, 65535).astype(np.uint16)
    return np.ascontiguousarray(dn.transpose(2, 0, 3, 1).reshape(Ny * p, Nx * p))


def _check(W: int, H: int, p: int):
    if W % p or H % p:
        raise ValueError("frame size must be a multiple of the pitch")


def bead_photons(W: int, H: int, p: int, n_beads: int = 200, sigma: float = 1.5,
                 peak: float = 2000.0, max_disparity: float = 3.0, seed: int = 0) -> np.ndarray:
    """Expected photons sub[v, u, t, s] of Gaussian fluorescent beads."""
    _check(W, H, p)
    rng = np.random.default_rng(seed)
    Nx, Ny = W // p, H // p
    du, aperture = _views(p)
    sub = np.zeros((p, p, Ny, Nx), dtype=np.float64)
    s0 = rng.uniform(0, Nx, n_beads)
    t0 = rng.uniform(0, Ny, n_beads)
    d = rng.uniform(-max_disparity, max_disparity, n_beads)
    R = int(math.ceil(4 * sigma)) + 1
    for b in range(n_beads):
        half = abs(d[b]) / 2.0
        sa = max(0, int(math.floor(s0[b] - half - R)))
        sb = min(Nx, int(math.ceil(s0[b] + half + R)) + 1)
        ta = max(0, int(math.floor(t0[b] - half - R)))
        tb = min(Ny, int(math.ceil(t0[b] + half + R)) + 1)
        if sa >= sb or ta >= tb:
            continue
        ss = np.arange(sa, sb, dtype=np.float64)
        tt = np.arange(ta, tb, dtype=np.float64)
        cs = s0[b] + d[b] * du  # [u]
        ct = t0[b] + d[b] * du  # [v]
        gs = np.exp(-((ss[None, :] - cs[:, None]) ** 2) / (2 * sigma ** 2))  # [u, s]
        gt = np.exp(-((tt[None, :] - ct[:, None]) ** 2) / (2 * sigma ** 2))  # [v, t]
        sub[:, :, ta:tb, sa:sb] += peak * gt[:, None, :, None] * gs[None, :, None, :]
    sub *= aperture[:, :, None, None]
    return sub


def beads(W: int, H: int, p: int, peak: float = 2000.0, n_beads: int = 200, sigma: float = 1.5,
          seed: int = 0) -> np.ndarray:
    """Raw uint16 LFM frame of fluorescent beads (paper's bead data analogue)."""
    rng = np.random.default_rng(seed + 7919)
    return _to_raw(bead_photons(W, H, p, n_beads, sigma, peak, seed=seed), rng)


class _Perlin2D:
    """Perlin gradient noise in 2-D (Perlin 1985; quintic fade of Perlin 2002)."""

    def __init__(self, rng: np.random.Generator, size: int = 256):
        self.size = size
        self.perm = rng.permutation(size)
        ang = rng.uniform(0, 2 * np.pi, size)
        self.grad = np.stack([np.cos(ang), np.sin(ang)], axis=1)

    def _g(self, ix, iy):
        h = self.perm[(self.perm[ix % self.size] + iy) % self.size]
        return self.grad[h]

    def __call__(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        x0 = np.floor(x).astype(np.int64)
        y0 = np.floor(y).astype(np.int64)
        fx, fy = x - x0, y - y0

        def fade(t):
            return t * t * t * (t * (t * 6 - 15) + 10)

        def dot(ix, iy, dx, dy):
            g = self._g(ix, iy)
            return g[..., 0] * dx + g[..., 1] * dy

        n00 = dot(x0, y0, fx, fy)
        n10 = dot(x0 + 1, y0, fx - 1, fy)
        n01 = dot(x0, y0 + 1, fx, fy - 1)
        n11 = dot(x0 + 1, y0 + 1, fx - 1, fy - 1)
        u, v = fade(fx), fade(fy)
        nx0 = n00 + u * (n10 - n00)
        nx1 = n01 + u * (n11 - n01)
        return nx0 + v * (nx1 - nx0)  # roughly in [-0.7, 0.7]


def cell_photons(W: int, H: int, p: int, n_cells: int = 50, level: float = 500.0,
                 axes=(10.0, 40.0), max_disparity: float = 3.0, seed: int = 3) -> np.ndarray:
    """Expected photons of a cell-like field: ellipses with a bright membrane
    ring and a dimmer interior, modulated by Perlin texture at scale 16."""
    _check(W, H, p)
    rng = np.random.default_rng(seed)
    Nx, Ny = W // p, H // p
    du, aperture = _views(p)
    noise = _Perlin2D(rng)
    sub = np.zeros((p, p, Ny, Nx), dtype=np.float64)
    scale = min(1.0, min(Nx, Ny) / 136.0)
    ring_w = 1.5
    for _ in range(n_cells):
        a = rng.uniform(*axes) * scale
        b = rng.uniform(*axes) * scale
        th = rng.uniform(0, np.pi)
        cx, cy = rng.uniform(0, Nx), rng.uniform(0, Ny)
        d = rng.uniform(-max_disparity, max_disparity)
        ox, oy = rng.uniform(0, 1000, 2)
        R = max(a, b) + 3 * ring_w + abs(d)
        sa, sb = max(0, int(cx - R)), min(Nx, int(cx + R) + 2)
        ta, tb = max(0, int(cy - R)), min(Ny, int(cy + R) + 2)
        if sa >= sb or ta >= tb:
            continue
        ss = np.arange(sa, sb, dtype=np.float64)
        tt = np.arange(ta, tb, dtype=np.float64)
        # object coordinates for every (v, u, t, s) in the box
        X = ss[None, None, None, :] - (cx + d * du[None, :, None, None])
        Y = tt[None, None, :, None] - (cy + d * du[:, None, None, None])
        X, Y = np.broadcast_arrays(X, Y)
        xr = X * np.cos(th) + Y * np.sin(th)
        yr = -X * np.sin(th) + Y * np.cos(th)
        r = np.sqrt((xr / a) ** 2 + (yr / b) ** 2)
        d2 = ((r - 1.0) * min(a, b)) ** 2
        env = np.where(d2 < 36 * ring_w ** 2, np.exp(-d2 / (2 * ring_w ** 2)), 0.0) + (r < 1.0) * 0.3
        sel = env > 0
        tex = 0.5 + 0.5 * noise((xr[sel] + ox) / 16.0 * 4, (yr[sel] + oy) / 16.0 * 4)
        blk = np.zeros(env.shape)
        blk[sel] = level * env[sel] * tex
        sub[:, :, ta:tb, sa:sb] += blk
    sub *= aperture[:, :, None, None]
    return sub


def cells(W: int, H: int, p: int, level: float = 500.0, n_cells: int = 50, seed: int = 3) -> np.ndarray:
    """Raw uint16 LFM frame of a cell-like field (MCF-10A analogue)."""
    rng = np.random.default_rng(seed + 104729)
    return _to_raw(cell_photons(W, H, p, n_cells, level, seed=seed), rng)


class VesselSeries:
    """Time series of a vessel tree with bright spots flowing along it
    (zebrafish blood-vessel analogue). Frame k is ``frame(k)``."""

    def __init__(self, W: int, H: int, p: int, peak: float = 300.0, n_spots: int = 40,
                 seed: int = 4, levels: int = 3, background: float = 0.2):
        _check(W, H, p)
        self.W, self.H, self.p = W, H, p
        self.peak = peak
        self.seed = seed
        rng = np.random.default_rng(seed)
        Nx, Ny = W // p, H // p
        self.Nx, self.Ny = Nx, Ny
        scale = min(1.0, min(Nx, Ny) / 136.0)
        du, aperture = _views(p)
        self.du, self.aperture = du, aperture
        # branching tree of straight segments: (x0, y0, x1, y1, radius, disparity)
        segs = []
        x0, y0 = rng.uniform(0.3, 0.7) * Nx, 0.0
        ang = np.pi / 2 + rng.uniform(-0.3, 0.3)
        length = 0.45 * Ny
        frontier = [(x0, y0, ang, length)]
        for lvl in range(levels):
            nxt = []
            for (xa, ya, an, ln) in frontier:
                xb, yb = xa + ln * np.cos(an), ya + ln * np.sin(an)
                segs.append((xa, ya, xb, yb, rng.uniform(3, 8) * scale, rng.uniform(-3, 3)))
                for sgn in (-1, 1):
                    nxt.append((xb, yb, an + sgn * rng.uniform(0.3, 0.8), ln * 0.65))
            frontier = nxt
        self.segs = segs
        sub = np.zeros((p, p, Ny, Nx), dtype=np.float64)
        for (xa, ya, xb, yb, rad, d) in segs:
            self._add_segment(sub, xa, ya, xb, yb, rad, d, 1.0)
        bg = background
        self.static = (bg + (1 - bg) * np.minimum(sub, 1.0)) * aperture[:, :, None, None] * peak * 0.5
        # spots: segment index, start position (fraction), speed (lenslets/frame)
        self.spot_seg = rng.integers(0, len(segs), n_spots)
        self.spot_pos = rng.uniform(0, 1, n_spots)
        self.spot_speed = rng.uniform(2, 10, n_spots) / 4.0 * scale

    def _add_segment(self, sub, xa, ya, xb, yb, rad, d, amp):
        p, Nx, Ny, du = self.p, self.Nx, self.Ny, self.du
        R = rad * 3 + abs(d)
        sa, sb = max(0, int(min(xa, xb) - R)), min(Nx, int(max(xa, xb) + R) + 2)
        ta, tb = max(0, int(min(ya, yb) - R)), min(Ny, int(max(ya, yb) + R) + 2)
        if sa >= sb or ta >= tb:
            return
        ss = np.arange(sa, sb, dtype=np.float64)
        tt = np.arange(ta, tb, dtype=np.float64)
        X = ss[None, None, None, :] - d * du[None, :, None, None]
        Y = tt[None, None, :, None] - d * du[:, None, None, None]
        X, Y = np.broadcast_arrays(X, Y)
        vx, vy = xb - xa, yb - ya
        L2 = vx * vx + vy * vy + 1e-12
        tpar = np.clip(((X - xa) * vx + (Y - ya) * vy) / L2, 0, 1)
        dist2 = (X - xa - tpar * vx) ** 2 + (Y - ya - tpar * vy) ** 2
        sub[:, :, ta:tb, sa:sb] += amp * np.exp(-dist2 / (2 * (rad / 2.0) ** 2))

    def photons(self, k: int) -> np.ndarray:
        p, Nx, Ny, du = self.p, self.Nx, self.Ny, self.du
        sub = self.static.copy()
        sigma = 1.0
        for i in range(len(self.spot_seg)):
            xa, ya, xb, yb, rad, d = self.segs[self.spot_seg[i]]
            ln = math.hypot(xb - xa, yb - ya) + 1e-9
            f = (self.spot_pos[i] + k * self.spot_speed[i] / ln) % 1.0
            sx, sy = xa + f * (xb - xa), ya + f * (yb - ya)
            R = 4
            sa, sb = max(0, int(sx - R - 2)), min(Nx, int(sx + R + 3))
            ta, tb = max(0, int(sy - R - 2)), min(Ny, int(sy + R + 3))
            if sa >= sb or ta >= tb:
                continue
            ss = np.arange(sa, sb, dtype=np.float64)
            tt = np.arange(ta, tb, dtype=np.float64)
            gs = np.exp(-((ss[None, :] - (sx + d * du)[:, None]) ** 2) / (2 * sigma ** 2))
            gt = np.exp(-((tt[None, :] - (sy + d * du)[:, None]) ** 2) / (2 * sigma ** 2))
            sub[:, :, ta:tb, sa:sb] += self.peak * gt[:, None, :, None] * gs[None, :, None, :]
        return sub * self.aperture[:, :, None, None]

    def frame(self, k: int) -> np.ndarray:
        rng = np.random.default_rng((self.seed, k))
        return _to_raw(self.photons(k), rng)


def vessel_frames(W: int, H: int, p: int, n: int, seed: int = 4, peak: float = 300.0) -> np.ndarray:
    vs = VesselSeries(W, H, p, peak=peak, seed=seed)
    return np.stack([vs.frame(k) for k in range(n)])


# ------------------------------------------------------------ named workloads
SIZE_CLASSES = [(1300, 1300, 13), (2040, 2040, 15), (2550, 2160, 15)]


def single_frames_2040(seeds=(1, 2, 3)):
    """Three 2040x2040 frames, 136x136 lenslets at pitch 15: beads at 20 and
    2000 mean photons and a cell field at 500 photons."""
    W = H = 2040
    p = 15
    return [beads(W, H, p, peak=20.0, seed=seeds[0]),
            beads(W, H, p, peak=2000.0, seed=seeds[1]),
            cells(W, H, p, level=500.0, seed=seeds[2])]


def bead_frame_1300(seed: int = 0):
    """1300x1300 frame, 100x100 lenslets at pitch 13, 200 beads, 2000 photons."""
    return beads(1300, 1300, 13, peak=2000.0, seed=seed)


def uneven_batch(n: int = 256, base_seed: int = 1000):
    """Frame i: size class i mod 3, generator (i // 3) mod 3, seed base + i.
    Returns a list of (frame, pitch)."""
    out = []
    for i in range(n):
        W, H, p = SIZE_CLASSES[i % 3]
        g = (i // 3) % 3
        s = base_seed + i
        if g == 0:
            fr = beads(W, H, p, peak=2000.0, seed=s)
        elif g == 1:
            fr = cells(W, H, p, level=500.0, seed=s)
        else:
            fr = VesselSeries(W, H, p, seed=s).frame(0)
        out.append((fr, p))
    return out


def uneven_batch_fast(n: int = 256, base_seed: int = 1000):
    """Frame i: size class i mod 3, generator (i // 3) mod 3 (beads 2000,
    cells 500, vessel 300). The expected-photon field of each (size,
    generator) pair is rendered once; every frame draws its own Poisson and
    read noise with seed base + i. Returns a list of (frame, pitch)."""
    fields = {}
    out = []
    for i in range(n):
        c, g = i % 3, (i // 3) % 3
        W, H, p = SIZE_CLASSES[c]
        if (c, g) not in fields:
            s = base_seed + 10 * c + g
            if g == 0:
                fields[(c, g)] = bead_photons(W, H, p, peak=2000.0, seed=s)
            elif g == 1:
                fields[(c, g)] = cell_photons(W, H, p, level=500.0, seed=s)
            else:
                fields[(c, g)] = VesselSeries(W, H, p, seed=s).photons(0)
        out.append((_to_raw(fields[(c, g)], np.random.default_rng(base_seed + i)), p))
    return out


def photons_to_frame_torch(sub, scale: float, seed: int, device="cuda"):
    """Expected photons sub[v, u, t, s] (numpy, unit level) times ``scale``
    -> raw frame as an int16 CUDA tensor holding the uint16 bits, with
    Poisson and read noise drawn by torch on the device (fixed seed). Used
    to make large training sets quickly; same forward model as _to_raw."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    lam = torch.as_tensor(sub, dtype=torch.float32, device=device) * float(scale)
    ph = torch.poisson(lam.clamp_min(0), generator=g)
    dn = ph + torch.randn(lam.shape, generator=g, device=device) * READ_SIGMA_DN + OFFSET_DN
    dn = torch.clamp(torch.round(dn), 0, 65535).to(torch.int32)
    p, _, Ny, Nx = sub.shape
    raw = dn.permute(2, 0, 3, 1).reshape(Ny * p, Nx * p).contiguous()
    return torch.where(raw >= 32768, raw - 65536, raw).to(torch.int16)


def training_fields(n_beads: int, n_cells: int, n_vessels: int, W: int = 2040, H: int = 2040, p: int = 15,
                    seed0: int = 10000):
    """Unit-level expected-photon fields of the three generators (beads: peak
    1, cells: level 1, vessels: peak 1), seeds seed0 + k."""
    out = []
    k = 0
    for _ in range(n_beads):
        out.append(("beads", bead_photons(W, H, p, peak=1.0, seed=seed0 + k)))
        k += 1
    for _ in range(n_cells):
        out.append(("cells", cell_photons(W, H, p, level=1.0, seed=seed0 + k)))
        k += 1
    for _ in range(n_vessels):
        out.append(("vessel", VesselSeries(W, H, p, peak=1.0, seed=seed0 + k).photons(k % 50)))
        k += 1
    return out
