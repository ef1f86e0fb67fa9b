"""Layered synthetic stereo scenes with exact ground truth.

Every scene is a stack of layers.  A layer has a footprint in left-image
coordinates, a disparity surface d_k(x, y) (constant, planar or quadratic)
and its own procedural texture, painted on the surface and parameterised by
the left-image coordinate of the surface point.  The left image shows, at
each pixel, the front-most layer (largest disparity) whose footprint covers
it.  The right image at (x_r, y) is rendered by solving x - d_k(x, y) = x_r
for every layer (closed form for all three surface kinds), keeping the
front-most layer whose footprint contains the solution and sampling that
layer's texture there.  Ground truth and occlusion masks come out of the same
pass.  Noise is added as round(I + N(0, sigma^2)) clamped to [0, 255].

The Middlebury 2001/2003 scenes the method was evaluated on are not used;
these scenes stand in for them with the sizes, disparity ranges and
parameters of each workload.  All randomness comes from numpy's PCG64
generator seeded by the caller, so a (workload, seed) pair is reproducible.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy import ndimage

# ----------------------------------------------------------------------------
# Workload table.  Keys name the workload by what it is; values are the
# stereo parameters (radius = aggregation radius rho, sigma_s = gamma_d,
# sigma_r = gamma_r, tau = truncation of the TAD cost mode).
# ----------------------------------------------------------------------------
WORKLOADS = {
    # 160x120 grey, uniform random texture, rectangles of constant disparity.
    "gray160x120_d16_r4": dict(H=120, W=160, C=1, D=16, radius=4, sigma_s=4.0,
                               sigma_r=10.0, tau=20.0, texture="uniform",
                               surfaces="rect_const", noise=2.0,
                               layers=(3, 5), drange=(0, 15)),
    # 640x480 RGB, fractal value noise, slanted planes with occlusion bands.
    "rgb640x480_d64_r7": dict(H=480, W=640, C=3, D=64, radius=7, sigma_s=7.0,
                              sigma_r=12.0, tau=30.0, texture="fractal5",
                              surfaces="planes", noise=2.0,
                              layers=(3, 6), drange=(0, 63)),
    # 1280x960 RGB, multi-octave texture, planes plus quadratic surfaces.
    "rgb1280x960_d128_r15": dict(H=960, W=1280, C=3, D=128, radius=15,
                                 sigma_s=15.0, sigma_r=12.0, tau=30.0,
                                 texture="fractal6", surfaces="planes_quad",
                                 noise=3.0, layers=(3, 6), drange=(0, 127)),
    # 1920x1080 RGB for the band-restricted path.
    "rgb1920x1080_d256_r9": dict(H=1080, W=1920, C=3, D=256, radius=9,
                                 sigma_s=9.0, sigma_r=12.0, tau=30.0,
                                 texture="fractal5", surfaces="planes_quad",
                                 noise=2.0, layers=(3, 6), drange=(0, 255)),
}


@dataclass
class Pair:
    """One synthetic stereo pair plus the parameters it should be matched with."""

    left: np.ndarray          # (H, W, C) uint8, row-major HWC
    right: np.ndarray         # (H, W, C) uint8
    gt: np.ndarray            # (H, W) float64 left-view disparity
    occ: np.ndarray           # (H, W) bool, True where the left pixel is hidden in the right view
    H: int
    W: int
    C: int
    D: int
    radius: int
    sigma_s: float
    sigma_r: float
    tau: float
    name: str = ""
    seed: int = 0
    meta: dict = field(default_factory=dict)

    def params(self):
        return dict(H=self.H, W=self.W, C=self.C, D=self.D, radius=self.radius,
                    sigma_s=self.sigma_s, sigma_r=self.sigma_r, tau=self.tau)


# ----------------------------------------------------------------------------
# Textures
# ----------------------------------------------------------------------------
class _Texture:
    """Value-noise texture over a bounded rectangle of left coordinates.

    ``kind`` is "uniform" (an independent uniform value per integer
    coordinate, looked up by nearest neighbour) or "fractalN" (N octaves of
    bilinear value noise, finest cell 2 px, amplitude halving per octave).
    """

    def __init__(self, rng, kind, C, xlo, xhi, ylo, yhi):
        self.kind = kind
        self.C = C
        self.xlo, self.ylo = xlo - 4, ylo - 4
        nx = int(np.ceil(xhi - xlo)) + 12
        ny = int(np.ceil(yhi - ylo)) + 12
        if kind == "uniform":
            self.grids = [[rng.random((ny, nx)) for _ in range(C)]]
            self.cells = [1.0]
            self.amps = [1.0]
        else:
            octaves = int(kind[len("fractal"):])
            self.cells, self.amps, self.grids = [], [], []
            for o in range(octaves):
                cell = 2.0 ** (octaves - o)          # coarse to fine, finest 2 px
                gx = int(np.ceil(nx / cell)) + 3
                gy = int(np.ceil(ny / cell)) + 3
                self.cells.append(cell)
                self.amps.append(0.5 ** (octaves - 1 - o) if o else 1.0)
                self.grids.append([rng.random((gy, gx)) for _ in range(C)])
            # gentle weighting: coarse octaves carry more energy
            self.amps = [0.55 ** o for o in range(octaves)]

    def sample(self, x, y):
        """Intensity in [0, 255] (float64) at left coordinates (x, y), shape (n, C)."""
        x = np.asarray(x, np.float64) - self.xlo
        y = np.asarray(y, np.float64) - self.ylo
        out = np.zeros((x.size, self.C))
        if self.kind == "uniform":
            ix = np.rint(x).astype(np.int64)
            iy = np.rint(y).astype(np.int64)
            for c in range(self.C):
                out[:, c] = self.grids[0][c][iy, ix]
            return out * 255.0
        total = sum(self.amps)
        for cell, amp, grids in zip(self.cells, self.amps, self.grids):
            coords = np.stack([y / cell, x / cell])
            for c in range(self.C):
                out[:, c] += amp * ndimage.map_coordinates(grids[c], coords, order=1, mode="nearest")
        out /= total
        # stretch contrast around 0.5 so the full uint8 range is used
        out = np.clip(0.5 + (out - 0.5) * 2.6, 0.0, 1.0)
        return out * 255.0


# ----------------------------------------------------------------------------
# Surfaces
# ----------------------------------------------------------------------------
class _Layer:
    """A textured surface with a footprint in left-image coordinates.

    kind "const": d = c;  "plane": d = a*x + b*y + c;
    "quad": d = c + alpha*(x - x0)^2 + beta*(y - y0)^2.
    Footprint: "all", ("rect", x0, x1, y0, y1) or ("ellipse", cx, cy, rx, ry).
    """

    def __init__(self, kind, params, footprint, texture):
        self.kind = kind
        self.p = params
        self.footprint = footprint
        self.texture = texture

    def disp(self, x, y):
        p = self.p
        if self.kind == "const":
            return np.full(np.broadcast(x, y).shape, float(p["c"]))
        if self.kind == "plane":
            return p["a"] * x + p["b"] * y + p["c"]
        return p["c"] + p["alpha"] * (x - p["x0"]) ** 2 + p["beta"] * (y - p["y0"]) ** 2

    def solve(self, xr, y):
        """Left coordinate x with x - d(x, y) = xr (unique for |slope| < 1)."""
        p = self.p
        if self.kind == "const":
            return xr + p["c"]
        if self.kind == "plane":
            return (xr + p["b"] * y + p["c"]) / (1.0 - p["a"])
        # alpha*t^2 - t + K = 0 with t = x - x0, K = xr - x0 + c + beta*(y-y0)^2
        al = p["alpha"]
        K = xr - p["x0"] + p["c"] + p["beta"] * (y - p["y0"]) ** 2
        if abs(al) < 1e-15:
            t = K
        else:
            disc = np.maximum(1.0 - 4.0 * al * K, 0.0)
            t = 2.0 * K / (1.0 + np.sqrt(disc))      # root continuous at al -> 0
        return p["x0"] + t

    def inside(self, x, y):
        f = self.footprint
        if f == "all":
            return np.ones(np.broadcast(x, y).shape, bool)
        if f[0] == "rect":
            _, x0, x1, y0, y1 = f
            return (x >= x0) & (x < x1) & (y >= y0) & (y < y1)
        _, cx, cy, rx, ry = f
        return ((x - cx) / rx) ** 2 + ((y - cy) / ry) ** 2 <= 1.0


def _select(layers, xs_of_layer, y):
    """Front-most layer index per point.  xs_of_layer[k] is the left coordinate
    of the point on layer k; a layer is a candidate where its footprint covers it."""
    best = np.full(y.shape, -1, np.int64)
    bestd = np.full(y.shape, -np.inf)
    for k, layer in enumerate(layers):
        x = xs_of_layer[k]
        ok = layer.inside(x, y)
        d = layer.disp(x, y)
        better = ok & (d > bestd)
        best[better] = k
        bestd[better] = d[better]
    return best, bestd


def _render(layers, H, W, C, noise, rng):
    yy, xx = np.mgrid[0:H, 0:W]
    x = xx.ravel().astype(np.float64)
    y = yy.ravel().astype(np.float64)
    # left view: every layer is sampled at the pixel itself
    kl, dl = _select(layers, [x] * len(layers), y)
    left = np.zeros((x.size, C))
    for k, layer in enumerate(layers):
        m = kl == k
        if m.any():
            left[m] = layer.texture.sample(x[m], y[m])
    # right view: back-project the right pixel onto every layer
    xs = [layer.solve(x, y) for layer in layers]
    kr, _ = _select(layers, xs, y)
    right = np.zeros((x.size, C))
    for k, layer in enumerate(layers):
        m = kr == k
        if m.any():
            right[m] = layer.texture.sample(xs[k][m], y[m])
    # occlusion: the left point projects to x - d; hidden if outside the right
    # view or if another layer is in front there
    xr = x - dl
    xs2 = [layer.solve(xr, y) for layer in layers]
    k2, _ = _select(layers, xs2, y)
    occ = (xr < -0.5) | (k2 != kl)
    out = []
    for img in (left, right):
        if noise > 0:
            img = img + rng.normal(0.0, noise, img.shape)
        out.append(np.clip(np.rint(img), 0, 255).astype(np.uint8).reshape(H, W, C))
    return out[0], out[1], dl.reshape(H, W), occ.reshape(H, W)


def _plane_params(rng, W, H, lo, hi):
    """Plane d = a x + b y + c whose values over [0,W]x[0,H] stay in [lo, hi]."""
    for _ in range(1000):
        d00, d10, d01 = rng.uniform(lo, hi, 3)
        d11 = d10 + d01 - d00
        if lo <= d11 <= hi:
            return dict(a=(d10 - d00) / W, b=(d01 - d00) / H, c=d00)
    return dict(a=0.0, b=0.0, c=0.5 * (lo + hi))


def _quad_params(rng, W, H, lo, hi):
    """d = c + alpha (x-x0)^2 + beta (y-y0)^2 staying within [lo, hi] over the image
    and with |d/dx| < 0.5 so the right-view solve stays monotone."""
    x0, y0 = rng.uniform(0.2 * W, 0.8 * W), rng.uniform(0.2 * H, 0.8 * H)
    span = hi - lo
    rx2 = max(x0, W - x0) ** 2
    ry2 = max(y0, H - y0) ** 2
    amp = rng.uniform(0.2, 0.45) * span
    sign = rng.choice([-1.0, 1.0])
    alpha = sign * amp / (rx2 + ry2)
    beta = alpha * rng.uniform(0.5, 1.5)
    if abs(2 * alpha * max(x0, W - x0)) > 0.5:
        alpha = np.sign(alpha) * 0.25 / max(x0, W - x0)
    extreme = alpha * rx2 + beta * ry2
    c = lo + (span - extreme if sign < 0 else 0.0) + rng.uniform(0, 0.2) * span
    c = float(np.clip(c, lo - min(0.0, extreme), hi - max(0.0, extreme)))
    return dict(alpha=alpha, beta=beta, x0=x0, y0=y0, c=c)


def make_pair(name: str, seed: int, H=None, W=None, D=None, radius=None, sigma_s=None) -> Pair:
    """Render one pair of workload ``name`` (a key of WORKLOADS).

    H, W, D, radius, sigma_s override the table (used for row bands, batch
    members and small test cases); the scene recipe is unchanged.
    """
    spec = dict(WORKLOADS[name])
    for key, val in (("H", H), ("W", W), ("D", D), ("radius", radius), ("sigma_s", sigma_s)):
        if val is not None:
            spec[key] = val
    if D is not None and radius is not None and sigma_s is None:
        spec["sigma_s"] = float(radius)
    H, W, C, D = spec["H"], spec["W"], spec["C"], spec["D"]
    lo, hi = spec["drange"]
    hi = min(hi, D - 1)
    lo = min(lo, hi)
    rng = np.random.Generator(np.random.PCG64(seed))
    nlayers = int(rng.integers(spec["layers"][0], spec["layers"][1] + 1))
    surfaces = spec["surfaces"]
    layers = []

    def texture():
        return _Texture(rng, spec["texture"], C, -2.0, W + hi + 4.0, -2.0, H + 2.0)

    if surfaces == "rect_const":
        # background: constant integer disparity in the lower part of the range
        dbg = int(rng.integers(lo, lo + max(1, (hi - lo) // 3) + 1))
        layers.append(_Layer("const", dict(c=dbg), "all", texture()))
        for _ in range(nlayers - 1):
            d = int(rng.integers(dbg + 1 if dbg < hi else hi, hi + 1))
            w_ = int(rng.integers(W // 6, W // 2))
            h_ = int(rng.integers(H // 6, H // 2))
            x0 = int(rng.integers(0, W - w_))
            y0 = int(rng.integers(0, H - h_))
            layers.append(_Layer("const", dict(c=d), ("rect", x0, x0 + w_, y0, y0 + h_), texture()))
    else:
        bg_hi = lo + 0.35 * (hi - lo)
        layers.append(_Layer("plane", _plane_params(rng, W, H, lo, bg_hi), "all", texture()))
        for i in range(nlayers - 1):
            f_lo = lo + rng.uniform(0.2, 0.6) * (hi - lo)
            f_hi = min(hi, f_lo + rng.uniform(0.1, 0.4) * (hi - lo))
            use_quad = surfaces == "planes_quad" and (i % 2 == 1)
            if use_quad:
                params, kind = _quad_params(rng, W, H, f_lo, f_hi), "quad"
            else:
                params, kind = _plane_params(rng, W, H, f_lo, f_hi), "plane"
            if rng.random() < 0.5:
                w_ = rng.uniform(0.15, 0.5) * W
                h_ = rng.uniform(0.15, 0.5) * H
                x0 = rng.uniform(0, W - w_)
                y0 = rng.uniform(0, H - h_)
                fp = ("rect", x0, x0 + w_, y0, y0 + h_)
            else:
                fp = ("ellipse", rng.uniform(0.15, 0.85) * W, rng.uniform(0.15, 0.85) * H,
                      rng.uniform(0.08, 0.3) * W, rng.uniform(0.08, 0.3) * H)
            layers.append(_Layer(kind, params, fp, texture()))
    left, right, gt, occ = _render(layers, H, W, C, spec["noise"], rng)
    return Pair(left=left, right=right, gt=gt, occ=occ, H=H, W=W, C=C, D=D,
                radius=spec["radius"], sigma_s=float(spec["sigma_s"]),
                sigma_r=float(spec["sigma_r"]), tau=float(spec["tau"]),
                name=name, seed=seed, meta=dict(layers=nlayers))


def render_layers(specs, H, W, C=3, noise=0.0, seed=0, texture="uniform"):
    """Render an explicit scene: specs is a list of (kind, params, footprint)
    as for the layers of make_pair (kind "const" {c}, "plane" {a, b, c} or
    "quad" {c, alpha, beta, x0, y0}; footprint "all", ("rect", x0, x1, y0, y1)
    or ("ellipse", cx, cy, rx, ry)), each layer with its own texture of the
    given kind.  Returns (left, right, gt, occ) as make_pair's Pair holds them;
    with known surfaces the ground truth and the occlusion masks have closed
    forms (the tests check them)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    layers = [_Layer(kind, dict(params), fp, _Texture(rng, texture, C, -2.0, W + 300.0, -2.0, H + 2.0))
              for kind, params, fp in specs]
    return _render(layers, H, W, C, noise, rng)


def regions(pair, textured_std=4.0, jump=1.0, margin=3):
    """Evaluation regions of a synthetic pair, the counterparts of the paper's
    region names: "non_occ" = pixels visible in the right view; "non_occ_textl"
    = visible and textured (grey standard deviation over the 9x9 window >=
    textured_std levels); "non_occ_discont" = visible and farther than margin
    pixels (Chebyshev) from a ground-truth depth discontinuity (|gt| jumping by
    more than jump between 4-neighbours)."""
    grey = pair.left.astype(np.float64).mean(axis=2)
    m1 = ndimage.uniform_filter(grey, 9)
    m2 = ndimage.uniform_filter(grey * grey, 9)
    textured = np.sqrt(np.maximum(m2 - m1 * m1, 0.0)) >= textured_std
    j = np.zeros(pair.gt.shape, bool)
    dx = np.abs(np.diff(pair.gt, axis=1)) > jump
    dy = np.abs(np.diff(pair.gt, axis=0)) > jump
    j[:, 1:] |= dx
    j[:, :-1] |= dx
    j[1:, :] |= dy
    j[:-1, :] |= dy
    discont = ndimage.maximum_filter(j, size=2 * margin + 1)
    vis = ~pair.occ
    return {"non_occ": vis, "non_occ_textl": vis & textured, "non_occ_discont": vis & ~discont}


def make_workload(name: str, seed: int = 0) -> Pair:
    """The full-size pair of a workload."""
    return make_pair(name, seed)


def shifted_texture_pair(H, W, C, d0, seed, noise=0.0):
    """Known-answer pair: right = left shifted by the constant disparity d0.

    The texture is an independent uniform value per pixel of a world strip
    W + d0 wide, so I_l(x, y) = T(x, y) and I_r(x, y) = T(x + d0, y): the left
    pixel x appears at x - d0 in the right image.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    T = rng.integers(0, 256, size=(H, W + d0, C)).astype(np.float64)
    left = T[:, :W]
    right = T[:, d0:d0 + W]
    out = []
    for img in (left, right):
        if noise > 0:
            img = img + rng.normal(0.0, noise, img.shape)
        out.append(np.clip(np.rint(img), 0, 255).astype(np.uint8))
    return out[0], out[1]


def constant_image(H, W, C, value):
    return np.full((H, W, C), value, np.uint8)


def random_batch_specs(seed: int, n: int = 64, wrange=(320, 1024), hrange=(240, 768),
                       dchoices=(32, 64, 128, 192), rchoices=(4, 7, 11)):
    """Shapes of an uneven batch: W, H uniform integers, D and radius drawn from sets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(n):
        W = int(rng.integers(wrange[0], wrange[1] + 1))
        H = int(rng.integers(hrange[0], hrange[1] + 1))
        D = int(rng.choice(dchoices))
        r = int(rng.choice(rchoices))
        specs.append(dict(H=H, W=W, D=D, radius=r, sigma_s=float(r), sigma_r=12.0,
                          tau=30.0, seed=int(rng.integers(0, 2**31 - 1))))
    return specs
