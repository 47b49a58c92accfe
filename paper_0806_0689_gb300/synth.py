"""Seeded synthetic luma video: the input generator shared by tests and bench.

The paper's 18 test sequences are not available, so inputs are generated with
the shapes and motion statistics of its CIF/QCIF workloads (Sec. II-C and
Sec. IV): 8-bit luma frames, a horizontally biased motion field that is zero
about half of the time, and a few independently moving textured objects.

This module holds no motion-estimation arithmetic; it only draws frames.

Recipe (one frame sequence):

* texture  = Gaussian blur (sigma 1.5 px, radius 5, reflected border) of white
  noise with standard deviation 40 (noise drawn before the blur);
* frame 0  = clip(128 + texture) for the background layer, plus ``n_objects``
  rectangles with sides uniform in [16, 48] px, each with its own texture;
* every later frame: the background pans by a motion drawn as (0,0) with
  probability 1/2, otherwise (round(Laplace(0, sx)), round(Laplace(0, sy)))
  clamped to +-``max_motion``; the exposed strip gets fresh texture.  Each
  object moves by its own motion drawn the same way and is kept inside the
  frame;
* the rendered frame adds N(0, 1.5^2) noise per pixel, rounds and clips to
  [0, 255].

A frame pair is (cur = frame t+1, ref = frame t).
"""
from __future__ import annotations

import dataclasses

import numpy as np

_SIGMA = 1.5
_RADIUS = 5


def _kernel():
    x = np.arange(-_RADIUS, _RADIUS + 1, dtype=np.float64)
    k = np.exp(-(x * x) / (2.0 * _SIGMA * _SIGMA))
    return k / k.sum()


_K = _kernel()


def _blur(img):
    """Separable Gaussian blur with reflected borders (float64)."""
    h, w = img.shape
    p = np.pad(img, ((_RADIUS, _RADIUS), (_RADIUS, _RADIUS)), mode="reflect")
    t = np.zeros((h + 2 * _RADIUS, w), np.float64)
    for i, c in enumerate(_K):
        t += c * p[:, i:i + w]
    out = np.zeros((h, w), np.float64)
    for i, c in enumerate(_K):
        out += c * t[i:i + h, :]
    return out


def texture(rng, h, w, std=40.0):
    """Zero-mean blurred noise of shape (h, w)."""
    return _blur(rng.normal(0.0, std, size=(h, w)))


def _draw_motion(rng, scale, max_motion):
    if rng.random() < 0.5:
        return 0, 0
    mx = int(np.round(rng.laplace(0.0, scale[0])))
    my = int(np.round(rng.laplace(0.0, scale[1])))
    return int(np.clip(mx, -max_motion, max_motion)), int(np.clip(my, -max_motion, max_motion))


@dataclasses.dataclass
class _Obj:
    x: int
    y: int
    tex: np.ndarray


class Sequence:
    """Frame-by-frame generator; ``next()`` returns a uint8 (h, w) frame."""

    def __init__(self, w, h, seed, n_objects=3, scale=(2.0, 1.0), max_motion=7, noise=1.5):
        self.w, self.h = int(w), int(h)
        self.rng = np.random.default_rng(seed)
        self.scale = scale
        self.max_motion = int(max_motion)
        self.noise = float(noise)
        self.bg = 128.0 + texture(self.rng, self.h, self.w)
        self.objs = []
        for _ in range(n_objects):
            ow = int(self.rng.integers(16, 49))
            oh = int(self.rng.integers(16, 49))
            ow, oh = min(ow, self.w), min(oh, self.h)
            x = int(self.rng.integers(0, self.w - ow + 1))
            y = int(self.rng.integers(0, self.h - oh + 1))
            self.objs.append(_Obj(x, y, 128.0 + texture(self.rng, oh, ow)))
        self.t = 0

    def _pan(self, px, py):
        h, w = self.h, self.w
        new = np.empty_like(self.bg)
        # content moves by (px, py): new(x, y) = old(x - px, y - py)
        ys, yd = (slice(0, h - py), slice(py, h)) if py >= 0 else (slice(-py, h), slice(0, h + py))
        xs, xd = (slice(0, w - px), slice(px, w)) if px >= 0 else (slice(-px, w), slice(0, w + px))
        new[yd, xd] = self.bg[ys, xs]
        m = _RADIUS
        if px > 0:
            new[:, :px] = 128.0 + texture(self.rng, h, px + 2 * m)[:, m:m + px]
        elif px < 0:
            new[:, w + px:] = 128.0 + texture(self.rng, h, -px + 2 * m)[:, m:m - px]
        if py > 0:
            new[:py, :] = 128.0 + texture(self.rng, py + 2 * m, w)[m:m + py, :]
        elif py < 0:
            new[h + py:, :] = 128.0 + texture(self.rng, -py + 2 * m, w)[m:m - py, :]
        self.bg = new

    def _advance(self):
        px, py = _draw_motion(self.rng, self.scale, self.max_motion)
        if px or py:
            self._pan(px, py)
        for o in self.objs:
            mx, my = _draw_motion(self.rng, self.scale, self.max_motion)
            oh, ow = o.tex.shape
            o.x = int(np.clip(o.x + mx, 0, self.w - ow))
            o.y = int(np.clip(o.y + my, 0, self.h - oh))

    def next(self):
        if self.t > 0:
            self._advance()
        self.t += 1
        img = self.bg.copy()
        for o in self.objs:
            oh, ow = o.tex.shape
            img[o.y:o.y + oh, o.x:o.x + ow] = o.tex
        img += self.rng.normal(0.0, self.noise, size=img.shape)
        return np.clip(np.round(img), 0, 255).astype(np.uint8)


def sequence(w, h, n_frames, seed, n_objects=3, scale=(2.0, 1.0), max_motion=7):
    """Return a uint8 array (n_frames, h, w)."""
    g = Sequence(w, h, seed, n_objects=n_objects, scale=scale, max_motion=max_motion)
    return np.stack([g.next() for _ in range(n_frames)])


def pairs(frames):
    """(cur, ref) index pairs of a sequence: cur = t+1, ref = t."""
    return [(t + 1, t) for t in range(len(frames) - 1)]


# Workloads (seed = 1000*k + stream), sizes in pixels.
WORKLOADS = {
    "qcif": dict(w=176, h=144, n_objects=3),
    "cif": dict(w=352, h=288, n_objects=8),
    "720p": dict(w=1280, h=720, n_objects=8),
    "1080p": dict(w=1920, h=1088, n_objects=8),
    "2160p": dict(w=3840, h=2160, n_objects=8),
}


def workload_sequence(name, n_frames, seed, max_motion=7, scale=(2.0, 1.0)):
    p = WORKLOADS[name]
    return sequence(p["w"], p["h"], n_frames, seed, n_objects=p["n_objects"], scale=scale,
                    max_motion=max_motion)


def textured_frame(rng, h, w):
    """A strongly textured frame (white noise, no blur) for shift-recovery tests."""
    return rng.integers(0, 256, size=(h, w), dtype=np.uint8)


def shifted_pair(rng, h, w, sx, sy, margin=40):
    """(cur, ref) such that cur(x, y) = ref(x + sx, y + sy) everywhere.

    A larger textured canvas is cropped twice; every block's true motion
    vector is exactly (sx, sy) wherever that displacement stays in the frame.
    """
    big = rng.integers(0, 256, size=(h + 2 * margin, w + 2 * margin), dtype=np.uint8)
    ref = big[margin:margin + h, margin:margin + w].copy()
    cur = big[margin + sy:margin + sy + h, margin + sx:margin + sx + w].copy()
    return cur, ref
