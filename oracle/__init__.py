"""CPU oracle for block-matching motion estimation -- TEST INFRASTRUCTURE ONLY.

Plain single-threaded C (``me_oracle.c``) behind ctypes.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares nothing with the CUDA library: no code,
headers, tables or constants.

Functions (each follows a passage of Jia & Zhang, "Directional Cross Diamond
Search Algorithm for Fast Block Motion Estimation"):

* :func:`fs`      -- full search, Sec. I / Table IX row "FS";
* :func:`dcds`    -- DCDS, Sec. III-B steps 1-4, switching strategies one/two;
                     ``simplified=True`` gives DCDS^S of Sec. IV-C;
* :func:`search`  -- the same DCDS search with a caller-supplied distortion
                     function, used for the ideal-condition analysis of
                     Sec. III-C-2 (Table VII);
* :func:`evaluate` -- the six measures of Sec. IV (MAD, MSE, NSP, PSNR,
                     distance and probability relative to FS).

Parity: FS, DCDS and evaluate are pinned by the tests (brute force, Table
VII, the counts of Sec. III-C-1, Table VI, closed forms).  The paper prints
only sequence averages for DCDS^S; it is pinned by examples worked by hand
from Sec. IV-C on the ideal surface (which fix its side rule, its tie rule
and what it counts) and by its exact recovery of every interior MV there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "me_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BDM_FN = ctypes.CFUNCTYPE(ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, no tuning)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [_SRC] + [os.path.join(_HERE, f) for f in os.listdir(_HERE) if f.endswith(".c") and f != "me_oracle.c"]
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in srcs)
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_sad.restype = ctypes.c_uint32
            lib.oracle_sad.argtypes = [P, P, I, I, I, I, I, I]
            lib.oracle_fs_frame.restype = I
            lib.oracle_fs_frame.argtypes = [P, P, I, I, I, I, I, P, P, P]
            lib.oracle_dcds_frame.restype = I
            lib.oracle_dcds_frame.argtypes = [P, P, I, I, I, I, I, I, P, P, P]
            lib.oracle_fs_blocks.restype = I
            lib.oracle_fs_blocks.argtypes = [P, P, I, I, I, I, I, P, I, P, P, P]
            lib.oracle_dcds_blocks.restype = I
            lib.oracle_dcds_blocks.argtypes = [P, P, I, I, I, I, I, I, P, I, P, P, P]
            lib.oracle_search.restype = I
            lib.oracle_search.argtypes = [BDM_FN, P, I, I, I, I, I, I, P]
            lib.oracle_eval_frame.restype = I
            lib.oracle_eval_frame.argtypes = [P, P, I, I, I, I, P, P, P, P]
            lib.oracle_hcsp_offsets.restype = None
            lib.oracle_hcsp_offsets.argtypes = [P]
            lib.oracle_search_from.restype = I
            lib.oracle_search_from.argtypes = [BDM_FN, P, I, I, I, I, I, I, I, I, I, I, I, P]
            lib.oracle_dcds_block_from.restype = I
            lib.oracle_dcds_block_from.argtypes = [P, P, I, I, I, I, I, I, I, I, I, I, I, I, P]
            lib.oracle_dcds_from_starts.restype = I
            lib.oracle_dcds_from_starts.argtypes = [P, P, I, I, I, I, I, P, P, P, P, P]
            lib.oracle_cnn_nparams.restype = I
            lib.oracle_cnn_features.restype = None
            lib.oracle_cnn_features.argtypes = [P, P, I, I, I, I, I, P, I, P, P]
            lib.oracle_cnn_forward.restype = None
            lib.oracle_cnn_forward.argtypes = [P, P, P, P]
            lib.oracle_cnn_loss_grad.restype = ctypes.c_double
            lib.oracle_cnn_loss_grad.argtypes = [P, P, P, I, I, I, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _frames(cur, ref):
    cur = np.ascontiguousarray(cur, dtype=np.uint8)
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    if cur.shape != ref.shape or cur.ndim != 2:
        raise ValueError("cur and ref must be 2-D uint8 frames of one shape")
    return cur, ref


def sad(cur, ref, bx, by, block, dx, dy) -> int:
    cur, ref = _frames(cur, ref)
    return int(_load().oracle_sad(_ptr(cur), _ptr(ref), cur.shape[1], bx, by, block, dx, dy))


def hcsp_offsets():
    out = np.zeros(14, dtype=np.int32)
    _load().oracle_hcsp_offsets(_ptr(out))
    return [tuple(int(v) for v in out[2 * i:2 * i + 2]) for i in range(7)]


def fs(cur, ref, block, rng):
    """Full search.  Returns (mv int16[nb,2], sad uint32[nb], nsp uint16[nb])."""
    cur, ref = _frames(cur, ref)
    h, w = cur.shape
    nb = (w // block) * (h // block)
    mv = np.zeros((nb, 2), np.int16)
    sd = np.zeros(nb, np.uint32)
    ns = np.zeros(nb, np.uint16)
    rc = _load().oracle_fs_frame(_ptr(cur), _ptr(ref), w, h, w, block, rng, _ptr(mv), _ptr(sd), _ptr(ns))
    if rc:
        raise ValueError("oracle_fs_frame rejected its arguments")
    return mv, sd, ns


def dcds(cur, ref, block, rng, simplified=False):
    """DCDS (or DCDS^S).  Returns (mv int16[nb,2], sad uint32[nb], nsp uint16[nb])."""
    cur, ref = _frames(cur, ref)
    h, w = cur.shape
    nb = (w // block) * (h // block)
    mv = np.zeros((nb, 2), np.int16)
    sd = np.zeros(nb, np.uint32)
    ns = np.zeros(nb, np.uint16)
    rc = _load().oracle_dcds_frame(_ptr(cur), _ptr(ref), w, h, w, block, rng, int(bool(simplified)),
                                   _ptr(mv), _ptr(sd), _ptr(ns))
    if rc:
        raise ValueError("oracle_dcds_frame rejected its arguments")
    return mv, sd, ns


def fs_blocks(cur, ref, block, rng, idx):
    """Full search for the raster block indices ``idx`` only."""
    cur, ref = _frames(cur, ref)
    h, w = cur.shape
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n = len(idx)
    mv = np.zeros((n, 2), np.int16)
    sd = np.zeros(n, np.uint32)
    ns = np.zeros(n, np.uint16)
    rc = _load().oracle_fs_blocks(_ptr(cur), _ptr(ref), w, h, w, block, rng, _ptr(idx), n,
                                  _ptr(mv), _ptr(sd), _ptr(ns))
    if rc:
        raise ValueError("oracle_fs_blocks rejected its arguments")
    return mv, sd, ns


def dcds_blocks(cur, ref, block, rng, idx, simplified=False):
    """DCDS (or DCDS^S) for the raster block indices ``idx`` only."""
    cur, ref = _frames(cur, ref)
    h, w = cur.shape
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n = len(idx)
    mv = np.zeros((n, 2), np.int16)
    sd = np.zeros(n, np.uint32)
    ns = np.zeros(n, np.uint16)
    rc = _load().oracle_dcds_blocks(_ptr(cur), _ptr(ref), w, h, w, block, rng, int(bool(simplified)),
                                    _ptr(idx), n, _ptr(mv), _ptr(sd), _ptr(ns))
    if rc:
        raise ValueError("oracle_dcds_blocks rejected its arguments")
    return mv, sd, ns


def search(bdm, rng, dx_lim=(-10**6, 10**6), dy_lim=(-10**6, 10**6), simplified=False):
    """DCDS search with a Python distortion function ``bdm(dx, dy) -> int``.

    Returns (mvx, mvy, bdm_at_mv, nsp).
    """
    cb = BDM_FN(lambda _u, dx, dy: int(bdm(dx, dy)))
    out = (ctypes.c_int64 * 4)()
    rc = _load().oracle_search(cb, None, rng, dx_lim[0], dx_lim[1], dy_lim[0], dy_lim[1],
                               int(bool(simplified)), ctypes.cast(out, ctypes.c_void_p))
    if rc:
        raise MemoryError("oracle_search failed")
    return int(out[0]), int(out[1]), int(out[2]), int(out[3])


def search_from(bdm, rng, start=(0, 0), prior_v=False, dx_lim=(-10**6, 10**6), dy_lim=(-10**6, 10**6),
                simplified=False, cand=(0, 0)):
    """DCDS from a proposal: the origin, ``cand`` and ``start`` are evaluated in
    this order and the best (the earliest on a tie) centres the first
    pattern, the HCSP or (prior_v) its transpose; then DCDS steps 2-4.
    Returns (mvx, mvy, bdm_at_mv, nsp)."""
    cb = BDM_FN(lambda _u, dx, dy: int(bdm(dx, dy)))
    out = (ctypes.c_int64 * 4)()
    rc = _load().oracle_search_from(cb, None, rng, dx_lim[0], dx_lim[1], dy_lim[0], dy_lim[1], int(cand[0]),
                                    int(cand[1]), int(start[0]), int(start[1]), int(bool(prior_v)),
                                    int(bool(simplified)), ctypes.cast(out, ctypes.c_void_p))
    if rc:
        raise MemoryError("oracle_search_from failed")
    return int(out[0]), int(out[1]), int(out[2]), int(out[3])


def dcds_from_starts(cur, ref, block, rng, starts, cands=None):
    """DCDS of every block from per-block (sx, sy, prior_v) starts (int16
    [nb, 3]), with cands (int16 [nb, 2], None = the origin) evaluated before
    each start."""
    cur, ref = _frames(cur, ref)
    h, w = cur.shape
    nb = (w // block) * (h // block)
    starts = np.ascontiguousarray(starts, dtype=np.int16).reshape(nb, 3)
    cands = None if cands is None else np.ascontiguousarray(cands, dtype=np.int16).reshape(nb, 2)
    mv = np.zeros((nb, 2), np.int16)
    sd = np.zeros(nb, np.uint32)
    ns = np.zeros(nb, np.uint16)
    rc = _load().oracle_dcds_from_starts(_ptr(cur), _ptr(ref), w, h, w, block, rng, _ptr(starts), _ptr(cands),
                                         _ptr(mv), _ptr(sd), _ptr(ns))
    if rc:
        raise ValueError("oracle_dcds_from_starts rejected its arguments")
    return mv, sd, ns


# ---------------------------------------------------------------- learned proposal

def cnn_nparams():
    return int(_load().oracle_cnn_nparams())


def cnn_features(cur, ref, px, py, nbr=None, block=16):
    """(x [2, 32, 32] float64, mvf [8] float64) of the 16x16 region at (px, py);
    nbr is the motion field in the grid of `block` (8 or 16) pixels."""
    cur, ref = _frames(cur, ref)
    h, w = cur.shape
    x = np.zeros((2, 32, 32), np.float64)
    mvf = np.zeros(8, np.float64)
    nbr = None if nbr is None else np.ascontiguousarray(nbr, dtype=np.int16)
    _load().oracle_cnn_features(_ptr(cur), _ptr(ref), w, h, w, px, py, _ptr(nbr), block, _ptr(x), _ptr(mvf))
    return x, mvf


def cnn_forward(params, x, mvf):
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    mvf = np.ascontiguousarray(mvf, dtype=np.float64)
    out = np.zeros(68, np.float64)
    _load().oracle_cnn_forward(_ptr(params), _ptr(x), _ptr(mvf), _ptr(out))
    return out


def cnn_loss_grad(params, x, mvf, labels, grad=None):
    """Loss of one block and its gradient (added into ``grad`` if given)."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    mvf = np.ascontiguousarray(mvf, dtype=np.float64)
    if grad is None:
        grad = np.zeros_like(params)
    loss = _load().oracle_cnn_loss_grad(_ptr(params), _ptr(x), _ptr(mvf), int(labels[0]), int(labels[1]),
                                        int(labels[2]), _ptr(grad))
    return float(loss), grad


def cnn_start(logits, px, py, w, h, rng, block=16):
    """cnn_raw_start clamped to the window and the frame of the block of
    `block` pixels at (px, py)."""
    sx, sy, pv = cnn_raw_start(logits)
    sx = max(max(-rng, -px), min(min(rng, w - block - px), sx))
    sy = max(max(-rng, -py), min(min(rng, h - block - py), sy))
    return sx, sy, pv


def median_start(mv, k, nbx, px, py, w, h, rng, block=16):
    """Start of the non-learned control for block k (of `block` pixels, at
    (px, py)): the component-wise median of the left, top and top-right final
    MVs (absent neighbours count as (0,0)), clamped to the window and the
    frame; vertical prior when the median's |dy| > |dx|."""
    bx, by = k % nbx, k // nbx
    cand = []
    for ax, ay in ((bx - 1, by), (bx, by - 1), (bx + 1, by - 1)):
        if 0 <= ax < nbx and ay >= 0:
            cand.append((int(mv[ay * nbx + ax][0]), int(mv[ay * nbx + ax][1])))
        else:
            cand.append((0, 0))
    sx = sorted(c[0] for c in cand)[1]
    sy = sorted(c[1] for c in cand)[1]
    pv = int(abs(sy) > abs(sx))
    sx = max(max(-rng, -px), min(min(rng, w - block - px), sx))
    sy = max(max(-rng, -py), min(min(rng, h - block - py), sy))
    return sx, sy, pv


def _regions(w, h, block):
    """The 16x16 regions of a frame in raster order, each with the indices
    and pixel origins of its blocks (one 16x16 block, or four 8x8 blocks in
    the order top-left, top-right, bottom-left, bottom-right)."""
    nbx = w // block
    per = 16 // block
    for ry in range(h // 16):
        for rx in range(w // 16):
            blocks = []
            for j in range(per):
                for i in range(per):
                    bx, by = rx * per + i, ry * per + j
                    blocks.append((by * nbx + bx, bx * block, by * block))
            yield rx * 16, ry * 16, blocks


def _search_regions(cur, ref, rng, block, propose):
    """DCDS of every block from a start shared by the blocks of its 16x16
    region.  Regions run in raster order, so the left, top and top-right
    neighbours of a region's top-left block are final before it starts.
    propose(mv, k0, px, py) returns the region's raw start (sx, sy, prior_v)
    and the candidate evaluated before it (ax, ay), k0 being the index of its
    top-left block; every block clamps both to its own window and frame.
    Returns (mv, sad, nsp, starts)."""
    cur, ref = _frames(cur, ref)
    h, w = cur.shape
    if w % 16 or h % 16 or block not in (8, 16):
        raise ValueError("shared-start searches need w, h multiples of 16 and 8x8 or 16x16 blocks")
    nb = (w // block) * (h // block)
    mv = np.zeros((nb, 2), np.int16)
    sd = np.zeros(nb, np.uint32)
    ns = np.zeros(nb, np.uint16)
    starts = np.zeros((nb, 3), np.int16)
    out = (ctypes.c_int64 * 4)()
    L = _load()
    for px, py, blocks in _regions(w, h, block):
        sx, sy, pv, ax, ay = propose(mv, blocks[0][0], px, py)
        for k, bx, by in blocks:
            starts[k] = (max(max(-rng, -bx), min(min(rng, w - block - bx), sx)),
                         max(max(-rng, -by), min(min(rng, h - block - by), sy)), pv)
            rc = L.oracle_dcds_block_from(_ptr(cur), _ptr(ref), w, h, w, block, rng, bx, by, int(ax), int(ay),
                                          int(sx), int(sy), int(pv), ctypes.cast(out, ctypes.c_void_p))
            if rc:
                raise MemoryError("oracle_dcds_block_from failed")
            mv[k] = (out[0], out[1])
            sd[k] = out[2]
            ns[k] = out[3]
    return mv, sd, ns, starts


def median_dcds(cur, ref, rng, block=16):
    """DCDS from the neighbour-median start: 16x16 blocks each take the median
    of their own left, top and top-right neighbours; 8x8 blocks share the
    start of their 16x16 region, the median of the neighbours of its
    top-left block.  Returns (mv, sad, nsp, starts)."""
    h, w = np.asarray(cur).shape
    nbx = w // block

    def propose(mv, k0, px, py):
        sx, sy = neighbour_median(mv, k0, nbx)
        return sx, sy, int(abs(sy) > abs(sx)), 0, 0

    return _search_regions(cur, ref, rng, block, propose)


def neighbour_median(mv, k0, nbx):
    """Component-wise median of the left, top and top-right final MVs of block
    k0 (an absent neighbour counts as (0,0))."""
    cand = []
    bx, by = k0 % nbx, k0 // nbx
    for ax, ay in ((bx - 1, by), (bx, by - 1), (bx + 1, by - 1)):
        ok = 0 <= ax < nbx and ay >= 0
        cand.append((int(mv[ay * nbx + ax][0]), int(mv[ay * nbx + ax][1])) if ok else (0, 0))
    return sorted(c[0] for c in cand)[1], sorted(c[1] for c in cand)[1]


def region_medians(field, w, h, block):
    """Per block (int16 [nb, 2]): the neighbour median of its 16x16 region's
    top-left block, taken from a final motion field -- the candidate the
    learned search evaluates before the network's start."""
    nbx = w // block
    out = np.zeros(((w // block) * (h // block), 2), np.int16)
    for _, _, blocks in _regions(w, h, block):
        out[[k for k, _, _ in blocks]] = neighbour_median(field, blocks[0][0], nbx)
    return out


def mvp_counts(frames, R):
    """Counts of the Sec. II-C statistics (the layout of me_mvp_stats) for 16x16
    blocks.  frames: list of (cur, ref, mv_fs, range).  Each block's current
    best-matched point in a set is the strict SAD minimum over the set's points
    inside the window and the frame, the centre compared first."""
    side = 2 * R + 1
    q = side * side
    out = np.zeros(35 * q, np.int64)
    s1 = [(0, 0), (-2, 0), (-1, 0), (1, 0), (2, 0), (0, 2), (0, 1), (0, -1), (0, -2)]
    s2 = [(0, 0)] + [(i % 5 - 2, i // 5 - 2) for i in range(25) if i != 12]
    for cur, ref, mv_fs, rf in frames:
        cur_c, ref_c = _frames(cur, ref)
        h, w = cur_c.shape
        nbx = w // 16
        for k in range(nbx * (h // 16)):
            bx, by = k % nbx, k // nbx
            px, py = bx * 16, by * 16

            def ok(dx, dy):
                return -rf <= dx <= rf and -rf <= dy <= rf and 0 <= px + dx <= w - 16 and 0 <= py + dy <= h - 16

            def best(points):
                bi, bs = None, None
                for i, (dx, dy) in enumerate(points):
                    if not ok(dx, dy):
                        continue
                    s = sad(cur_c, ref_c, px, py, 16, dx, dy)
                    if bs is None or s < bs:
                        bi, bs = i, s
                return bi

            p1 = best(s1)
            p2s = s2[best(s2)]
            p2 = (p2s[1] + 2) * 5 + (p2s[0] + 2)
            qx, qy = int(mv_fs[k][0]), int(mv_fs[k][1])
            if abs(qx) > R or abs(qy) > R:
                continue
            qi = (qy + R) * side + (qx + R)
            out[qi] += 1
            out[q + p1 * q + qi] += 1
            out[10 * q + qi * 25 + p2] += 1
    return out


START_GATE = 0.6


def start_confidence(logits):
    """Product of the softmax maxima of the dx and dy heads (fp64)."""
    z = np.asarray(logits, np.float64)
    p = 1.0
    for seg in (z[:33], z[33:66]):
        p /= float(np.sum(np.exp(seg - seg.max())))
    return p


def cnn_raw_start(logits):
    """(sx, sy, prior_v) from logits before clamping: the argmax of the dx and
    dy heads (ties go to the class nearest the centre, checked in the order
    0, -1, +1, -2, +2, ...), replaced by the origin when the network is not
    confident (start_confidence below START_GATE); vertical prior when the V
    logit is strictly larger."""
    def centre_out_argmax(z):
        best, bv = 0, z[16]
        for a in range(1, 17):
            for d in (-a, a):
                if z[d + 16] > bv:
                    best, bv = d, z[d + 16]
        return best
    sx, sy = centre_out_argmax(logits[:33]), centre_out_argmax(logits[33:66])
    if start_confidence(logits) < START_GATE:
        sx, sy = 0, 0
    return sx, sy, int(logits[67] > logits[66])


def learned_dcds(cur, ref, rng, params, block=16):
    """Learned-start DCDS of a frame: one proposal per 16x16 region (one
    16x16 block, or four 8x8 blocks that share it), regions in raster order
    so that the left, top and top-right neighbours of a region's top-left
    block are final before it starts.  Each block evaluates the origin, the
    neighbours' median and the network's start, in this order; the best
    centres the first pattern (HCSP, or its transpose for a vertical prior).
    Returns (mv, sad, nsp, starts, logits), logits per region in raster
    order."""
    h, w = np.asarray(cur).shape
    logits = np.zeros(((w // 16) * (h // 16), 68), np.float64)
    count = [0]
    nbx = w // block

    def propose(mv, k0, px, py):
        x, mvf = cnn_features(cur, ref, px, py, mv, block)
        lg = cnn_forward(params, x, mvf)
        logits[count[0]] = lg
        count[0] += 1
        sx, sy, pv = cnn_raw_start(lg)
        mx, my = neighbour_median(mv, k0, nbx)
        return sx, sy, pv, mx, my

    mv, sd, ns, starts = _search_regions(cur, ref, rng, block, propose)
    return mv, sd, ns, starts, logits


def evaluate(cur, ref, block, mv, mv_fs=None, nsp=None):
    """The six measures of Sec. IV for one frame.  Returns a dict."""
    cur, ref = _frames(cur, ref)
    h, w = cur.shape
    mv = np.ascontiguousarray(mv, dtype=np.int16)
    mv_fs = None if mv_fs is None else np.ascontiguousarray(mv_fs, dtype=np.int16)
    nsp = None if nsp is None else np.ascontiguousarray(nsp, dtype=np.uint16)
    out = np.zeros(6, np.float64)
    rc = _load().oracle_eval_frame(_ptr(cur), _ptr(ref), w, h, w, block, _ptr(mv), _ptr(mv_fs),
                                   _ptr(nsp), _ptr(out))
    if rc:
        raise ValueError("oracle_eval_frame rejected its arguments")
    return dict(mad=out[0], mse=out[1], nsp=out[2], psnr=out[3], distance=out[4], probability=out[5])
