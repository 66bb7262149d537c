"""CPU oracle of the registration + merge path (ctypes binding of hdrreg_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library
and its Python binding never do. The C source restates the paper's steps in
plain FP64 / integer loops and shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional, Sequence

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "hdrreg_oracle.c")
_LIB = os.path.join(_DIR, "liboracle.so")
_LIB_OMP = os.path.join(_DIR, "liboracle_omp.so")
_libs = {}
_parallel = False

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-Wall",
          "-Wno-unknown-pragmas", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary64 in the written order: no contraction), once
    serial (liboracle.so) and once with OpenMP over its independent loops
    (liboracle_omp.so)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_DIR, "hdrreg_oracle.h")))
    for out, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
            tmp = out + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", *CFLAGS, *extra, "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, out)
    return _LIB


def set_parallel(on: bool) -> None:
    """Route every oracle call to the OpenMP build (True) or the serial one (False, the
    default). The OpenMP build uses OMP_NUM_THREADS threads, else all cores."""
    global _parallel
    _parallel = bool(on)


def threads() -> int:
    """Threads the OpenMP build runs with (1 for the serial build)."""
    if not _parallel:
        return 1
    return int(C.CDLL(_LIB_OMP).orc_max_threads())


class Params(C.Structure):
    _fields_ = [
        ("tile", C.c_int), ("radius", C.c_int), ("patch_half", C.c_int),
        ("levels_max", C.c_int), ("min_level_size", C.c_int), ("grid_half", C.c_int),
        ("quad", C.c_int), ("corner_thresh", C.c_int), ("weed_iters", C.c_int),
        ("weed_delta_min", C.c_int), ("weed_delta_div", C.c_int), ("norm_mode", C.c_int),
        ("dt_iters", C.c_int), ("ssim_radius", C.c_int), ("propagate_full", C.c_int),
        ("pad_", C.c_int),
        ("weed_eps", C.c_double), ("sigma_s", C.c_double), ("sigma_r", C.c_double),
        ("ssim_sigma", C.c_double), ("we_sigma", C.c_double), ("flow_eps", C.c_double),
        ("weed_seed", C.c_uint64),
    ]


def make_params(cfg: Dict) -> Params:
    p = Params()
    for name, _ in Params._fields_:
        if name == "pad_":
            continue
        setattr(p, name, cfg[name])
    return p


def lib():
    path = _LIB_OMP if _parallel else _LIB
    if path not in _libs:
        build()
        _libs[path] = C.CDLL(path)
    return _libs[path]


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- a1
def normalize_ratio(ref, src, num, den):
    ref, src = _u8(ref), _u8(src)
    rn, sn = np.empty_like(ref), np.empty_like(src)
    lib().orc_normalize_ratio(_p(ref), _p(src), C.c_long(ref.size), num, den, _p(rn), _p(sn))
    return rn, sn


def histeq_lut(img):
    img = _u8(img)
    lut = np.empty(256, np.uint8)
    lib().orc_histeq_lut(_p(img), C.c_long(img.size), _p(lut))
    return lut


# ---------------------------------------------------------------- a2
def num_levels(w, h, levels_max=5, min_size=100):
    return lib().orc_num_levels(w, h, levels_max, min_size)


def downsample(img):
    img = _u8(img)
    h, w = img.shape
    out = np.empty((h // 2, w // 2), np.uint8)
    lib().orc_downsample(_p(img), w, h, _p(out))
    return out


def pyramid(img, levels):
    out = [_u8(img)]
    for _ in range(1, levels):
        out.append(downsample(out[-1]))
    return out


# ---------------------------------------------------------------- a3
def cornerness(img, x, y, q):
    img = _u8(img)
    h, w = img.shape
    sums = (C.c_long * 4)()
    c, m = C.c_long(), C.c_long()
    lib().orc_cornerness(_p(img), w, h, x, y, q, sums, C.byref(c), C.byref(m))
    return list(sums), c.value, m.value


def pick_corners(img, cfg):
    img = _u8(img)
    h, w = img.shape
    n = (w // cfg["tile"]) * (h // cfg["tile"])
    cxy = np.zeros((max(n, 1), 2), np.int32)
    valid = np.zeros(max(n, 1), np.uint8)
    score = np.zeros(max(n, 1), np.int64)
    prm = make_params(cfg)
    lib().orc_pick_corners(_p(img), w, h, C.byref(prm), _p(cxy), _p(valid), _p(score))
    return cxy[:n], valid[:n], score[:n]


# ---------------------------------------------------------------- a4
def project(H, x, y, w, h):
    H = _f64(H).reshape(9)
    xs, ys = C.c_double(), C.c_double()
    ok = lib().orc_project(_p(H), int(x), int(y), w, h, C.byref(xs), C.byref(ys))
    return xs.value, ys.value, bool(ok)


def search_center(H, x, y, w, h):
    H = _f64(H).reshape(9)
    cx, cy = C.c_int32(), C.c_int32()
    lib().orc_search_center(_p(H), int(x), int(y), w, h, C.byref(cx), C.byref(cy))
    return cx.value, cy.value


# ---------------------------------------------------------------- a5
def search(ref_n, src_n, H, cfg, corner_xy, valid):
    ref_n, src_n = _u8(ref_n), _u8(src_n)
    h, w = ref_n.shape
    H = _f64(H).reshape(9)
    cxy, valid = _i32(corner_xy).reshape(-1, 2), _u8(valid)
    n = valid.size
    ctr = np.zeros((max(n, 1), 2), np.int32)
    mxy = np.zeros((max(n, 1), 2), np.int32)
    cost = np.zeros(max(n, 1), np.uint32)
    prm = make_params(cfg)
    lib().orc_search(_p(ref_n), _p(src_n), w, h, _p(H), C.byref(prm), n, _p(cxy), _p(valid),
                     _p(ctr), _p(mxy), _p(cost))
    return ctr[:n], mxy[:n], cost[:n]


# ---------------------------------------------------------------- a-L
def predictor_input(ref_q, src_q, H):
    ref_q, src_q = _u8(ref_q), _u8(src_q)
    h, w = ref_q.shape
    out = np.zeros((h, w, 2))
    lib().orc_predictor_input(_p(ref_q), _p(src_q), w, h, _p(_f64(H).reshape(9)), _p(out))
    return out


def tile_labels(corner_xy, match_xy, valid, w, h, H):
    cxy, mxy, valid = _i32(corner_xy).reshape(-1, 2), _i32(match_xy).reshape(-1, 2), _u8(valid)
    n = valid.size
    lab = np.zeros((max(n, 1), 2), np.float32)
    lib().orc_tile_labels(_p(cxy), _p(mxy), _p(valid), n, w, h, _p(_f64(H).reshape(9)), _p(lab))
    return lab[:n]


def search_predicted(ref_n, src_n, H, cfg, corner_xy, valid, pred, fallback_cost, refine=0):
    ref_n, src_n = _u8(ref_n), _u8(src_n)
    h, w = ref_n.shape
    cxy, valid = _i32(corner_xy).reshape(-1, 2), _u8(valid)
    pred = np.ascontiguousarray(pred, np.float32).reshape(-1, 2)
    n = valid.size
    mxy = np.zeros((max(n, 1), 2), np.int32)
    cost = np.zeros(max(n, 1), np.uint32)
    fb = np.zeros(max(n, 1), np.uint8)
    prm = make_params(cfg)
    lib().orc_search_predicted(_p(ref_n), _p(src_n), w, h, _p(_f64(H).reshape(9)), C.byref(prm), n,
                               _p(cxy), _p(valid), _p(pred), int(refine),
                               C.c_uint32(int(fallback_cost)),
                               _p(mxy), _p(cost), _p(fb))
    return mxy[:n], cost[:n], fb[:n]


# ---------------------------------------------------------------- a6
def splitmix64_at(seed, k):
    f = lib().orc_splitmix64_at
    f.restype = C.c_uint64
    return f(C.c_uint64(seed), C.c_uint64(k))


def weed_sample(seed, it, nv):
    pick = (C.c_int * 4)()
    ok = lib().orc_weed_sample(C.c_uint64(seed), C.c_long(it), nv, pick)
    return (list(pick) if ok else None)


def solve8(A, b, tol=1e-12):
    A, b = _f64(A).reshape(64), _f64(b).reshape(8)
    x = np.zeros(8)
    st = lib().orc_solve8(_p(A), _p(b), _p(x), C.c_double(tol))
    return x, st


def mask_words(n):
    return np.zeros(n // 32 + 1, np.uint32)


def mask_to_bool(bits, n):
    bits = np.asarray(bits, np.uint32)
    idx = np.arange(n)
    return ((bits[idx >> 5] >> (idx & 31).astype(np.uint32)) & 1).astype(bool)


def weed(corner_xy, match_xy, valid, w, h, cfg, seed, iter_begin=0, iter_end=None, bits=None):
    cxy, mxy, valid = _i32(corner_xy).reshape(-1, 2), _i32(match_xy).reshape(-1, 2), _u8(valid)
    n = valid.size
    if iter_end is None:
        iter_end = cfg["weed_iters"]
    if bits is None:
        bits = mask_words(n)
    acc = C.c_int32()
    prm = make_params(cfg)
    lib().orc_weed(_p(cxy), _p(mxy), _p(valid), n, w, h, C.byref(prm), C.c_uint64(seed),
                   iter_begin, iter_end, _p(bits), C.byref(acc))
    return bits, acc.value


# ---------------------------------------------------------------- a7
def fit_homography(corner_xy, match_xy, bits, w, h, H_prev=None):
    cxy, mxy = _i32(corner_xy).reshape(-1, 2), _i32(match_xy).reshape(-1, 2)
    n = cxy.shape[0]
    bits = np.ascontiguousarray(bits, np.uint32)
    Hp = _f64(np.eye(3) if H_prev is None else H_prev).reshape(9)
    Ho = np.zeros(9)
    st = lib().orc_fit_homography(_p(cxy), _p(mxy), _p(bits), n, w, h, _p(Hp), _p(Ho))
    return Ho.reshape(3, 3), st


def fit_homography_real(p_xy, q_xy):
    p_xy, q_xy = _f64(p_xy).reshape(-1, 2), _f64(q_xy).reshape(-1, 2)
    Ho = np.zeros(9)
    st = lib().orc_fit_homography_real(_p(p_xy), _p(q_xy), p_xy.shape[0], _p(Ho))
    return Ho.reshape(3, 3), st


def match(ref_n, src_n, cfg):
    ref_n, src_n = _u8(ref_n), _u8(src_n)
    h, w = ref_n.shape
    n = (w // cfg["tile"]) * (h // cfg["tile"])
    cxy = np.zeros((max(n, 1), 2), np.int32)
    mxy = np.zeros((max(n, 1), 2), np.int32)
    cost = np.zeros(max(n, 1), np.uint32)
    valid = np.zeros(max(n, 1), np.uint8)
    bits = mask_words(n)
    H0 = np.zeros(9)
    stats = np.zeros(4 * 8, np.int32)
    prm = make_params(cfg)
    L = lib().orc_match(_p(ref_n), _p(src_n), w, h, C.byref(prm), _p(H0), _p(cxy), _p(mxy),
                        _p(cost), _p(valid), _p(bits), _p(stats))
    return dict(H0=H0.reshape(3, 3), corner_xy=cxy[:n], match_xy=mxy[:n], cost=cost[:n],
                valid=valid[:n], bits=bits, levels=L, level_stats=stats[:4 * L].reshape(L, 4))


# ---------------------------------------------------------------- a8
def dt_sigma(sigma_s, iters, i):
    s, a = C.c_double(), C.c_double()
    lib().orc_dt_sigma(C.c_double(sigma_s), iters, i, C.byref(s), C.byref(a))
    return s.value, a.value


def dt_filter(planes: Sequence[np.ndarray], guide, sigma_s, sigma_r, iters):
    guide = _u8(guide)
    h, w = guide.shape
    planes = [_f64(p).copy() for p in planes]
    arr = (C.c_void_p * len(planes))(*[p.ctypes.data for p in planes])
    lib().orc_dt_filter(arr, len(planes), _p(guide), w, h, C.c_double(sigma_s),
                        C.c_double(sigma_r), iters)
    return planes


def flow(guide, corner_xy, match_xy, bits, H0, cfg):
    guide = _u8(guide)
    h, w = guide.shape
    cxy, mxy = _i32(corner_xy).reshape(-1, 2), _i32(match_xy).reshape(-1, 2)
    bits = np.ascontiguousarray(bits, np.uint32)
    H0 = _f64(H0).reshape(9)
    fu, fv, nt = np.zeros((h, w)), np.zeros((h, w)), np.zeros((h, w))
    prm = make_params(cfg)
    lib().orc_flow(_p(guide), w, h, cxy.shape[0], _p(cxy), _p(mxy), _p(bits), _p(H0),
                   C.byref(prm), _p(fu), _p(fv), _p(nt))
    return fu, fv, nt


# ---------------------------------------------------------------- a9
def bilinear(img, x, y):
    img = _u8(img)
    h, w = img.shape
    f = lib().orc_bilinear
    f.restype = C.c_double
    return f(_p(img), w, h, C.c_double(x), C.c_double(y))


def bilinear_clipped(img, x, y):
    img = _u8(img)
    h, w = img.shape
    return bool(lib().orc_bilinear_clipped(_p(img), w, h, C.c_double(x), C.c_double(y)))


def warp(src_y, src_u, src_v, H0, flow_u, flow_v, want_clip=False):
    """(y, u, v) warped planes; with want_clip also the luma clip flags (uint8)."""
    src_y = _u8(src_y)
    h, w = src_y.shape
    H0 = _f64(H0).reshape(9)
    fu, fv = _f64(flow_u), _f64(flow_v)
    oy = np.zeros((h, w))
    clip = np.zeros((h, w), np.uint8)
    chroma = src_u is not None
    su = _u8(src_u) if chroma else None
    sv = _u8(src_v) if chroma else None
    ou = np.zeros((h // 2, w // 2)) if chroma else None
    ov = np.zeros((h // 2, w // 2)) if chroma else None
    lib().orc_warp(_p(src_y), _p(su), _p(sv), w, h, _p(H0), _p(fu), _p(fv), _p(oy), _p(ou),
                   _p(ov), _p(clip))
    return (oy, ou, ov, clip) if want_clip else (oy, ou, ov)


def clip_fragile(src_y, H0, flow_u, flow_v, delta=1e-3):
    """Reference pixels whose clip decision (orc_bilinear_clipped at H0(p) + F(p)) is not
    the same at every corner of the square of half-side ``delta`` pixels around the sample
    position: there a position error below ``delta`` (a float32 flow, float32 evaluation
    of H0) can flip the decision, so the merge weight of the sample is not determined by
    the position to that accuracy. Returns a bool map."""
    fu, fv = _f64(flow_u), _f64(flow_v)
    base = warp(src_y, None, None, H0, fu, fv, want_clip=True)[3]
    out = np.zeros(base.shape, bool)
    for sx in (-delta, delta):
        for sy in (-delta, delta):
            c = warp(src_y, None, None, H0, fu + sx, fv + sy, want_clip=True)[3]
            out |= c != base
    return out


# ---------------------------------------------------------------- a10
def ssim(x, y, sigma=1.5, radius=5):
    x, y = _f64(x), _f64(y)
    h, w = x.shape
    out = np.zeros((h, w))
    lib().orc_ssim(_p(x), _p(y), w, h, C.c_double(sigma), radius, _p(out))
    return out


def ghost_mask(ref_n, warped_y, mode=0, gain=1.0, src_lut=None, sigma=1.5, radius=5):
    ref_n, wy = _u8(ref_n), _f64(warped_y)
    h, w = ref_n.shape
    lut = _u8(np.arange(256) if src_lut is None else src_lut)
    q = np.zeros((h, w))
    lib().orc_ghost_mask(_p(ref_n), _p(wy), w, h, mode, C.c_double(gain), _p(lut),
                         C.c_double(sigma), radius, _p(q))
    return q


# ---------------------------------------------------------------- a11
def well_exposedness(z, sigma=0.2):
    f = lib().orc_well_exposedness
    f.restype = C.c_double
    return f(C.c_double(z), C.c_double(sigma))


def merge(ref_y, ref_u, ref_v, warped, qmaps, ratios, we_sigma=0.2, clips=None):
    """warped: list of (y, u, v) float arrays per source; ratios: list of floats t_k / t_ref;
    clips: per source the uint8 clip flags of the warped luma (``warp(..., want_clip=True)``),
    or None to take a sample as clipped when its value is <= 0 or >= 255."""
    ref_y = _u8(ref_y)
    h, w = ref_y.shape
    chroma = ref_u is not None
    k = len(warped)
    wy = [_f64(x[0]) for x in warped]
    wu = [_f64(x[1]) for x in warped] if chroma else []
    wv = [_f64(x[2]) for x in warped] if chroma else []
    qs = [_f64(q) for q in qmaps]
    arr = lambda L: (C.c_void_p * max(len(L), 1))(*[a.ctypes.data for a in L])
    rat = _f64(ratios)
    oy = np.zeros((h, w))
    ou = np.zeros((h // 2, w // 2)) if chroma else None
    ov = np.zeros((h // 2, w // 2)) if chroma else None
    ru, rv = (_u8(ref_u), _u8(ref_v)) if chroma else (None, None)
    cl = None if clips is None else [_u8(c) for c in clips]
    lib().orc_merge(w, h, _p(ref_y), _p(ru), _p(rv), k, arr(wy), arr(wu), arr(wv), arr(qs),
                    arr(cl) if cl is not None else None, _p(rat), C.c_double(we_sigma), _p(oy),
                    _p(ou), _p(ov))
    return oy, ou, ov


# ---------------------------------------------------------------- whole path
def register_merge(ref, srcs, ratios, cfg, want_intermediates=False):
    """ref: object with .y/.u/.v uint8 planes; srcs: list of such; ratios: list of (num, den)."""
    ry = _u8(ref.y)
    h, w = ry.shape
    chroma = ref.u is not None
    k = len(srcs)
    sy = [_u8(s.y) for s in srcs]
    su = [_u8(s.u) for s in srcs] if chroma else []
    sv = [_u8(s.v) for s in srcs] if chroma else []
    arr = lambda L: (C.c_void_p * max(len(L), 1))(*[a.ctypes.data for a in L]) if L else None
    num = np.array([r[0] for r in ratios], np.int32)
    den = np.array([r[1] for r in ratios], np.int32)
    oy = np.zeros((h, w))
    ou = np.zeros((h // 2, w // 2)) if chroma else None
    ov = np.zeros((h // 2, w // 2)) if chroma else None
    H0 = np.zeros((k, 9))
    inter = {}
    if want_intermediates:
        inter = {n: [np.zeros((h, w)) for _ in range(k)] for n in ("warped_y", "flow_u", "flow_v", "q")}
        inter["clip"] = [np.zeros((h, w), np.uint8) for _ in range(k)]
    prm = make_params(cfg)
    ru, rv = (_u8(ref.u), _u8(ref.v)) if chroma else (None, None)
    lib().orc_register_merge(
        w, h, _p(ry), _p(ru), _p(rv), k, arr(sy), arr(su), arr(sv), _p(num), _p(den),
        C.byref(prm), _p(oy), _p(ou), _p(ov), _p(H0),
        arr(inter["warped_y"]) if inter else None, arr(inter["flow_u"]) if inter else None,
        arr(inter["flow_v"]) if inter else None, arr(inter["q"]) if inter else None,
        arr(inter["clip"]) if inter else None)
    out = dict(y=oy, u=ou, v=ov, H0=H0.reshape(k, 3, 3))
    out.update(inter)
    return out


def is_inlier(H, p, q, w, h, eps):
    H = _f64(H).reshape(9)
    return bool(lib().orc_is_inlier(_p(H), int(p[0]), int(p[1]), int(q[0]), int(q[1]), w, h,
                                    C.c_double(eps)))


def pow2_scale(w):
    return lib().orc_pow2_scale(int(w))


def to_scaled(H, w):
    """A homography in Eq. 3's normalized coordinates rewritten for the S-scaled ones."""
    H = np.asarray(H, np.float64).reshape(3, 3)
    r = pow2_scale(w) / w
    T = H.copy()
    T[0, 2] /= r
    T[1, 2] /= r
    T[2, 0] *= r
    T[2, 1] *= r
    return T
