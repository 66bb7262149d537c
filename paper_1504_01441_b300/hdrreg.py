"""Python binding of the hdrreg C ABI (include/hdrreg.h).

Argument marshalling only: every step runs in the CUDA kernels of
libhdrreg.so. PyTorch provides device memory and the current stream. If the
library is missing or cannot be loaded this module raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, List, Optional, Sequence, Tuple

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhdrreg.so")

NORM_RATIO = 0
NORM_HISTEQ = 1

STATUS = {0: "OK", 1: "E_INVALID_ARG", 2: "E_CUDA", 3: "E_DEGENERATE", 4: "E_TIMEOUT",
          5: "E_UNSUPPORTED", 6: "E_WORKSPACE"}

EXPORTS = [
    "hdrreg_params_default", "hdrreg_params_paper", "hdrreg_last_error", "hdrreg_version", "hdrreg_launch_count",
    "hdrreg_num_levels",
    "hdrreg_validate_params", "hdrreg_num_tiles", "hdrreg_normalize_workspace_size",
    "hdrreg_normalize_exposure", "hdrreg_pyramid_bytes", "hdrreg_build_pyramid",
    "hdrreg_local_search", "hdrreg_weed_workspace_size", "hdrreg_weed", "hdrreg_weed_static",
    "hdrreg_fit_homography", "hdrreg_weed_fit_supported", "hdrreg_weed_fit",
    "hdrreg_flow_workspace_size", "hdrreg_flow_upsample", "hdrreg_warp", "hdrreg_merge",
    "hdrreg_register_merge_workspace_size", "hdrreg_register_merge",
    "hdrreg_register_merge_batch_workspace_size", "hdrreg_register_merge_batch",
    "hdrreg_register_merge_multi_workspace_size", "hdrreg_register_merge_multi",
    "hdrreg_register_merge_staged_workspace_size", "hdrreg_register_merge_staged",
    "hdrreg_register_merge_host_workspace_size", "hdrreg_register_merge_host",
    "hdrreg_fuse_workspace_size", "hdrreg_fuse",
    "hdrreg_gemm_bf16", "hdrreg_cnn_workspace_size", "hdrreg_cnn_out_dims", "hdrreg_cnn_forward",
    "hdrreg_cnn_backward", "hdrreg_cnn_adam", "hdrreg_cnn_activation",
    "hdrreg_cnn_infer_workspace_size", "hdrreg_cnn_infer", "hdrreg_predictor_input",
    "hdrreg_tile_labels",
    "hdrreg_predictor_crops", "hdrreg_local_search_predicted",
]

CNN_PARAMS = 119538

MAX_LANES = 16


class HdrregError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hdrreg {STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("tile", C.c_int), ("radius", C.c_int), ("patch_half", C.c_int),
        ("levels_max", C.c_int), ("min_level_size", C.c_int), ("grid_half", C.c_int),
        ("quad", C.c_int), ("corner_thresh", C.c_int), ("weed_iters", C.c_int),
        ("weed_delta_min", C.c_int), ("weed_delta_div", C.c_int), ("norm_mode", C.c_int),
        ("dt_iters", C.c_int), ("ssim_radius", C.c_int), ("propagate_full", C.c_int),
        ("output_mode", C.c_int),
        ("weed_eps", C.c_double), ("sigma_s", C.c_double), ("sigma_r", C.c_double),
        ("ssim_sigma", C.c_double), ("we_sigma", C.c_double), ("flow_eps", C.c_double),
        ("weed_seed", C.c_uint64), ("predictor", C.c_void_p), ("fallback_cost", C.c_uint32),
        ("predictor_refine", C.c_int32), ("search_threads", C.c_int32),
    ]

    def as_dict(self) -> Dict:
        return {n: getattr(self, n) for n, _ in self._fields_
                if n not in ("predictor", "fallback_cost", "predictor_refine")}


class Frame(C.Structure):
    _fields_ = [("y", C.c_void_p), ("u", C.c_void_p), ("v", C.c_void_p)]


class PlanesF32(C.Structure):
    _fields_ = [("y", C.c_void_p), ("u", C.c_void_p), ("v", C.c_void_p)]


class MergeSrc(C.Structure):
    _fields_ = [("y", C.c_void_p), ("u", C.c_void_p), ("v", C.c_void_p), ("ref_n", C.c_void_p),
                ("src_lut", C.c_void_p), ("ratio_num", C.c_int), ("ratio_den", C.c_int),
                ("clip", C.c_void_p)]


class Stack(C.Structure):
    _fields_ = [("ref", C.POINTER(Frame)), ("srcs", C.POINTER(Frame)),
                ("ratio_num", C.POINTER(C.c_int)), ("ratio_den", C.POINTER(C.c_int)),
                ("out", PlanesF32), ("diag", C.c_void_p)]


class FuseSrc(C.Structure):
    _fields_ = [("y", C.c_void_p), ("u", C.c_void_p), ("v", C.c_void_p), ("q", C.c_void_p)]


class StackEx(C.Structure):
    _fields_ = [("s", Stack), ("w", C.c_int), ("h", C.c_int), ("nsrc", C.c_int),
                ("p", C.POINTER(Params))]


class Diag(C.Structure):
    _fields_ = [("H0", C.c_double * 9), ("levels", C.c_int32), ("tiles", C.c_int32),
                ("valid", C.c_int32), ("kept", C.c_int32), ("fit_status", C.c_int32),
                ("fallbacks", C.c_int32), ("flow_status", C.c_int32), ("reserved", C.c_int32)]


_lib = None


def lib():
    """Load libhdrreg.so (built in-tree by build.py); raise if it is not there."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"hdrreg CUDA library not built: {LIB_PATH} (run build.py)")
        L = C.CDLL(LIB_PATH)
        sz = C.c_size_t
        vp = C.c_void_p
        i = C.c_int
        L.hdrreg_last_error.restype = C.c_char_p
        L.hdrreg_version.restype = C.c_char_p
        L.hdrreg_launch_count.restype = C.c_ulonglong
        L.hdrreg_params_default.argtypes = [C.POINTER(Params)]
        L.hdrreg_params_paper.argtypes = [C.POINTER(Params)]
        L.hdrreg_validate_params.argtypes = [C.POINTER(Params)]
        L.hdrreg_num_levels.argtypes = [i, i, C.POINTER(Params)]
        L.hdrreg_num_tiles.argtypes = [i, i, i]
        L.hdrreg_normalize_workspace_size.restype = sz
        L.hdrreg_normalize_workspace_size.argtypes = [i]
        L.hdrreg_normalize_exposure.argtypes = [vp, vp, i, i, i, i, i, vp, vp, vp, vp, sz, vp]
        L.hdrreg_pyramid_bytes.restype = sz
        L.hdrreg_pyramid_bytes.argtypes = [i, i, i]
        L.hdrreg_build_pyramid.argtypes = [vp, i, i, i, vp, vp]
        L.hdrreg_local_search.argtypes = [vp, vp, i, i, vp, C.POINTER(Params), vp, vp, vp, vp, vp]
        L.hdrreg_weed_workspace_size.restype = sz
        L.hdrreg_weed_workspace_size.argtypes = [i]
        L.hdrreg_weed.argtypes = [vp, vp, vp, i, i, i, C.POINTER(Params), C.c_uint64, i, i, vp,
                                  vp, sz, vp]
        L.hdrreg_weed_static.argtypes = [vp, vp, vp, i, i, i, C.POINTER(Params), C.c_uint64, i,
                                         i, vp, vp]
        L.hdrreg_fit_homography.argtypes = [vp, vp, vp, i, i, i, vp, vp, vp, vp]
        L.hdrreg_weed_fit_supported.argtypes = [i]
        L.hdrreg_weed_fit.argtypes = [vp, vp, vp, i, i, i, C.POINTER(Params), C.c_uint64, i, i,
                                      vp, vp, vp, vp, vp, vp]
        L.hdrreg_flow_workspace_size.restype = sz
        L.hdrreg_flow_workspace_size.argtypes = [i, i]
        L.hdrreg_flow_upsample.argtypes = [vp, i, i, vp, vp, vp, i, vp, C.POINTER(Params), vp,
                                           vp, vp, sz, vp]
        L.hdrreg_warp.argtypes = [C.POINTER(Frame), i, i, vp, vp, vp, C.POINTER(PlanesF32), vp,
                                  vp]
        L.hdrreg_merge.argtypes = [C.POINTER(Frame), i, i, i, C.POINTER(MergeSrc),
                                   C.POINTER(Params), C.POINTER(PlanesF32), vp, vp]
        L.hdrreg_register_merge_workspace_size.restype = sz
        L.hdrreg_register_merge_workspace_size.argtypes = [i, i, i, C.POINTER(Params)]
        L.hdrreg_register_merge.argtypes = [C.POINTER(Frame), i, i, i, C.POINTER(Frame),
                                            C.POINTER(C.c_int), C.POINTER(C.c_int),
                                            C.POINTER(Params), vp, sz, C.POINTER(PlanesF32),
                                            vp, vp]
        L.hdrreg_register_merge_batch_workspace_size.restype = sz
        L.hdrreg_register_merge_batch_workspace_size.argtypes = [i, i, i, i, C.POINTER(Params)]
        L.hdrreg_register_merge_batch.argtypes = [C.POINTER(Stack), i, i, i, i, i,
                                                  C.POINTER(Params), vp, sz, vp]
        L.hdrreg_fuse_workspace_size.restype = sz
        L.hdrreg_fuse_workspace_size.argtypes = [i, i, i, i]
        L.hdrreg_fuse.argtypes = [C.POINTER(Frame), i, i, i, C.POINTER(FuseSrc), i, C.c_double,
                                  C.POINTER(PlanesF32), vp, sz, vp]
        L.hdrreg_register_merge_host_workspace_size.restype = sz
        L.hdrreg_register_merge_host_workspace_size.argtypes = [i, i, i, i, C.POINTER(Params)]
        L.hdrreg_register_merge_host.argtypes = [C.POINTER(Stack), i, i, i, i, i,
                                                 C.POINTER(Params), vp, sz, vp]
        L.hdrreg_register_merge_multi_workspace_size.restype = sz
        L.hdrreg_register_merge_multi_workspace_size.argtypes = [C.POINTER(StackEx), i, i]
        L.hdrreg_register_merge_multi.argtypes = [C.POINTER(StackEx), i, i, vp, sz, vp]
        L.hdrreg_register_merge_staged_workspace_size.restype = sz
        L.hdrreg_register_merge_staged_workspace_size.argtypes = [C.POINTER(StackEx), i, i]
        L.hdrreg_register_merge_staged.argtypes = [C.POINTER(StackEx), i, i, vp, sz, vp]
        L.hdrreg_gemm_bf16.argtypes = [vp, i, vp, i, i, i, i, vp, i, vp, vp]
        L.hdrreg_cnn_workspace_size.restype = sz
        L.hdrreg_cnn_workspace_size.argtypes = [i, i, i]
        L.hdrreg_cnn_out_dims.argtypes = [i, i, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.hdrreg_cnn_forward.argtypes = [vp, vp, i, i, i, vp, vp, sz, vp, vp]
        L.hdrreg_cnn_backward.argtypes = [vp, vp, i, i, i, vp, vp, vp, vp, vp, vp, sz, vp, vp]
        L.hdrreg_cnn_infer_workspace_size.restype = sz
        L.hdrreg_cnn_infer_workspace_size.argtypes = [i, i, i]
        L.hdrreg_cnn_infer.argtypes = [vp, vp, i, i, i, vp, vp, sz, vp, vp]
        L.hdrreg_cnn_adam.argtypes = [vp, vp, vp, vp, i, C.c_float, vp]
        L.hdrreg_cnn_activation.argtypes = [vp, i, i, i, i, C.POINTER(C.c_void_p),
                                             C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.hdrreg_predictor_input.argtypes = [vp, vp, i, i, vp, vp, vp]
        L.hdrreg_tile_labels.argtypes = [vp, vp, vp, i, i, i, vp, vp, vp]
        L.hdrreg_predictor_crops.argtypes = [vp, i, i, vp, vp, i, i, vp, i, i, C.c_float, vp, vp,
                                             vp, vp]
        L.hdrreg_local_search_predicted.argtypes = [vp, vp, i, i, vp, C.POINTER(Params), vp, i, i,
                                                    i, C.c_uint32, vp, vp, vp, vp, vp, vp]
        for name in EXPORTS:
            if not hasattr(L, name):
                raise ImportError(f"libhdrreg.so does not export {name}")
        _lib = L
    return _lib


def version() -> str:
    return lib().hdrreg_version().decode()


def launch_count() -> int:
    """Kernels enqueued by the library so far in this process."""
    return int(lib().hdrreg_launch_count())


def params(**over) -> Params:
    """Library defaults (the paper's values where it gives them), with overrides."""
    p = Params()
    lib().hdrreg_params_default(C.byref(p))
    for k, v in over.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def params_paper(**over) -> Params:
    """The paper-exact preset: the defaults with the corners' whole displacement spread by
    the flow (Sec. 2.4), with overrides."""
    p = Params()
    lib().hdrreg_params_paper(C.byref(p))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def params_from_dict(d: Dict) -> Params:
    return params(**{k: v for k, v in d.items() if k != "pad_"})


def _check(st: int):
    if st != 0:
        raise HdrregError(st, lib().hdrreg_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("hdrreg expects CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("hdrreg expects contiguous tensors")
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _empty(shape, dtype, like):
    import torch
    return torch.empty(shape, dtype=dtype, device=like.device)


def num_levels(w: int, h: int, p: Params) -> int:
    return lib().hdrreg_num_levels(w, h, C.byref(p))


def num_tiles(w: int, h: int, tile: int) -> int:
    return lib().hdrreg_num_tiles(w, h, tile)


# ---------------------------------------------------------------- a1
def normalize_exposure(ref_y, src_y, mode=NORM_RATIO, ratio=(1, 1), stream=None):
    """-> (ref_n, src_n, luts[2, 256])"""
    import torch
    h, w = ref_y.shape
    ref_n, src_n = torch.empty_like(ref_y), torch.empty_like(src_y)
    luts = _empty((2, 256), torch.uint8, ref_y)
    ws_n = lib().hdrreg_normalize_workspace_size(mode)
    ws = _empty((max(ws_n, 1),), torch.uint8, ref_y)
    _check(lib().hdrreg_normalize_exposure(_ptr(ref_y), _ptr(src_y), w, h, mode, ratio[0],
                                           ratio[1], _ptr(ref_n), _ptr(src_n), _ptr(luts),
                                           _ptr(ws), ws_n, _stream(stream)))
    return ref_n, src_n, luts


# ---------------------------------------------------------------- a2
def build_pyramid(level0, levels: int, stream=None) -> List:
    import torch
    h, w = level0.shape
    nb = lib().hdrreg_pyramid_bytes(w, h, levels)
    buf = _empty((max(nb, 1),), torch.uint8, level0)
    _check(lib().hdrreg_build_pyramid(_ptr(level0), w, h, levels, _ptr(buf), _stream(stream)))
    out, off = [level0], 0
    for l in range(1, levels):
        lw, lh = w >> l, h >> l
        out.append(buf[off:off + lw * lh].view(lh, lw))
        off += lw * lh
    return out


# ---------------------------------------------------------------- a3-a5
def local_search(ref_n, src_n, H, p: Params, stream=None):
    """-> corner_xy [n,2] int32, match_xy [n,2] int32, cost [n] int32 (uint32 bits), valid [n] u8"""
    import torch
    h, w = ref_n.shape
    n = num_tiles(w, h, p.tile)
    corner = _empty((max(n, 1), 2), torch.int32, ref_n)
    match = _empty((max(n, 1), 2), torch.int32, ref_n)
    cost = _empty((max(n, 1),), torch.int32, ref_n)
    valid = _empty((max(n, 1),), torch.uint8, ref_n)
    _check(lib().hdrreg_local_search(_ptr(ref_n), _ptr(src_n), w, h, _ptr(H), C.byref(p),
                                     _ptr(corner), _ptr(match), _ptr(cost), _ptr(valid),
                                     _stream(stream)))
    return corner[:n], match[:n], cost[:n], valid[:n]


# ---------------------------------------------------------------- a6
def weed(corner_xy, match_xy, valid, w: int, h: int, p: Params, seed: int, iter_begin=0,
         iter_end=None, mask=None, stream=None):
    """OR the inliers of iterations [iter_begin, iter_end) into mask (int32 words); -> mask"""
    import torch
    n = valid.numel()
    if iter_end is None:
        iter_end = p.weed_iters
    if mask is None:
        mask = torch.zeros((n // 32 + 1,), dtype=torch.int32, device=valid.device)
    ws_n = lib().hdrreg_weed_workspace_size(n)
    ws = _empty((ws_n,), torch.uint8, valid)
    _check(lib().hdrreg_weed(_ptr(corner_xy), _ptr(match_xy), _ptr(valid), n, w, h, C.byref(p),
                             C.c_uint64(seed), iter_begin, iter_end, _ptr(mask), _ptr(ws), ws_n,
                             _stream(stream)))
    return mask


# ---------------------------------------------------------------- a7
def fit_homography(corner_xy, match_xy, mask, w: int, h: int, H_prev, stream=None):
    """-> (H [9] float64 device, status [1] int32 device)"""
    import torch
    n = corner_xy.shape[0]
    H = _empty((9,), torch.float64, H_prev)
    st = _empty((1,), torch.int32, H_prev)
    _check(lib().hdrreg_fit_homography(_ptr(corner_xy), _ptr(match_xy), _ptr(mask), n, w, h,
                                       _ptr(H_prev), _ptr(H), _ptr(st), _stream(stream)))
    return H, st


# ---------------------------------------------------------- a6 + a7
def weed_fit(corner_xy, match_xy, valid, w: int, h: int, p: Params, seed: int, H_prev,
             iter_begin=0, iter_end=None, counter=None, stream=None):
    """Weeding and level fit of one level in one launch -> (mask, H, status)"""
    import torch
    n = valid.numel()
    if iter_end is None:
        iter_end = p.weed_iters
    mask = torch.empty((n // 32 + 1,), dtype=torch.int32, device=valid.device)
    H = _empty((9,), torch.float64, H_prev)
    st = _empty((1,), torch.int32, H_prev)
    if counter is None:
        counter = torch.zeros((1,), dtype=torch.int32, device=valid.device)
    _check(lib().hdrreg_weed_fit(_ptr(corner_xy), _ptr(match_xy), _ptr(valid), n, w, h,
                                 C.byref(p), C.c_uint64(seed), iter_begin, iter_end, _ptr(mask),
                                 _ptr(H_prev), _ptr(H), _ptr(st), _ptr(counter),
                                 _stream(stream)))
    return mask, H, st


# ---------------------------------------------------------------- a8
def flow_upsample(guide_n, corner_xy, match_xy, mask, H, p: Params, stream=None):
    import torch
    h, w = guide_n.shape
    n = corner_xy.shape[0]
    fu = _empty((h, w), torch.float32, guide_n)
    fv = _empty((h, w), torch.float32, guide_n)
    ws_n = lib().hdrreg_flow_workspace_size(w, h)
    ws = _empty((ws_n,), torch.uint8, guide_n)
    _check(lib().hdrreg_flow_upsample(_ptr(guide_n), w, h, _ptr(corner_xy), _ptr(match_xy),
                                      _ptr(mask), n, _ptr(H), C.byref(p), _ptr(fu), _ptr(fv),
                                      _ptr(ws), ws_n, _stream(stream)))
    return fu, fv


# ---------------------------------------------------------------- a9
def warp(src_y, src_u, src_v, H, flow_u, flow_v, stream=None, want_clip=False):
    """-> (y, u, v) FP32 planes, and with want_clip the uint8 clip flags of the luma samples"""
    import torch
    h, w = src_y.shape
    oy = _empty((h, w), torch.float32, src_y)
    clip = _empty((h, w), torch.uint8, src_y) if want_clip else None
    chroma = src_u is not None
    ou = _empty((h // 2, w // 2), torch.float32, src_y) if chroma else None
    ov = _empty((h // 2, w // 2), torch.float32, src_y) if chroma else None
    f = Frame(_ptr(src_y), _ptr(src_u), _ptr(src_v))
    o = PlanesF32(_ptr(oy), _ptr(ou), _ptr(ov))
    _check(lib().hdrreg_warp(C.byref(f), w, h, _ptr(H), _ptr(flow_u), _ptr(flow_v), C.byref(o),
                             _ptr(clip), _stream(stream)))
    return (oy, ou, ov, clip) if want_clip else (oy, ou, ov)


# ---------------------------------------------------------------- a10-a11
def merge(ref_y, ref_u, ref_v, sources: Sequence[Dict], p: Params, want_q=False, stream=None):
    """sources: dicts with y, u, v (warped FP32), ref_n (u8), ratio (num, den), lut (HISTEQ),
    clip (optional uint8 clip flags of the warped luma, as warp(want_clip=True) returns)."""
    import torch
    h, w = ref_y.shape
    chroma = ref_u is not None
    k = len(sources)
    arr = (MergeSrc * k)()
    for i, s in enumerate(sources):
        arr[i] = MergeSrc(_ptr(s["y"]), _ptr(s.get("u")), _ptr(s.get("v")), _ptr(s["ref_n"]),
                          _ptr(s.get("lut")), s["ratio"][0], s["ratio"][1], _ptr(s.get("clip")))
    oy = _empty((h, w), torch.float32, ref_y)
    ou = _empty((h // 2, w // 2), torch.float32, ref_y) if chroma else None
    ov = _empty((h // 2, w // 2), torch.float32, ref_y) if chroma else None
    q = _empty((k, h, w), torch.float32, ref_y) if want_q else None
    f = Frame(_ptr(ref_y), _ptr(ref_u), _ptr(ref_v))
    o = PlanesF32(_ptr(oy), _ptr(ou), _ptr(ov))
    _check(lib().hdrreg_merge(C.byref(f), w, h, k, arr, C.byref(p), C.byref(o), _ptr(q),
                              _stream(stream)))
    return oy, ou, ov, q


# ---------------------------------------------------------------- f1
def fuse(ref_y, ref_u, ref_v, sources: Sequence[Dict], use_contrast=True, we_sigma=0.2,
         stream=None):
    """Error-tolerant exposure fusion (Sec. 2.5). sources: dicts with y, u, v (warped FP32)
    and q (SSIM map FP32, as merge(want_q=True) returns). -> (Y, U - 128, V - 128) FP32."""
    import torch
    h, w = ref_y.shape
    chroma = ref_u is not None
    k = len(sources)
    arr = (FuseSrc * k)(*[FuseSrc(_ptr(s["y"]), _ptr(s.get("u")), _ptr(s.get("v")), _ptr(s["q"]))
                          for s in sources])
    oy = _empty((h, w), torch.float32, ref_y)
    ou = _empty((h // 2, w // 2), torch.float32, ref_y) if chroma else None
    ov = _empty((h // 2, w // 2), torch.float32, ref_y) if chroma else None
    n = lib().hdrreg_fuse_workspace_size(w, h, k, int(chroma))
    ws = _empty((max(n, 1),), torch.uint8, ref_y)
    f = Frame(_ptr(ref_y), _ptr(ref_u), _ptr(ref_v))
    o = PlanesF32(_ptr(oy), _ptr(ou), _ptr(ov))
    _check(lib().hdrreg_fuse(C.byref(f), w, h, k, arr, int(use_contrast), C.c_double(we_sigma),
                             C.byref(o), _ptr(ws), n, _stream(stream)))
    return oy, ou, ov


# ---------------------------------------------------------------- fused
def register_merge_workspace_size(w: int, h: int, nsrc: int, p: Params) -> int:
    return lib().hdrreg_register_merge_workspace_size(w, h, nsrc, C.byref(p))


class RegisterMerge:
    """Reusable fused call for one stack shape: owns the workspace and output planes."""

    def __init__(self, w: int, h: int, nsrc: int, p: Params, chroma: bool, device="cuda"):
        import torch
        self.w, self.h, self.nsrc, self.p, self.chroma = w, h, nsrc, p, chroma
        n = register_merge_workspace_size(w, h, nsrc, p)
        if n == 0:
            raise HdrregError(1, "bad shape or parameters for register_merge")
        self.ws = torch.empty((n,), dtype=torch.uint8, device=device)
        self.out_y = torch.empty((h, w), dtype=torch.float32, device=device)
        self.out_u = torch.empty((h // 2, w // 2), dtype=torch.float32, device=device) if chroma else None
        self.out_v = torch.empty((h // 2, w // 2), dtype=torch.float32, device=device) if chroma else None
        self.diag = torch.zeros((nsrc, C.sizeof(Diag)), dtype=torch.uint8, device=device)

    def __call__(self, ref, srcs, ratios, stream=None):
        """ref, srcs[k]: (y, u, v) uint8 CUDA tensors (u = v = None for luma-only)."""
        k = len(srcs)
        if k != self.nsrc:
            raise ValueError("number of sources differs from the one this call was built for")
        fr = Frame(_ptr(ref[0]), _ptr(ref[1]) if self.chroma else None,
                   _ptr(ref[2]) if self.chroma else None)
        fs = (Frame * k)(*[Frame(_ptr(s[0]), _ptr(s[1]) if self.chroma else None,
                                 _ptr(s[2]) if self.chroma else None) for s in srcs])
        num = (C.c_int * k)(*[r[0] for r in ratios])
        den = (C.c_int * k)(*[r[1] for r in ratios])
        o = PlanesF32(_ptr(self.out_y), _ptr(self.out_u), _ptr(self.out_v))
        _check(lib().hdrreg_register_merge(C.byref(fr), self.w, self.h, k, fs, num, den,
                                           C.byref(self.p), _ptr(self.ws), self.ws.numel(),
                                           C.byref(o), _ptr(self.diag), _stream(stream)))
        return self.out_y, self.out_u, self.out_v

    def diagnostics(self) -> List[Diag]:
        raw = self.diag.cpu().numpy().tobytes()
        n = C.sizeof(Diag)
        return [Diag.from_buffer_copy(raw[i * n:(i + 1) * n]) for i in range(self.nsrc)]


def gemm_bf16(A, B, stream=None):
    """C = A @ B.T for bf16 CUDA matrices A [M, K], B [N, K] (row-major) -> FP32 [M, N]."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    st = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().hdrreg_gemm_bf16(_ptr(A), A.stride(0), _ptr(B), B.stride(0), M, N, K, _ptr(C),
                                  N, _ptr(st), _stream(stream)))
    return C, st


class Predictor:
    """The learned tile-displacement network on the GPU: FP32 parameters, Adam state and a
    workspace for one batch shape (n, h, w) of quarter-resolution inputs."""

    def __init__(self, n: int, h: int, w: int, theta=None, device="cuda"):
        import torch
        self.n, self.h, self.w = n, h, w
        ho, wo = C.c_int(), C.c_int()
        if lib().hdrreg_cnn_out_dims(h, w, C.byref(ho), C.byref(wo)):
            raise HdrregError(1, "bad predictor input size")
        self.ho, self.wo = ho.value, wo.value
        nb = lib().hdrreg_cnn_workspace_size(n, h, w)
        if nb == 0:
            raise HdrregError(1, "bad predictor batch")
        self.ws = torch.empty((nb,), dtype=torch.uint8, device=device)
        self.theta = (torch.zeros(CNN_PARAMS, dtype=torch.float32, device=device) if theta is None
                      else torch.as_tensor(theta, dtype=torch.float32).to(device).contiguous())
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.grad = torch.zeros_like(self.theta)
        self.out = torch.zeros((n, self.ho, self.wo, 2), dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.t = 0
        self._infer_ws = None

    def forward(self, x, stream=None):
        """x: bfloat16 [n, h, w, 2] CUDA tensor -> out FP32 [n, ho, wo, 2]."""
        _check(lib().hdrreg_cnn_forward(_ptr(self.theta), _ptr(x), self.n, self.h, self.w,
                                        _ptr(self.out), _ptr(self.ws), self.ws.numel(),
                                        _ptr(self.status), _stream(stream)))
        return self.out

    def infer(self, x, stream=None):
        """Inference form (implicit-GEMM convolutions, no stored intermediates): x bfloat16
        [n, h, w, 2] -> a new FP32 [n, ho, wo, 2]."""
        import torch
        if self._infer_ws is None:
            nb = lib().hdrreg_cnn_infer_workspace_size(self.n, self.h, self.w)
            self._infer_ws = torch.empty((nb,), dtype=torch.uint8, device=self.theta.device)
        out = torch.zeros_like(self.out)
        _check(lib().hdrreg_cnn_infer(_ptr(self.theta), _ptr(x), self.n, self.h, self.w,
                                      _ptr(out), _ptr(self._infer_ws), self._infer_ws.numel(),
                                      _ptr(self.status), _stream(stream)))
        return out

    def backward(self, x, label, valid, stream=None):
        _check(lib().hdrreg_cnn_backward(_ptr(self.theta), _ptr(x), self.n, self.h, self.w,
                                         _ptr(self.out), _ptr(label), _ptr(valid), _ptr(self.grad),
                                         _ptr(self.loss), _ptr(self.ws), self.ws.numel(),
                                         _ptr(self.status), _stream(stream)))
        return self.loss, self.grad

    def activation(self, layer: int):
        """Copy of what the last forward stored for `layer` (-1 = features) as FP32 [rows, cols]."""
        import torch
        ptr, rows, cols = C.c_void_p(), C.c_int(), C.c_int()
        _check(lib().hdrreg_cnn_activation(_ptr(self.ws), self.n, self.h, self.w, layer,
                                           C.byref(ptr), C.byref(rows), C.byref(cols)))
        off = ptr.value - self.ws.data_ptr()
        nb = rows.value * cols.value * 2
        return self.ws[off:off + nb].view(torch.bfloat16).float().reshape(rows.value, cols.value)

    def adam(self, lr=1e-3, stream=None):
        self.t += 1
        _check(lib().hdrreg_cnn_adam(_ptr(self.theta), _ptr(self.m), _ptr(self.v), _ptr(self.grad),
                                     self.t, C.c_float(lr), _stream(stream)))


def predictor_input(ref_q, src_q, H, stream=None):
    """Network input (bfloat16 [h, w, 2]) from quarter-resolution reference and source levels."""
    import torch
    h, w = ref_q.shape
    x = torch.empty((h, w, 2), dtype=torch.bfloat16, device=ref_q.device)
    _check(lib().hdrreg_predictor_input(_ptr(ref_q), _ptr(src_q), w, h, _ptr(H), _ptr(x),
                                        _stream(stream)))
    return x


def tile_labels(corner_xy, match_xy, valid, w: int, h: int, H, stream=None):
    import torch
    n = valid.numel()
    lab = torch.empty((n, 2), dtype=torch.float32, device=valid.device)
    _check(lib().hdrreg_tile_labels(_ptr(corner_xy), _ptr(match_xy), _ptr(valid), n, w, h, _ptr(H),
                                    _ptr(lab), _stream(stream)))
    return lab


def predictor_crops(x_full, label_full, valid_full, ntx: int, nty: int, origins, crop_tiles=8,
                    label_bound=1e30, stream=None):
    """Gather training crops (origins: int32 [n, 4] CUDA tensor of tile x, tile y, symmetry,
    unused) -> (x, label, valid)."""
    import torch
    hq, wq = x_full.shape[0], x_full.shape[1]
    n = origins.shape[0]
    side = 8 * crop_tiles
    x = torch.empty((n, side, side, 2), dtype=torch.bfloat16, device=x_full.device)
    lab = torch.empty((n, crop_tiles, crop_tiles, 2), dtype=torch.float32, device=x_full.device)
    val = torch.empty((n, crop_tiles, crop_tiles), dtype=torch.uint8, device=x_full.device)
    _check(lib().hdrreg_predictor_crops(_ptr(x_full), wq, hq, _ptr(label_full), _ptr(valid_full),
                                        ntx, nty, _ptr(origins), n, crop_tiles,
                                        C.c_float(label_bound), _ptr(x), _ptr(lab), _ptr(val),
                                        _stream(stream)))
    return x, lab, val


def local_search_predicted(ref_n, src_n, H, p: Params, pred, fallback_cost: int, refine=0,
                           stream=None):
    """pred: FP32 [rows, cols, 2] with cols >= tiles across -> (corner, match, cost, valid,
    fell_back)."""
    import torch
    h, w = ref_n.shape
    n = num_tiles(w, h, p.tile)
    dev = ref_n.device
    corner = torch.empty((max(n, 1), 2), dtype=torch.int32, device=dev)
    match = torch.empty((max(n, 1), 2), dtype=torch.int32, device=dev)
    cost = torch.empty((max(n, 1),), dtype=torch.int32, device=dev)
    valid = torch.empty((max(n, 1),), dtype=torch.uint8, device=dev)
    fb = torch.empty((max(n, 1),), dtype=torch.uint8, device=dev)
    _check(lib().hdrreg_local_search_predicted(_ptr(ref_n), _ptr(src_n), w, h, _ptr(H), C.byref(p),
                                               _ptr(pred), pred.shape[0], pred.shape[1], refine,
                                               C.c_uint32(fallback_cost),
                                               _ptr(corner), _ptr(match), _ptr(cost), _ptr(valid),
                                               _ptr(fb), _stream(stream)))
    return corner[:n], match[:n], cost[:n], valid[:n], fb[:n]


class RegisterMergeBatch:
    """Batched fused call for stacks of one shape on `lanes` concurrent lanes: owns the
    lane workspaces and one set of output planes per stack slot."""

    def __init__(self, w: int, h: int, nsrc: int, p: Params, chroma: bool, slots: int,
                 lanes: int = 4, device="cuda"):
        import torch
        self.w, self.h, self.nsrc, self.p, self.chroma = w, h, nsrc, p, chroma
        self.lanes = lanes
        n = lib().hdrreg_register_merge_batch_workspace_size(w, h, nsrc, lanes, C.byref(p))
        if n == 0:
            raise HdrregError(1, "bad shape, lanes or parameters for register_merge_batch")
        self.ws = torch.empty((n,), dtype=torch.uint8, device=device)

        def plane(hh, ww):
            return torch.empty((hh, ww), dtype=torch.float32, device=device)
        self.outs = [(plane(h, w), plane(h // 2, w // 2) if chroma else None,
                      plane(h // 2, w // 2) if chroma else None) for _ in range(slots)]
        self.diag = torch.zeros((slots, nsrc, C.sizeof(Diag)), dtype=torch.uint8, device=device)
        self._keep = None

    def __call__(self, stacks, stream=None):
        """stacks: list of (ref, srcs, ratios) as for RegisterMerge; -> list of planes."""
        k = len(stacks)
        if k > len(self.outs):
            raise ValueError("more stacks than output slots")
        arr = (Stack * max(k, 1))()
        keep = []
        for i, (ref, srcs, ratios) in enumerate(stacks):
            if len(srcs) != self.nsrc:
                raise ValueError("number of sources differs from the one this call was built for")
            fr = Frame(_ptr(ref[0]), _ptr(ref[1]) if self.chroma else None,
                       _ptr(ref[2]) if self.chroma else None)
            fs = (Frame * self.nsrc)(*[Frame(_ptr(s[0]), _ptr(s[1]) if self.chroma else None,
                                             _ptr(s[2]) if self.chroma else None) for s in srcs])
            num = (C.c_int * self.nsrc)(*[r[0] for r in ratios])
            den = (C.c_int * self.nsrc)(*[r[1] for r in ratios])
            o = self.outs[i]
            arr[i].ref = C.pointer(fr)
            arr[i].srcs = C.cast(fs, C.POINTER(Frame))
            arr[i].ratio_num = C.cast(num, C.POINTER(C.c_int))
            arr[i].ratio_den = C.cast(den, C.POINTER(C.c_int))
            arr[i].out = PlanesF32(_ptr(o[0]), _ptr(o[1]), _ptr(o[2]))
            arr[i].diag = _ptr(self.diag[i])
            keep.append((fr, fs, num, den))
        _check(lib().hdrreg_register_merge_batch(arr, k, self.w, self.h, self.nsrc, self.lanes,
                                                 C.byref(self.p), _ptr(self.ws),
                                                 self.ws.numel(), _stream(stream)))
        self._keep = keep
        return self.outs[:k]

    def diagnostics(self, slot: int) -> List[Diag]:
        raw = self.diag[slot].cpu().numpy().tobytes()
        n = C.sizeof(Diag)
        return [Diag.from_buffer_copy(raw[i * n:(i + 1) * n]) for i in range(self.nsrc)]


class RegisterMergeHost:
    """Batched fused call for stacks of one shape held in (page-locked) host memory: the
    library stages each stack through its lane's device buffers. The caller passes host
    uint8 planes and receives the merged FP32 planes in host arrays it provides."""

    def __init__(self, w: int, h: int, nsrc: int, p: Params, lanes: int = 4, device="cuda"):
        import torch
        self.w, self.h, self.nsrc, self.p, self.lanes = w, h, nsrc, p, lanes
        n = lib().hdrreg_register_merge_host_workspace_size(w, h, nsrc, lanes, C.byref(p))
        if n == 0:
            raise HdrregError(1, "bad shape, lanes or parameters for register_merge_host")
        self.ws = torch.empty((n,), dtype=torch.uint8, device=device)
        self._keep = None

    def __call__(self, stacks, outs, stream=None):
        """stacks: (ref, srcs, ratios) with CPU uint8 tensors (y, u, v) (u = v = None for
        luma); outs: one (y, u, v) of CPU FP32 tensors per stack. Enqueues only: the outputs
        are valid after the stream is synchronized."""
        k = len(stacks)
        arr = (Stack * max(k, 1))()
        keep = []

        def hp(t):
            if t is None:
                return None
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("host planes must be contiguous CPU tensors")
            return t.data_ptr()
        for i, (ref, srcs, ratios) in enumerate(stacks):
            if len(srcs) != self.nsrc:
                raise ValueError("number of sources differs from the one this call was built for")
            fr = Frame(hp(ref[0]), hp(ref[1]), hp(ref[2]))
            fs = (Frame * self.nsrc)(*[Frame(hp(s[0]), hp(s[1]), hp(s[2])) for s in srcs])
            num = (C.c_int * self.nsrc)(*[r[0] for r in ratios])
            den = (C.c_int * self.nsrc)(*[r[1] for r in ratios])
            arr[i].ref = C.pointer(fr)
            arr[i].srcs = C.cast(fs, C.POINTER(Frame))
            arr[i].ratio_num = C.cast(num, C.POINTER(C.c_int))
            arr[i].ratio_den = C.cast(den, C.POINTER(C.c_int))
            o = outs[i]
            arr[i].out = PlanesF32(hp(o[0]), hp(o[1]), hp(o[2]))
            arr[i].diag = None
            keep.append((fr, fs, num, den))
        _check(lib().hdrreg_register_merge_host(arr, k, self.w, self.h, self.nsrc, self.lanes,
                                                C.byref(self.p), _ptr(self.ws), self.ws.numel(),
                                                _stream(stream)))
        self._keep = keep


class RegisterMergeMulti:
    """Batched fused call for stacks of different sizes, source counts and parameters on
    `lanes` concurrent lanes. `shapes` lists (w, h, nsrc, params, chroma) per stack slot;
    the object owns the workspace and each slot's output planes and diagnostics."""

    def __init__(self, shapes, lanes: int = 4, device="cuda", staged: bool = False):
        """staged: run the merges of all stacks as one stage after every registration
        (hdrreg_register_merge_staged) instead of each on its stack's lane."""
        import torch
        self.shapes = [(int(w), int(h), int(n), p, bool(c)) for w, h, n, p, c in shapes]
        self.lanes = lanes
        self.staged = staged
        self._params = [C.pointer(p) for _, _, _, p, _ in self.shapes]
        arr = self._array(len(self.shapes))
        size_fn = (lib().hdrreg_register_merge_staged_workspace_size if staged else
                   lib().hdrreg_register_merge_multi_workspace_size)
        n = size_fn(arr, len(self.shapes), lanes)
        if n == 0:
            raise HdrregError(1, "bad shape, lanes or parameters for register_merge_multi")
        self.ws = torch.empty((n,), dtype=torch.uint8, device=device)

        def plane(hh, ww):
            return torch.empty((hh, ww), dtype=torch.float32, device=device)
        self.outs = [(plane(h, w), plane(h // 2, w // 2) if c else None,
                      plane(h // 2, w // 2) if c else None) for w, h, _, _, c in self.shapes]
        self.diag = [torch.zeros((n, C.sizeof(Diag)), dtype=torch.uint8, device=device)
                     for _, _, n, _, _ in self.shapes]
        self._keep = None

    def _array(self, k):
        arr = (StackEx * max(k, 1))()
        for i in range(k):
            w, h, n, _, _ = self.shapes[i]
            arr[i].w, arr[i].h, arr[i].nsrc = w, h, n
            arr[i].p = self._params[i]
        return arr

    def __call__(self, stacks, stream=None):
        """stacks: one (ref, srcs, ratios) per slot, shaped as that slot was declared;
        -> the list of output planes."""
        k = len(stacks)
        if k != len(self.shapes):
            raise ValueError("one stack per declared slot is required")
        arr = self._array(k)
        keep = []
        for i, (ref, srcs, ratios) in enumerate(stacks):
            w, h, n, _, chroma = self.shapes[i]
            if len(srcs) != n or tuple(ref[0].shape) != (h, w):
                raise ValueError(f"stack {i} differs from its declared shape")
            fr = Frame(_ptr(ref[0]), _ptr(ref[1]) if chroma else None,
                       _ptr(ref[2]) if chroma else None)
            fs = (Frame * n)(*[Frame(_ptr(s[0]), _ptr(s[1]) if chroma else None,
                                     _ptr(s[2]) if chroma else None) for s in srcs])
            num = (C.c_int * n)(*[r[0] for r in ratios])
            den = (C.c_int * n)(*[r[1] for r in ratios])
            o = self.outs[i]
            arr[i].s.ref = C.pointer(fr)
            arr[i].s.srcs = C.cast(fs, C.POINTER(Frame))
            arr[i].s.ratio_num = C.cast(num, C.POINTER(C.c_int))
            arr[i].s.ratio_den = C.cast(den, C.POINTER(C.c_int))
            arr[i].s.out = PlanesF32(_ptr(o[0]), _ptr(o[1]), _ptr(o[2]))
            arr[i].s.diag = _ptr(self.diag[i])
            keep.append((fr, fs, num, den))
        fn = lib().hdrreg_register_merge_staged if self.staged else lib().hdrreg_register_merge_multi
        _check(fn(arr, k, self.lanes, _ptr(self.ws), self.ws.numel(), _stream(stream)))
        self._keep = keep
        return self.outs

    def diagnostics(self, slot: int) -> List[Diag]:
        raw = self.diag[slot].cpu().numpy().tobytes()
        n = C.sizeof(Diag)
        return [Diag.from_buffer_copy(raw[i * n:(i + 1) * n])
                for i in range(self.shapes[slot][2])]


def register_merge(ref, srcs, ratios, p: Params, stream=None):
    h, w = ref[0].shape
    rm = RegisterMerge(w, h, len(srcs), p, ref[1] is not None, device=ref[0].device)
    out = rm(ref, srcs, ratios, stream)
    return out, rm
