"""ctypes binding of the C ABI in ``include/pt.h`` (argument marshalling only).

Functions keep the C names (``pt_scene_create``, ``pt_bvh_build``,
``pt_render_forward``, ``pt_render_backward``, ...).  Device buffers are torch
CUDA tensors; only their raw pointers cross the boundary.  Every step of the
rendering runs in the CUDA library: if ``libptgb.so`` is missing this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import scenes as S

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libptgb.so")

PT_OK = 0
PT_ERR_ARG = -1
PT_ERR_CUDA = -2
PT_ERR_OOM = -3
PT_ERR_TIMEOUT = -4
PT_ERR_BVH = -5
PT_ERR_STATE = -6
PT_MAX_TEX = 8
PT_MAX_CAMS = 64
PT_BVH_BINARY = 0
PT_BVH_WIDE = 1
PT_DISPATCH_SWITCH = 0
PT_DISPATCH_MATCH = 1
PT_PRB_AUTO = 0
PT_PRB_FUSED = 1
PT_PRB_SPLIT = 2
PT_SCHED_AUTO = 0
PT_SCHED_PERSISTENT = 1
PT_SCHED_STATIC = 2
PT_WF_TRACED = 0
PT_WF_GROUPED = 1
PT_N_COUNTERS = 16
COUNTER_NAMES = ["paths", "rays", "shadow_rays", "nodes", "tri_tests", "tex_lookups", "atomics", "grad_terms"]


class PtError(RuntimeError):
    def __init__(self, fn, code):
        msg = _lib.pt_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{fn} failed: {code} ({msg})")
        self.code = code


class pt_shape(C.Structure):
    _fields_ = [("bsdf", C.c_int32), ("tex", C.c_int32), ("albedo_index", C.c_int32), ("rough_index", C.c_int32),
                ("alpha", C.c_float), ("eta", C.c_float), ("diffuse_weight", C.c_float),
                ("f0", C.c_float * 3), ("emission", C.c_float * 3)]


class pt_scene_desc(C.Structure):
    _fields_ = [("n_tris", C.c_int32), ("vertices", C.c_void_p), ("uvs", C.c_void_p), ("tri_shape", C.c_void_p),
                ("n_shapes", C.c_int32), ("shapes", C.c_void_p), ("env_w", C.c_int32), ("env_h", C.c_int32),
                ("env", C.c_void_p)]


class pt_bvh_opts(C.Structure):
    _fields_ = [("layout", C.c_int32), ("max_leaf_tris", C.c_int32), ("n_bins", C.c_int32)]


class pt_scene_info(C.Structure):
    _fields_ = [("n_tris", C.c_int64), ("n_nodes", C.c_int64), ("node_bytes", C.c_int64), ("tri_bytes", C.c_int64),
                ("env_bytes", C.c_int64), ("layout", C.c_int32), ("depth", C.c_int32), ("sah_cost", C.c_double)]


class pt_camera(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3), ("vfov_deg", C.c_float)]


class pt_render_desc(C.Structure):
    _fields_ = [("n_cams", C.c_int32), ("cams", C.c_void_p), ("width", C.c_int32), ("height", C.c_int32),
                ("spp", C.c_int32), ("max_depth", C.c_int32), ("rr_depth", C.c_int32), ("nee", C.c_int32),
                ("seed", C.c_uint64), ("dispatch", C.c_int32),
                ("crop_x0", C.c_int32), ("crop_y0", C.c_int32), ("crop_w", C.c_int32), ("crop_h", C.c_int32),
                ("lanes_per_pixel", C.c_int32), ("block_size", C.c_int32), ("tex_aggregate", C.c_int32),
                ("dbg_sample_L", C.c_void_p), ("dbg_sample_hash", C.c_void_p), ("counters", C.c_void_p),
                ("cache", C.c_void_p), ("cache_bounce", C.c_int32), ("prb_mode", C.c_int32),
                ("schedule", C.c_int32)]


class pt_params(C.Structure):
    _fields_ = [("albedo", C.c_void_p), ("n_albedo", C.c_int32), ("tex", C.c_void_p * PT_MAX_TEX),
                ("tex_w", C.c_int32 * PT_MAX_TEX), ("tex_h", C.c_int32 * PT_MAX_TEX), ("n_tex", C.c_int32),
                ("roughness", C.c_void_p), ("n_rough", C.c_int32), ("env", C.c_void_p)]


class pt_grads(C.Structure):
    _fields_ = [("albedo", C.c_void_p), ("tex", C.c_void_p * PT_MAX_TEX), ("roughness", C.c_void_p),
                ("env", C.c_void_p)]


PT_CACHE_N_PARAMS = 20672


class pt_cache_desc(C.Structure):
    _fields_ = [("box_lo", C.c_float * 3), ("box_hi", C.c_float * 3), ("batch", C.c_int32),
                ("max_queries", C.c_int32), ("max_records", C.c_int32), ("max_paths", C.c_int32),
                ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("init_weights", C.c_void_p), ("seed", C.c_uint64), ("ema", C.c_float)]


class pt_job(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("camera", pt_camera), ("width", C.c_int32), ("height", C.c_int32),
                ("spp", C.c_int32), ("max_depth", C.c_int32), ("rr_depth", C.c_int32), ("nee", C.c_int32),
                ("seed", C.c_uint64), ("backward_seed", C.c_uint64), ("params", pt_params), ("grads", pt_grads),
                ("image", C.c_void_p), ("target", C.c_void_p)]


class pt_batch_opts(C.Structure):
    _fields_ = [("tile", C.c_int32), ("lanes_per_pixel", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("block_size", C.c_int32)]


class pt_wavefront_opts(C.Structure):
    _fields_ = [("calls", C.c_int32), ("wave_paths", C.c_int32)]


class pt_reparam_opts(C.Structure):
    _fields_ = [("n_aux", C.c_int32), ("kappa", C.c_float), ("kernel_scale", C.c_float), ("power", C.c_float),
                ("miss", C.c_float), ("eps", C.c_float), ("border", C.c_float), ("jackknife", C.c_int32),
                ("edge_spp", C.c_int32)]


_lib = None
_lock = threading.Lock()

# exported symbols with their argument/return types
SIGNATURES = {
    "pt_scene_create": ([C.POINTER(pt_scene_desc), C.POINTER(C.c_void_p)], C.c_int),
    "pt_scene_destroy": ([C.c_void_p], None),
    "pt_bvh_build": ([C.c_void_p, C.POINTER(pt_bvh_opts)], C.c_int),
    "pt_scene_get_info": ([C.c_void_p, C.POINTER(pt_scene_info)], C.c_int),
    "pt_render_forward": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params), C.c_void_p, C.c_void_p],
                          C.c_int),
    "pt_render_backward": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params), C.c_void_p,
                            C.POINTER(pt_grads), C.c_void_p], C.c_int),
    "pt_render_jvp": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params), C.POINTER(pt_params),
                       C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "pt_wavefront_forward": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params),
                              C.POINTER(pt_wavefront_opts), C.c_void_p, C.c_void_p], C.c_int),
    "pt_wavefront_backward": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params),
                               C.POINTER(pt_wavefront_opts), C.c_void_p, C.POINTER(pt_grads), C.c_void_p], C.c_int),
    "pt_ckpt_create": ([C.c_int64, C.c_int32, C.POINTER(C.c_void_p)], C.c_int),
    "pt_ckpt_destroy": ([C.c_void_p], None),
    "pt_ckpt_bytes": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "pt_ckpt_forward": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params), C.c_void_p, C.c_void_p,
                         C.c_void_p], C.c_int),
    "pt_ckpt_backward": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params), C.c_void_p, C.c_void_p,
                          C.POINTER(pt_grads), C.c_void_p], C.c_int),
    "pt_reparam_defaults": ([C.POINTER(pt_reparam_opts)], None),
    "pt_render_backward_reparam": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params),
                                    C.POINTER(pt_reparam_opts), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
                                   C.c_int),
    "pt_render_backward_reparam_vertices": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params),
                                             C.POINTER(pt_reparam_opts), C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p], C.c_int),
    "pt_render_jvp_reparam": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params),
                               C.POINTER(pt_reparam_opts), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p], C.c_int),
    "pt_render_jvp_reparam_vertices": ([C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params),
                                        C.POINTER(pt_reparam_opts), C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p], C.c_int),
    "pt_last_device_status": ([C.c_void_p, C.c_void_p, C.POINTER(C.c_int)], C.c_int),
    "pt_status_string": ([C.c_int], C.c_char_p),
    "pt_cache_create": ([C.POINTER(pt_cache_desc), C.POINTER(C.c_void_p)], C.c_int),
    "pt_cache_destroy": ([C.c_void_p], None),
    "pt_cache_set_engine": ([C.c_void_p, C.c_int], C.c_int),
    "pt_cache_status": ([C.c_void_p, C.c_void_p, C.POINTER(C.c_int)], C.c_int),
    "pt_cache_set_wait_limit": ([C.c_void_p, C.c_uint32], C.c_int),
    "pt_cache_get_state": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)], C.c_int),
    "pt_cache_set_state": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32], C.c_int),
    "pt_cache_get_weights": ([C.c_void_p, C.c_void_p], C.c_int),
    "pt_cache_get_average": ([C.c_void_p, C.c_void_p], C.c_int),
    "pt_cache_set_average": ([C.c_void_p, C.c_void_p], C.c_int),
    "pt_cache_set_weights": ([C.c_void_p, C.c_void_p], C.c_int),
    "pt_cache_query": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "pt_cache_encode": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "pt_trace_rays": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                       C.c_void_p], C.c_int),
    "pt_cache_train_records": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p], C.c_int),
    "pt_cache_last_loss": ([C.c_void_p, C.c_void_p, C.POINTER(C.c_float)], C.c_int),
    "pt_cache_train": ([C.c_void_p, C.c_void_p, C.POINTER(pt_render_desc), C.POINTER(pt_params), C.c_int,
                        C.c_void_p, C.POINTER(C.c_int)], C.c_int),
    "pt_batch_create": ([C.c_void_p, C.c_int, C.POINTER(pt_batch_opts), C.POINTER(C.c_void_p)], C.c_int),
    "pt_batch_run": ([C.c_void_p, C.c_void_p], C.c_int),
    "pt_batch_info": ([C.c_void_p, C.POINTER(C.c_int)], C.c_int),
    "pt_batch_destroy": ([C.c_void_p], None),
    "pt_render_batch": ([C.c_void_p, C.c_int, C.POINTER(pt_batch_opts), C.c_void_p], C.c_int),
    "pt_render_batch_noalloc": ([C.c_void_p, C.c_int, C.POINTER(pt_batch_opts), C.c_void_p], C.c_int),
    "pt_probe_read": ([C.c_void_p, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "pt_probe_atomic": ([C.c_void_p, C.c_longlong, C.c_longlong, C.c_int, C.c_void_p], C.c_int),
    "pt_cache_read_records": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)],
                              C.c_int),
}


def load(path: str = LIB_PATH):
    """Load libptgb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with paper_2202_01284_gb300.build.build() "
                                   "(there is no CPU fallback)")
            lib = C.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name, None)
                if fn is None:
                    continue
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def check(fn_name, code):
    if code != PT_OK:
        raise PtError(fn_name, code)


def _ptr(t):
    """Raw device (or host) pointer of a torch tensor / numpy array, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


# ------------------------------------------------------------------ marshalling helpers
def scene_desc(scene: "S.Scene"):
    """Build a pt_scene_desc from a generator Scene; returns (desc, keepalive)."""
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a
    n = scene.n_shapes
    shapes = (pt_shape * n)()
    for i in range(n):
        sh = shapes[i]
        sh.bsdf = int(scene.bsdf[i])
        sh.tex = int(scene.tex[i])
        sh.albedo_index = int(scene.albedo_index[i])
        sh.rough_index = int(scene.rough_index[i])
        sh.alpha = float(scene.alpha[i])
        sh.eta = float(scene.eta[i])
        sh.diffuse_weight = float(scene.diffuse_weight[i])
        sh.f0[:] = [float(x) for x in scene.f0[i]]
        sh.emission[:] = [float(x) for x in scene.emission[i]]
    keep.append(shapes)
    d = pt_scene_desc()
    d.n_tris = scene.n_tris
    d.vertices = _ptr(arr(scene.vertices, np.float32))
    d.uvs = _ptr(arr(scene.uvs, np.float32))
    d.tri_shape = _ptr(arr(scene.tri_shape, np.int32))
    d.n_shapes = n
    d.shapes = C.cast(shapes, C.c_void_p).value
    if scene.env is not None:
        d.env_w, d.env_h = int(scene.env.shape[1]), int(scene.env.shape[0])
        d.env = _ptr(arr(scene.env, np.float32))
    return d, keep


def camera_struct(cam: "S.Camera") -> pt_camera:
    c = pt_camera()
    c.origin[:] = cam.origin
    c.target[:] = cam.target
    c.up[:] = cam.up
    c.vfov_deg = cam.vfov_deg
    return c


def render_desc(cams, width, height, spp, max_depth, seed, rr_depth=-1, nee=True, dispatch=PT_DISPATCH_SWITCH,
                crop=None, lanes_per_pixel=0, block_size=0, tex_aggregate=0, dbg_L=None, dbg_hash=None,
                counters=None, cache=None, cache_bounce=1, prb_mode=0, schedule=0):
    cams = list(cams)
    arr = (pt_camera * len(cams))(*[camera_struct(c) for c in cams])
    r = pt_render_desc()
    r.n_cams = len(cams)
    r.cams = C.cast(arr, C.c_void_p).value
    r.width, r.height, r.spp, r.max_depth = width, height, spp, max_depth
    r.rr_depth, r.nee, r.seed, r.dispatch = rr_depth, int(bool(nee)), seed, dispatch
    if crop is not None:
        r.crop_x0, r.crop_y0, r.crop_w, r.crop_h = crop
    r.lanes_per_pixel, r.block_size, r.tex_aggregate = lanes_per_pixel, block_size, tex_aggregate
    r.dbg_sample_L = _ptr(dbg_L)
    r.dbg_sample_hash = _ptr(dbg_hash)
    r.counters = _ptr(counters)
    r.cache = cache
    r.cache_bounce = cache_bounce
    r.prb_mode = prb_mode
    r.schedule = schedule
    r._keep = arr
    return r


def params_struct(albedo=None, textures=(), roughness=None, env=None) -> pt_params:
    p = pt_params()
    if albedo is not None and albedo.numel() > 0:
        p.albedo = _ptr(albedo)
        p.n_albedo = int(albedo.shape[0])
    for i, t in enumerate(textures):
        p.tex[i] = _ptr(t)
        p.tex_w[i] = int(t.shape[1])
        p.tex_h[i] = int(t.shape[0])
    p.n_tex = len(textures)
    if roughness is not None and roughness.numel() > 0:
        p.roughness = _ptr(roughness)
        p.n_rough = int(roughness.shape[0])
    if env is not None:
        p.env = _ptr(env)
    return p


def grads_struct(albedo=None, textures=(), roughness=None, env=None) -> pt_grads:
    g = pt_grads()
    g.albedo = _ptr(albedo) if albedo is not None and albedo.numel() > 0 else None
    for i, t in enumerate(textures):
        g.tex[i] = _ptr(t)
    g.roughness = _ptr(roughness) if roughness is not None and roughness.numel() > 0 else None
    g.env = _ptr(env) if env is not None else None
    return g


# ------------------------------------------------------------------ C-named entry points
def pt_scene_create(scene: "S.Scene") -> int:
    L = load()
    d, keep = scene_desc(scene)
    h = C.c_void_p()
    check("pt_scene_create", L.pt_scene_create(C.byref(d), C.byref(h)))
    return h.value


def pt_scene_destroy(handle: int) -> None:
    if handle:
        load().pt_scene_destroy(handle)


def pt_bvh_build(handle: int, layout=PT_BVH_BINARY, max_leaf_tris=0, n_bins=0) -> None:
    o = pt_bvh_opts(layout, max_leaf_tris, n_bins)
    check("pt_bvh_build", load().pt_bvh_build(handle, C.byref(o)))


def pt_scene_get_info(handle: int) -> dict:
    i = pt_scene_info()
    check("pt_scene_get_info", load().pt_scene_get_info(handle, C.byref(i)))
    return {k: getattr(i, k) for k, _ in pt_scene_info._fields_}


def pt_render_forward(handle: int, desc: pt_render_desc, params: pt_params, image, stream: int = 0) -> None:
    check("pt_render_forward", load().pt_render_forward(handle, C.byref(desc), C.byref(params), _ptr(image),
                                                        stream or None))


def pt_render_backward(handle: int, desc: pt_render_desc, params: pt_params, grad_image, grads: pt_grads,
                       stream: int = 0) -> None:
    check("pt_render_backward", load().pt_render_backward(handle, C.byref(desc), C.byref(params),
                                                          _ptr(grad_image), C.byref(grads), stream or None))


def pt_render_jvp(handle: int, desc: pt_render_desc, params: pt_params, tangent: pt_params, image, image_dot,
                  stream: int = 0) -> None:
    check("pt_render_jvp", load().pt_render_jvp(handle, C.byref(desc), C.byref(params), C.byref(tangent),
                                                _ptr(image), _ptr(image_dot), stream or None))


def pt_wavefront_forward(handle: int, desc: pt_render_desc, params: pt_params, opts: pt_wavefront_opts, image,
                         stream: int = 0) -> None:
    check("pt_wavefront_forward", load().pt_wavefront_forward(handle, C.byref(desc), C.byref(params), C.byref(opts),
                                                              _ptr(image), stream or None))


def pt_wavefront_backward(handle: int, desc: pt_render_desc, params: pt_params, opts: pt_wavefront_opts, grad_image,
                          grads: pt_grads, stream: int = 0) -> None:
    check("pt_wavefront_backward", load().pt_wavefront_backward(handle, C.byref(desc), C.byref(params),
                                                                C.byref(opts), _ptr(grad_image), C.byref(grads),
                                                                stream or None))


def pt_ckpt_create(max_samples: int, max_depth: int) -> int:
    h = C.c_void_p()
    check("pt_ckpt_create", load().pt_ckpt_create(max_samples, max_depth, C.byref(h)))
    return h.value


def pt_ckpt_destroy(handle: int) -> None:
    load().pt_ckpt_destroy(handle)


def pt_ckpt_bytes(handle: int) -> int:
    v = C.c_int64(0)
    check("pt_ckpt_bytes", load().pt_ckpt_bytes(handle, C.byref(v)))
    return v.value


def pt_ckpt_forward(handle: int, desc: pt_render_desc, params: pt_params, ckpt: int, image, stream: int = 0) -> None:
    check("pt_ckpt_forward", load().pt_ckpt_forward(handle, C.byref(desc), C.byref(params), ckpt, _ptr(image),
                                                    stream or None))


def pt_ckpt_backward(handle: int, desc: pt_render_desc, params: pt_params, ckpt: int, grad_image, grads: pt_grads,
                     stream: int = 0) -> None:
    check("pt_ckpt_backward", load().pt_ckpt_backward(handle, C.byref(desc), C.byref(params), ckpt,
                                                      _ptr(grad_image), C.byref(grads), stream or None))


def reparam_opts(**kw) -> pt_reparam_opts:
    """pt_reparam_opts with the library's defaults, overridden by keyword."""
    o = pt_reparam_opts()
    load().pt_reparam_defaults(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown reparameterization option {k}")
        setattr(o, k, v)
    return o


def pt_render_backward_reparam(handle: int, desc: pt_render_desc, params: pt_params, opts: pt_reparam_opts,
                               grad_image, grad_translation, rays=None, stream: int = 0) -> None:
    check("pt_render_backward_reparam",
          load().pt_render_backward_reparam(handle, C.byref(desc), C.byref(params), C.byref(opts), _ptr(grad_image),
                                            _ptr(grad_translation), _ptr(rays), stream or None))


def pt_render_backward_reparam_vertices(handle: int, desc: pt_render_desc, params: pt_params, opts: pt_reparam_opts,
                                        grad_image, grad_vertices, rays=None, stream: int = 0) -> None:
    check("pt_render_backward_reparam_vertices",
          load().pt_render_backward_reparam_vertices(handle, C.byref(desc), C.byref(params), C.byref(opts),
                                                     _ptr(grad_image), _ptr(grad_vertices), _ptr(rays),
                                                     stream or None))


def pt_render_jvp_reparam(handle: int, desc: pt_render_desc, params: pt_params, opts: pt_reparam_opts,
                          dir_translation, image, image_dot, rays=None, stream: int = 0) -> None:
    check("pt_render_jvp_reparam",
          load().pt_render_jvp_reparam(handle, C.byref(desc), C.byref(params), C.byref(opts), _ptr(dir_translation),
                                       _ptr(image), _ptr(image_dot), _ptr(rays), stream or None))


def pt_render_jvp_reparam_vertices(handle: int, desc: pt_render_desc, params: pt_params, opts: pt_reparam_opts,
                                   dir_vertices, image, image_dot, rays=None, stream: int = 0) -> None:
    check("pt_render_jvp_reparam_vertices",
          load().pt_render_jvp_reparam_vertices(handle, C.byref(desc), C.byref(params), C.byref(opts),
                                                _ptr(dir_vertices), _ptr(image), _ptr(image_dot), _ptr(rays),
                                                stream or None))


def pt_last_device_status(handle: int, stream: int = 0) -> int:
    v = C.c_int(0)
    check("pt_last_device_status", load().pt_last_device_status(handle, stream or None, C.byref(v)))
    return v.value


# ------------------------------------------------------------------ radiance cache
def pt_cache_create(box_lo, box_hi, batch=65536, max_queries=0, max_records=0, max_paths=0, lr=5e-3,
                    beta1=0.9, beta2=0.99, eps=1e-8, init_weights=None, seed=0, ema=0.0) -> int:
    d = pt_cache_desc()
    d.box_lo[:] = [float(x) for x in box_lo]
    d.box_hi[:] = [float(x) for x in box_hi]
    d.batch, d.max_queries, d.max_records, d.max_paths = batch, max_queries, max_records, max_paths
    d.lr, d.beta1, d.beta2, d.eps = lr, beta1, beta2, eps
    w = None
    if init_weights is not None:
        w = np.ascontiguousarray(init_weights, np.float32)
        assert w.size == PT_CACHE_N_PARAMS
        d.init_weights = w.ctypes.data
    d.seed = seed
    d.ema = ema
    h = C.c_void_p()
    check("pt_cache_create", load().pt_cache_create(C.byref(d), C.byref(h)))
    return h.value


def pt_cache_destroy(handle: int) -> None:
    if handle:
        load().pt_cache_destroy(handle)


def pt_cache_get_weights(handle: int) -> np.ndarray:
    w = np.zeros(PT_CACHE_N_PARAMS, np.float32)
    check("pt_cache_get_weights", load().pt_cache_get_weights(handle, w.ctypes.data))
    return w


def pt_cache_get_average(handle: int) -> np.ndarray:
    w = np.zeros(PT_CACHE_N_PARAMS, np.float32)
    check("pt_cache_get_average", load().pt_cache_get_average(handle, w.ctypes.data))
    return w


def pt_cache_set_average(handle: int, w) -> None:
    w = np.ascontiguousarray(w, np.float32)
    assert w.size == PT_CACHE_N_PARAMS
    check("pt_cache_set_average", load().pt_cache_set_average(handle, w.ctypes.data))


def pt_cache_set_weights(handle: int, w) -> None:
    w = np.ascontiguousarray(w, np.float32)
    assert w.size == PT_CACHE_N_PARAMS
    check("pt_cache_set_weights", load().pt_cache_set_weights(handle, w.ctypes.data))


PT_CACHE_TCGEN05 = 0
PT_CACHE_MMA_SYNC = 1


def pt_cache_set_engine(handle: int, engine: int) -> None:
    check("pt_cache_set_engine", load().pt_cache_set_engine(handle, engine))


PT_CACHE_WAIT_LIMIT_DEFAULT = 1 << 22


def pt_cache_get_state(handle: int):
    """(weights, adam_m, adam_v, step): float32 arrays of PT_CACHE_N_PARAMS and the step."""
    w, m, v = (np.zeros(PT_CACHE_N_PARAMS, np.float32) for _ in range(3))
    step = C.c_int32(0)
    check("pt_cache_get_state", load().pt_cache_get_state(handle, w.ctypes.data, m.ctypes.data, v.ctypes.data,
                                                          C.byref(step)))
    return w, m, v, step.value


def pt_cache_set_state(handle: int, w, m, v, step: int) -> None:
    arrs = [np.ascontiguousarray(x, np.float32) for x in (w, m, v)]
    assert all(a.size == PT_CACHE_N_PARAMS for a in arrs)
    check("pt_cache_set_state", load().pt_cache_set_state(handle, *(a.ctypes.data for a in arrs), int(step)))


def pt_cache_set_wait_limit(handle: int, limit: int) -> None:
    check("pt_cache_set_wait_limit", load().pt_cache_set_wait_limit(handle, limit))


def pt_cache_status(handle: int, stream: int = 0) -> int:
    v = C.c_int(0)
    check("pt_cache_status", load().pt_cache_status(handle, stream or None, C.byref(v)))
    return v.value


def pt_cache_query(handle: int, raw, rgb, n: int, stream: int = 0) -> None:
    check("pt_cache_query", load().pt_cache_query(handle, _ptr(raw), _ptr(rgb), n, stream or None))


def pt_trace_rays(scene: int, rays, n: int, t, prim, tmax=None, uv=None, any_hit: bool = False,
                  stream: int = 0) -> None:
    """rays: device float32 [n][6]; t: float32 [n]; prim: int32 [n]; tmax, uv optional."""
    check("pt_trace_rays", load().pt_trace_rays(scene, _ptr(rays), _ptr(tmax), n, int(bool(any_hit)), _ptr(t),
                                               _ptr(prim), _ptr(uv), stream or None))


def pt_cache_encode(handle: int, raw, features, n: int, stream: int = 0) -> None:
    """features: device int16/uint16 [n][64] receiving the BF16 bits of the encoding."""
    check("pt_cache_encode", load().pt_cache_encode(handle, _ptr(raw), _ptr(features), n, stream or None))


def pt_cache_train_records(handle: int, raw, target, n: int, steps: int, stream: int = 0) -> None:
    check("pt_cache_train_records",
          load().pt_cache_train_records(handle, _ptr(raw), _ptr(target), n, steps, stream or None))


def pt_cache_last_loss(handle: int, stream: int = 0) -> float:
    v = C.c_float(0)
    check("pt_cache_last_loss", load().pt_cache_last_loss(handle, stream or None, C.byref(v)))
    return v.value


def pt_cache_train(cache: int, scene: int, desc: pt_render_desc, params: pt_params, steps: int,
                   stream: int = 0) -> int:
    n = C.c_int(0)
    check("pt_cache_train", load().pt_cache_train(cache, scene, C.byref(desc), C.byref(params), steps,
                                                  stream or None, C.byref(n)))
    return n.value


def pt_cache_read_records(cache: int, cap: int):
    raw = np.zeros((cap, 10), np.float32)
    tgt = np.zeros((cap, 3), np.float32)
    meta = np.zeros((cap, 2), np.int32)
    n = C.c_int(0)
    check("pt_cache_read_records", load().pt_cache_read_records(cache, cap, raw.ctypes.data, tgt.ctypes.data,
                                                                meta.ctypes.data, C.byref(n)))
    return raw[:n.value], tgt[:n.value], meta[:n.value]


# ------------------------------------------------------------------ batching
def pt_batch_create(jobs, opts) -> int:
    arr = (pt_job * len(jobs))(*jobs)
    h = C.c_void_p()
    check("pt_batch_create", load().pt_batch_create(C.cast(arr, C.c_void_p), len(jobs), C.byref(opts), C.byref(h)))
    return h.value


def pt_batch_run(handle: int, stream: int = 0) -> None:
    check("pt_batch_run", load().pt_batch_run(handle, stream or None))


def pt_batch_info(handle: int) -> int:
    n = C.c_int(0)
    check("pt_batch_info", load().pt_batch_info(handle, C.byref(n)))
    return n.value


def pt_batch_destroy(handle: int) -> None:
    if handle:
        load().pt_batch_destroy(handle)


def pt_render_batch(jobs, opts, stream: int = 0) -> None:
    arr = (pt_job * len(jobs))(*jobs)
    check("pt_render_batch", load().pt_render_batch(C.cast(arr, C.c_void_p), len(jobs), C.byref(opts),
                                                    stream or None))


def pt_render_batch_noalloc(jobs, opts, stream: int = 0) -> None:
    """Batched render whose scratch is a static device array (no device allocation)."""
    arr = (pt_job * len(jobs))(*jobs)
    check("pt_render_batch_noalloc", load().pt_render_batch_noalloc(C.cast(arr, C.c_void_p), len(jobs),
                                                                    C.byref(opts), stream or None))


def pt_probe_read(buf, passes: int, sink, stream: int = 0) -> None:
    """L2 / HBM read probe over the device tensor `buf` (sum added into `sink`)."""
    check("pt_probe_read", load().pt_probe_read(_ptr(buf), buf.numel() * buf.element_size(), int(passes),
                                                _ptr(sink), stream or None))


def pt_probe_atomic(dst, n_addr: int, n_updates: int, width: int, stream: int = 0) -> None:
    """Atomic-add probe: n_updates adds of 1.0 over the first n_addr elements of `dst`."""
    check("pt_probe_atomic", load().pt_probe_atomic(_ptr(dst), int(n_addr), int(n_updates), int(width),
                                                    stream or None))
