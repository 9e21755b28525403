"""FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``liboracle.so`` (built from
``oracle.cpp`` and ``mlp.cpp`` with g++; see ``build()``) through ctypes and
marshals the seeded scenes of ``paper_2202_01284_gb300.scenes`` into the
oracle's own input records.  Nothing here touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "oracle.cpp"), os.path.join(_HERE, "mlp.cpp")]
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (plain g++ -O2, no architecture flags)."""
    srcs = [s for s in _SOURCES if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class SceneIn(C.Structure):
    _fields_ = [
        ("n_tris", C.c_int), ("vertices", C.c_void_p), ("uvs", C.c_void_p), ("tri_shape", C.c_void_p),
        ("n_shapes", C.c_int), ("bsdf", C.c_void_p), ("tex", C.c_void_p), ("albedo_index", C.c_void_p),
        ("rough_index", C.c_void_p), ("alpha", C.c_void_p), ("f0", C.c_void_p), ("eta", C.c_void_p),
        ("emission", C.c_void_p), ("diffuse_weight", C.c_void_p),
        ("n_albedo", C.c_int), ("albedo", C.c_void_p),
        ("n_tex", C.c_int), ("tex_data", C.c_void_p), ("tex_w", C.c_void_p), ("tex_h", C.c_void_p),
        ("n_rough", C.c_int), ("roughness", C.c_void_p),
        ("env_w", C.c_int), ("env_h", C.c_int), ("env", C.c_void_p),
    ]


class RenderIn(C.Structure):
    _fields_ = [
        ("origin", C.c_double * 3), ("target", C.c_double * 3), ("up", C.c_double * 3),
        ("vfov_deg", C.c_double), ("width", C.c_int), ("height", C.c_int),
        ("spp", C.c_int), ("max_depth", C.c_int), ("rr_depth", C.c_int), ("nee", C.c_int),
        ("seed", C.c_uint64), ("cam_index", C.c_int),
        ("crop_x0", C.c_int), ("crop_y0", C.c_int), ("crop_w", C.c_int), ("crop_h", C.c_int),
        ("env_radiance", C.c_void_p),
    ]


class ReparamIn(C.Structure):
    _fields_ = [("n_aux", C.c_int), ("kappa", C.c_double), ("kernel_scale", C.c_double), ("power", C.c_double),
                ("miss", C.c_double), ("eps", C.c_double), ("jackknife", C.c_int),
                ("border", C.c_double), ("edge_spp", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            vp, ip, dp = C.c_void_p, C.c_int, C.c_double
            L.oracle_scene_new.restype = vp
            L.oracle_scene_new.argtypes = [C.POINTER(SceneIn)]
            L.oracle_scene_free.argtypes = [vp]
            L.oracle_render.argtypes = [vp, C.POINTER(RenderIn), vp, vp, vp, ip, vp]
            L.oracle_grad_tape.argtypes = [vp, C.POINTER(RenderIn), vp, vp, vp, vp, vp, ip, vp]
            L.oracle_grad_dual.argtypes = [vp, C.POINTER(RenderIn), vp, ip, vp, vp, ip]
            L.oracle_render_jvp.argtypes = [vp, C.POINTER(RenderIn), vp, vp, ip, vp, vp, vp, vp, ip]
            L.oracle_pcg32.argtypes = [C.c_uint64, C.c_uint64, ip, vp]
            L.oracle_trace.argtypes = [vp, ip, vp, vp, ip, vp, vp]
            L.oracle_bsdf_eval.argtypes = [ip, vp, vp, vp, vp, vp]
            L.oracle_bsdf_sample.argtypes = [ip, vp, vp, dp, dp, dp, vp]
            L.oracle_bsdf_sample.restype = ip
            L.oracle_bsdf_dfactors.argtypes = [ip, vp, vp, vp, vp]
            L.oracle_bsdf_normal_dlog.argtypes = [ip, vp, vp, vp, vp, vp, vp]
            L.oracle_dual_toys.argtypes = [dp, ip, dp, vp]
            L.oracle_fresnel.argtypes = [dp, dp]
            L.oracle_fresnel.restype = dp
            L.oracle_dielectric_sample.argtypes = [vp, vp, dp, dp, vp, vp]
            L.oracle_dielectric_sample.restype = ip
            L.oracle_ggx_terms.argtypes = [dp, dp, dp, vp]
            L.oracle_env_pdf.argtypes = [vp, vp]
            L.oracle_env_pdf.restype = dp
            L.oracle_frame.argtypes = [vp, vp, vp]
            L.oracle_render_cached.argtypes = [vp, C.POINTER(RenderIn), vp, vp, ip, vp, ip]
            L.oracle_grad_dual_cached.argtypes = [vp, C.POINTER(RenderIn), vp, vp, ip, vp, ip, vp, vp, ip]
            L.oracle_train_records.argtypes = [vp, C.POINTER(RenderIn), ip, vp, vp, vp]
            L.oracle_train_records.restype = ip
            L.oracle_mlp_n_params.restype = ip
            L.oracle_mlp_set_rounding.argtypes = [ip]
            L.oracle_mlp_forward.argtypes = [vp, ip, vp, vp]
            L.oracle_mlp_loss_grad.argtypes = [vp, ip, vp, vp, vp, vp]
            L.oracle_mlp_loss_grad.restype = dp
            L.oracle_mlp_adam.argtypes = [vp, vp, vp, vp, ip, dp, dp, dp, dp, ip]
            L.oracle_nrc_encode.argtypes = [ip, vp, vp, vp]
            L.oracle_grad_reparam.argtypes = [vp, C.POINTER(RenderIn), vp, C.POINTER(ReparamIn), ip, vp, vp, ip, vp,
                                              ip, vp]
            L.oracle_grad_reparam.restype = ip
            L.oracle_vmf.argtypes = [dp, dp, dp, vp]
            L.oracle_sphere_div.argtypes = [ip, vp, vp]
            L.oracle_sphere_div.restype = dp
            L.oracle_warp.argtypes = [vp, vp, vp, ip, vp, C.POINTER(ReparamIn), ip, vp, vp, vp, vp, vp]
            L.oracle_warp.restype = ip
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class OracleScene:
    """Oracle-side copy of a `scenes.Scene` (FP64, its own BVH and CDFs)."""

    def __init__(self, scene):
        L = lib()
        self._keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a
        s = scene
        si = SceneIn()
        si.n_tris = s.n_tris
        si.vertices = _ptr(arr(s.vertices, np.float32))
        si.uvs = _ptr(arr(s.uvs, np.float32))
        si.tri_shape = _ptr(arr(s.tri_shape, np.int32))
        si.n_shapes = s.n_shapes
        si.bsdf = _ptr(arr(s.bsdf, np.int32))
        si.tex = _ptr(arr(s.tex, np.int32))
        si.albedo_index = _ptr(arr(s.albedo_index, np.int32))
        si.rough_index = _ptr(arr(s.rough_index, np.int32))
        si.alpha = _ptr(arr(s.alpha, np.float32))
        si.f0 = _ptr(arr(s.f0, np.float32))
        si.eta = _ptr(arr(s.eta, np.float32))
        si.emission = _ptr(arr(s.emission, np.float32))
        si.diffuse_weight = _ptr(arr(s.diffuse_weight, np.float32))
        si.n_albedo = int(s.albedo.shape[0])
        si.albedo = _ptr(arr(s.albedo.reshape(-1, 3) if s.albedo.size else np.zeros((0, 3)), np.float32))
        texs = [arr(t, np.float32) for t in s.textures]
        ptrs = (C.c_void_p * max(1, len(texs)))(*[t.ctypes.data for t in texs])
        self._keep.append(ptrs)
        si.n_tex = len(texs)
        si.tex_data = C.cast(ptrs, C.c_void_p)
        si.tex_w = _ptr(arr([t.shape[1] for t in texs] or [0], np.int32))
        si.tex_h = _ptr(arr([t.shape[0] for t in texs] or [0], np.int32))
        si.n_rough = int(s.roughness.shape[0])
        si.roughness = _ptr(arr(s.roughness if s.roughness.size else np.zeros(1), np.float32))
        if s.env is not None:
            si.env_w, si.env_h = int(s.env.shape[1]), int(s.env.shape[0])
            si.env = _ptr(arr(s.env, np.float32))
        else:
            si.env_w = si.env_h = 0
            si.env = None
        self.handle = L.oracle_scene_new(C.byref(si))
        self._keep = []  # the oracle copied everything
        self.scene = scene

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.oracle_scene_free(self.handle)
            self.handle = None


def render_in(cam, spp, max_depth, seed, rr_depth=-1, nee=True, cam_index=0, crop=None,
              env_radiance=None) -> RenderIn:
    """Render settings.  env_radiance [env_h, env_w, 4]: radiance used for shading
    instead of the scene's map (sampling keeps the scene's map)."""
    r = RenderIn()
    if env_radiance is not None:
        e = np.ascontiguousarray(env_radiance, dtype=np.float64)
        r._env_keep = e
        r.env_radiance = e.ctypes.data
    r.origin[:] = cam.origin
    r.target[:] = cam.target
    r.up[:] = cam.up
    r.vfov_deg = cam.vfov_deg
    r.width, r.height = cam.width, cam.height
    r.spp, r.max_depth, r.rr_depth, r.nee = spp, max_depth, rr_depth, int(bool(nee))
    r.seed = seed
    r.cam_index = cam_index
    if crop is not None:
        r.crop_x0, r.crop_y0, r.crop_w, r.crop_h = crop
    return r


def _crop_shape(r: RenderIn):
    return (r.crop_h, r.crop_w) if r.crop_w > 0 else (r.height, r.width)


def render(osc: OracleScene, r: RenderIn, per_sample=False, threads=0, count_rays=False):
    """Image [h][w][3] (FP64); with per_sample also [h][w][spp][3] radiance and hashes.
    With count_rays the number of rays traced (closest-hit + shadow) is appended."""
    h, w = _crop_shape(r)
    img = np.zeros((h, w, 3))
    sl = np.zeros((h, w, r.spp, 3)) if per_sample else None
    sh = np.zeros((h, w, r.spp), np.uint32) if per_sample else None
    rays = np.zeros(1, np.uint64)
    lib().oracle_render(osc.handle, C.byref(r), _ptr(img), _ptr(sl), _ptr(sh), threads, _ptr(rays))
    out = (img, sl, sh) if per_sample else (img,)
    if count_rays:
        out = out + (int(rays[0]),)
    return out if len(out) > 1 else out[0]


def grad_tape(osc: OracleScene, r: RenderIn, grad_image: np.ndarray, threads=0, count_rays=False, env=False):
    """Gradients (albedo [A,3], textures list [h,w,4], roughness [R]) by the stored tape;
    with env=True also the environment-radiance gradient [env_h, env_w, 4] (after roughness)."""
    s = osc.scene
    gi = np.ascontiguousarray(grad_image, dtype=np.float64)
    ga = np.zeros((s.albedo.shape[0], 3))
    gt = [np.zeros(t.shape) for t in s.textures]
    gr = np.zeros(s.roughness.shape[0])
    ge = np.zeros(s.env.shape if s.env is not None else (0, 0, 4))
    tp = (C.c_void_p * max(1, len(gt)))(*[t.ctypes.data for t in gt])
    rays = np.zeros(1, np.uint64)
    lib().oracle_grad_tape(osc.handle, C.byref(r), _ptr(gi), _ptr(ga), C.cast(tp, C.c_void_p), _ptr(gr),
                           _ptr(ge) if ge.size else None, threads, _ptr(rays))
    out = (ga, gt, gr, ge) if env else (ga, gt, gr)
    return out + (int(rays[0]),) if count_rays else out


def grad_dual(osc: OracleScene, r: RenderIn, grad_image: np.ndarray, sel, threads=0):
    """Gradients of the selected parameters by forward-mode duals.

    sel: list of (kind, a, b, c): (0,row,ch,0) albedo, (1,tex,texel,ch) texel, (2,idx,0,0) roughness,
    (3,pixel,ch,0) environment radiance (pixel = y * env_w + x).
    """
    gi = np.ascontiguousarray(grad_image, dtype=np.float64)
    s = np.ascontiguousarray(np.asarray(sel, np.int32).reshape(-1, 4))
    out = np.zeros(s.shape[0])
    lib().oracle_grad_dual(osc.handle, C.byref(r), _ptr(gi), s.shape[0], _ptr(s), _ptr(out), threads)
    return out


def render_jvp(osc: OracleScene, r: RenderIn, t_albedo=None, t_textures=None, t_rough=None, t_env=None, threads=0):
    """(image, image_dot): the render and its derivative along the direction
    (t_albedo [A,3], t_textures [[H,W,4] or None, ...], t_rough [R], t_env [env_h, env_w, 4]);
    None = zero."""
    rows = r.crop_h if r.crop_w > 0 else r.height
    cols = r.crop_w if r.crop_w > 0 else r.width
    img = np.zeros((rows, cols, 3))
    dot = np.zeros((rows, cols, 3))
    keep = []

    def dptr(a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return _ptr(a)
    tex = list(t_textures or [])
    arr = (C.c_void_p * max(1, len(tex)))(*[(None if t is None else C.cast(dptr(t), C.c_void_p)) for t in tex])
    lib().oracle_render_jvp(osc.handle, C.byref(r), dptr(t_albedo), C.cast(arr, C.c_void_p), len(tex),
                            dptr(t_rough), dptr(t_env), _ptr(img), _ptr(dot), threads)
    return img, dot


# Options of the reparameterized translation derivative: auxiliary rays per
# traced ray, vMF concentration of their lobe, how much narrower the weighting
# kernel is, depth-weight exponent, weight of escaping rays, normaliser floor,
# leave-one-out correction on/off, width in pixels of an optional window that
# takes the camera-ray warp to zero at the image border (0: none), paths per pixel
# edge for the term of the pixels' own moving boundaries (0: off).
REPARAM_DEFAULTS = dict(n_aux=16, kappa=1000.0, kernel_scale=8.0, power=2.0, miss=0.01, eps=1e-4,
                        jackknife=1, border=0.0, edge_spp=1)


def _reparam_in(opts) -> ReparamIn:
    o = dict(REPARAM_DEFAULTS, **opts)
    return ReparamIn(int(o["n_aux"]), float(o["kappa"]), float(o["kernel_scale"]), float(o["power"]),
                     float(o["miss"]), float(o["eps"]), int(o["jackknife"]), float(o["border"]),
                     int(o["edge_spp"]))


def grad_reparam(osc: OracleScene, r: RenderIn, grad_image=None, dot_param=-1, threads=0, vertex=False,
                 dot_dir=None, **opts):
    """Gradients through reparameterized visibility, by forward mode.

    Returns (g, image [h, w, 3], image_dot [h, w, 3]): g = sum of grad_image * d image /
    d theta (zeros without grad_image) for one translation per shape (g [n_shapes, 3])
    or, with vertex=True, every triangle corner's position (g [n_tris, 3, 3]);
    image_dot = derivative along parameter `dot_param` (3 shape + axis, or 9 triangle +
    3 corner + axis; zeros if < 0), or along the direction dot_dir (the shape of g)."""
    o = _reparam_in(opts)
    h, w = _crop_shape(r)
    gi = None if grad_image is None else np.ascontiguousarray(grad_image, dtype=np.float64).reshape(h, w, 3)
    g = np.zeros((osc.scene.n_tris, 3, 3)) if vertex else np.zeros((osc.scene.n_shapes, 3))
    img = np.zeros((h, w, 3))
    dot = np.zeros((h, w, 3))
    dd = None
    if dot_dir is not None:
        dd = np.ascontiguousarray(dot_dir, dtype=np.float64)
        assert dd.shape == g.shape
    rc = lib().oracle_grad_reparam(osc.handle, C.byref(r), _ptr(gi), C.byref(o), int(bool(vertex)), _ptr(g),
                                   _ptr(img), int(dot_param), _ptr(dot), threads, _ptr(dd))
    if rc != 0:
        raise ValueError("oracle_grad_reparam: bad options")
    return g, img, dot


def vmf(u0: float, u1: float, kappa: float) -> np.ndarray:
    """The auxiliary-ray sampler's local direction (lobe axis +z)."""
    out = np.zeros(3)
    lib().oracle_vmf(float(u0), float(u1), float(kappa), _ptr(out))
    return out


def sphere_div(kind: int, u, e) -> float:
    """Divergence on the unit sphere at u of V = e (0), w x e (1), (I - w w^T) e (2)."""
    u = np.ascontiguousarray(u, np.float64)
    e = np.ascontiguousarray(e, np.float64)
    return lib().oracle_sphere_div(kind, _ptr(u), _ptr(e))


def warp(osc: OracleScene, o, u, s_o: int, uniforms, param: int, at=None, m=None, **opts):
    """One warp field: (V at `at` (default u), div V at u, log-derivative with covector m, n_hits)."""
    op = _reparam_in(opts)
    o = np.ascontiguousarray(o, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    uni = np.ascontiguousarray(uniforms, np.float64)
    assert uni.size == 2 * op.n_aux
    at_ = None if at is None else np.ascontiguousarray(at, np.float64)
    m_ = None if m is None else np.ascontiguousarray(m, np.float64)
    V = np.zeros(3)
    div = np.zeros(1)
    logd = np.zeros(1)
    n = lib().oracle_warp(osc.handle, _ptr(o), _ptr(u), int(s_o), _ptr(uni), C.byref(op), int(param), _ptr(at_),
                          _ptr(m_), _ptr(V), _ptr(div), _ptr(logd))
    if n < 0:
        raise ValueError("oracle_warp: bad options")
    return V, float(div[0]), float(logd[0]), n


def pcg32(initstate: int, initseq: int, n: int) -> np.ndarray:
    out = np.zeros(n, np.uint32)
    lib().oracle_pcg32(initstate, initseq, n, _ptr(out))
    return out


def trace(osc: OracleScene, o: np.ndarray, d: np.ndarray, brute=False):
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    n = o.shape[0]
    t = np.zeros(n)
    p = np.zeros(n, np.int32)
    lib().oracle_trace(osc.handle, n, _ptr(o), _ptr(d), int(brute), _ptr(t), _ptr(p))
    return t, p


def bsdf_params(albedo=(0.5, 0.5, 0.5), alpha=0.3, f0=(0.04, 0.04, 0.04), eta=1.5, wd=0.8):
    return np.array(list(albedo) + [alpha] + list(f0) + [eta, wd], np.float64)


def bsdf_eval(bsdf, params, wi, wo):
    f = np.zeros(3)
    pdf = np.zeros(1)
    lib().oracle_bsdf_eval(bsdf, _ptr(params), _ptr(np.asarray(wi, np.float64)),
                           _ptr(np.asarray(wo, np.float64)), _ptr(f), _ptr(pdf))
    return f, pdf[0]


def bsdf_sample(bsdf, params, wi, u3, u4, u5):
    wo = np.zeros(3)
    ok = lib().oracle_bsdf_sample(bsdf, _ptr(params), _ptr(np.asarray(wi, np.float64)), u3, u4, u5, _ptr(wo))
    return bool(ok), wo


def bsdf_dfactors(bsdf, params, wi, wo):
    out = np.zeros(6)
    lib().oracle_bsdf_dfactors(bsdf, _ptr(params), _ptr(np.asarray(wi, np.float64)),
                               _ptr(np.asarray(wo, np.float64)), _ptr(out))
    return out[:3], out[3:]


def bsdf_normal_dlog(bsdf, params, corners, n, wi, wo) -> np.ndarray:
    """d log f_c / d corner coordinate [3 corners, 3 axes, 3 channels] through the unit
    normal of the triangle `corners` [3, 3] (oriented like n); wi, wo world directions."""
    out = np.zeros(27)
    f64 = lambda a: np.ascontiguousarray(a, np.float64)
    lib().oracle_bsdf_normal_dlog(bsdf, _ptr(params), _ptr(f64(corners)), _ptr(f64(n)), _ptr(f64(wi)),
                                  _ptr(f64(wo)), _ptr(out))
    return out.reshape(3, 3, 3)


def dual_toys(x: float, n: int, a: float) -> np.ndarray:
    """[x^n, its x-derivative, a exp(-a x), its a-derivative] by the dual-number classes."""
    out = np.zeros(4)
    lib().oracle_dual_toys(float(x), int(n), float(a), _ptr(out))
    return out


def fresnel(cos_i, eta):
    return lib().oracle_fresnel(cos_i, eta)


def dielectric_sample(ng, wi, eta, u3):
    """(refracted?, wo, radiance weight) of the integrator's dielectric event."""
    wo = np.zeros(3)
    w = np.zeros(1)
    refr = lib().oracle_dielectric_sample(_ptr(np.asarray(ng, np.float64)), _ptr(np.asarray(wi, np.float64)),
                                          float(eta), float(u3), _ptr(wo), _ptr(w))
    return bool(refr), wo, float(w[0])


def ggx_terms(alpha, cos_h, cos_w):
    """(D(cos_h), G1(cos_w)) of the conductor lobe at roughness alpha."""
    out = np.zeros(2)
    lib().oracle_ggx_terms(float(alpha), float(cos_h), float(cos_w), _ptr(out))
    return float(out[0]), float(out[1])


def env_pdf(osc: OracleScene, d):
    return lib().oracle_env_pdf(osc.handle, _ptr(np.asarray(d, np.float64)))


def frame(n):
    s = np.zeros(3)
    t = np.zeros(3)
    lib().oracle_frame(_ptr(np.asarray(n, np.float64)), _ptr(s), _ptr(t))
    return s, t


# ---------------------------------------------------------------- radiance-cache MLP
def mlp_n_params() -> int:
    return lib().oracle_mlp_n_params()


def mlp_set_rounding(on: bool) -> None:
    """BF16 rounding of weights/activations (on by default; off = plain FP64 network)."""
    lib().oracle_mlp_set_rounding(int(bool(on)))


def nrc_encode(raw: np.ndarray, box_lo, box_hi) -> np.ndarray:
    raw = np.ascontiguousarray(raw, np.float64).reshape(-1, 10)
    box = np.ascontiguousarray(list(box_lo) + list(box_hi), np.float64)
    out = np.zeros((raw.shape[0], 64))
    lib().oracle_nrc_encode(raw.shape[0], _ptr(raw), _ptr(box), _ptr(out))
    return out


def mlp_forward(W: np.ndarray, enc: np.ndarray) -> np.ndarray:
    W = np.ascontiguousarray(W, np.float64)
    enc = np.ascontiguousarray(enc, np.float64).reshape(-1, 64)
    out = np.zeros((enc.shape[0], 3))
    lib().oracle_mlp_forward(_ptr(W), enc.shape[0], _ptr(enc), _ptr(out))
    return out


def mlp_loss_grad(W: np.ndarray, enc: np.ndarray, target: np.ndarray):
    """(loss, grad [n_params], outputs [n,3]) of the relative-L2 loss."""
    W = np.ascontiguousarray(W, np.float64)
    enc = np.ascontiguousarray(enc, np.float64).reshape(-1, 64)
    t = np.ascontiguousarray(target, np.float64).reshape(-1, 3)
    g = np.zeros(W.shape[0])
    out = np.zeros((enc.shape[0], 3))
    loss = lib().oracle_mlp_loss_grad(_ptr(W), enc.shape[0], _ptr(enc), _ptr(t), _ptr(g), _ptr(out))
    return loss, g, out


def mlp_adam(W, grad, m, v, t, lr=5e-3, b1=0.9, b2=0.99, eps=1e-8):
    """In-place Adam step on FP64 arrays."""
    lib().oracle_mlp_adam(_ptr(W), _ptr(np.ascontiguousarray(grad, np.float64)), _ptr(m), _ptr(v), t, lr, b1, b2,
                          eps, W.shape[0])


# ---------------------------------------------------------------- cache-terminated rendering
def render_cached(osc: OracleScene, r: RenderIn, W, box_lo, box_hi, bounce: int, threads=0):
    h, w = _crop_shape(r)
    img = np.zeros((h, w, 3))
    Wd = np.ascontiguousarray(W, np.float64)
    box = np.ascontiguousarray(list(box_lo) + list(box_hi), np.float64)
    lib().oracle_render_cached(osc.handle, C.byref(r), _ptr(Wd), _ptr(box), bounce, _ptr(img), threads)
    return img


def grad_dual_cached(osc: OracleScene, r: RenderIn, W, box_lo, box_hi, bounce, grad_image, sel, threads=0):
    Wd = np.ascontiguousarray(W, np.float64)
    box = np.ascontiguousarray(list(box_lo) + list(box_hi), np.float64)
    gi = np.ascontiguousarray(grad_image, dtype=np.float64)
    s = np.ascontiguousarray(np.asarray(sel, np.int32).reshape(-1, 4))
    out = np.zeros(s.shape[0])
    lib().oracle_grad_dual_cached(osc.handle, C.byref(r), _ptr(Wd), _ptr(box), bounce, _ptr(gi), s.shape[0],
                                  _ptr(s), _ptr(out), threads)
    return out


def train_records(osc: OracleScene, r: RenderIn, cap: int):
    """(raw [n,10], target [n,3], meta [n,2] = (sample index, depth)) of full-length paths."""
    raw = np.zeros((cap, 10))
    tgt = np.zeros((cap, 3))
    meta = np.zeros((cap, 2), np.int32)
    n = lib().oracle_train_records(osc.handle, C.byref(r), cap, _ptr(raw), _ptr(tgt), _ptr(meta))
    return raw[:n], tgt[:n], meta[:n]
