"""Device-side scene wrapper and the differentiable render (torch.autograd.Function).

``DeviceScene`` owns a pt_scene handle (geometry, materials, BVH in
library-owned device memory) plus the differentiable parameters as torch CUDA
tensors.  ``RenderFn`` calls ``pt_render_forward`` in its forward and
``pt_render_backward`` (path replay backpropagation) in its backward; torch
only provides memory and the stream.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import abi
from . import scenes as S


@dataclass
class RenderSettings:
    width: int
    height: int
    spp: int
    max_depth: int
    seed: int
    rr_depth: int = -1
    nee: bool = True
    dispatch: int = abi.PT_DISPATCH_SWITCH
    crop: Optional[tuple] = None       # (x0, y0, w, h)
    lanes_per_pixel: int = 0
    block_size: int = 0
    tex_aggregate: int = 0
    backward_seed: Optional[int] = None  # None: same seed as forward (correlated); else decorrelated
    cache: Optional[int] = None          # pt_cache handle: cache-terminated paths
    cache_bounce: int = 1
    prb_mode: int = 0                    # backward: 0 auto (= split), 1 fused PRB, 2 split (abi.PT_PRB_*)
    schedule: int = 0                    # 0 auto (= static), 1 persistent lanes, 2 static (abi.PT_SCHED_*)

    def rows_cols(self):
        return (self.crop[3], self.crop[2]) if self.crop else (self.height, self.width)


class DeviceScene:
    """A scene uploaded through the C ABI, with device copies of its parameters."""

    def __init__(self, scene: S.Scene, layout: int = abi.PT_BVH_BINARY, max_leaf_tris: int = 0, device="cuda"):
        self.scene = scene
        self.handle = abi.pt_scene_create(scene)
        try:
            abi.pt_bvh_build(self.handle, layout, max_leaf_tris)
        except Exception:
            abi.pt_scene_destroy(self.handle)
            self.handle = None
            raise
        dev = torch.device(device)
        self.device = dev
        self.albedo = torch.as_tensor(scene.albedo, dtype=torch.float32).reshape(-1, 3).to(dev).contiguous()
        self.textures = [torch.as_tensor(t, dtype=torch.float32).to(dev).contiguous() for t in scene.textures]
        self.roughness = torch.as_tensor(scene.roughness, dtype=torch.float32).to(dev).contiguous()
        # environment radiance (a differentiable emitter; sampling keeps the scene's map)
        self.env = (torch.as_tensor(scene.env, dtype=torch.float32).to(dev).contiguous()
                    if scene.env is not None else None)
        self.cameras = list(scene.cameras)
        self.n_shapes = scene.n_shapes

    def info(self) -> dict:
        return abi.pt_scene_get_info(self.handle)

    def rebuild_bvh(self, layout=abi.PT_BVH_BINARY, max_leaf_tris=0):
        abi.pt_bvh_build(self.handle, layout, max_leaf_tris)

    def close(self):
        if getattr(self, "handle", None):
            abi.pt_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ raw calls
    def _desc(self, cams, st: RenderSettings, seed=None, dbg_L=None, dbg_hash=None, counters=None):
        return abi.render_desc(cams, st.width, st.height, st.spp, st.max_depth,
                               st.seed if seed is None else seed, st.rr_depth, st.nee, st.dispatch, st.crop,
                               st.lanes_per_pixel, st.block_size, st.tex_aggregate, dbg_L, dbg_hash, counters,
                               st.cache, st.cache_bounce, st.prb_mode, st.schedule)

    def forward(self, st: RenderSettings, cams: Optional[Sequence[S.Camera]] = None, albedo=None, textures=None,
                roughness=None, out=None, per_sample=False, counters=None, env=None):
        cams = list(cams) if cams is not None else self.cameras
        rows, cols = st.rows_cols()
        dev = self.albedo.device
        img = out if out is not None else torch.empty((len(cams), rows, cols, 3), device=dev, dtype=torch.float32)
        dL = dh = None
        if per_sample:
            dL = torch.empty((len(cams), rows, cols, st.spp, 3), device=dev, dtype=torch.float32)
            dh = torch.empty((len(cams), rows, cols, st.spp), device=dev, dtype=torch.int32)
        p = abi.params_struct(self.albedo if albedo is None else albedo,
                              self.textures if textures is None else textures,
                              self.roughness if roughness is None else roughness, env)
        desc = self._desc(cams, st, dbg_L=dL, dbg_hash=dh, counters=counters)
        abi.pt_render_forward(self.handle, desc, p, img, torch.cuda.current_stream(dev).cuda_stream)
        return (img, dL, dh) if per_sample else img

    def backward(self, st: RenderSettings, grad_image, cams=None, albedo=None, textures=None, roughness=None,
                 g_albedo=None, g_textures=None, g_roughness=None, seed=None, counters=None, env=None, g_env=None):
        cams = list(cams) if cams is not None else self.cameras
        p = abi.params_struct(self.albedo if albedo is None else albedo,
                              self.textures if textures is None else textures,
                              self.roughness if roughness is None else roughness, env)
        g = abi.grads_struct(g_albedo, g_textures or (), g_roughness, g_env)
        desc = self._desc(cams, st, seed=seed, counters=counters)
        abi.pt_render_backward(self.handle, desc, p, grad_image.contiguous(), g,
                               torch.cuda.current_stream(grad_image.device).cuda_stream)

    def backward_reparam(self, st: RenderSettings, grad_image, g_translation=None, cams=None, albedo=None,
                         textures=None, roughness=None, env=None, seed=None, rays=None, g_vertices=None, **opts):
        """Reparameterized PRB (Sec. 4.7): accumulate the gradient of sum(grad_image *
        image) with respect to one translation per shape into g_translation
        [n_shapes, 3] (pt_render_backward_reparam) and/or with respect to every
        triangle corner's position into g_vertices [n_tris, 3, 3]
        (pt_render_backward_reparam_vertices).  opts: pt_reparam_opts fields; rays:
        optional int64 device counter of the rays traced."""
        cams = list(cams) if cams is not None else self.cameras
        p = abi.params_struct(self.albedo if albedo is None else albedo,
                              self.textures if textures is None else textures,
                              self.roughness if roughness is None else roughness, env)
        desc = self._desc(cams, st, seed=seed)
        stream = torch.cuda.current_stream(grad_image.device).cuda_stream
        if g_translation is None and g_vertices is None:
            raise ValueError("pass g_translation and/or g_vertices")
        for g, shape, name in ((g_translation, (self.n_shapes, 3), "g_translation"),
                               (g_vertices, (self.scene.n_tris, 3, 3), "g_vertices")):
            if g is not None and (g.dtype != torch.float32 or not g.is_contiguous() or tuple(g.shape) != shape):
                raise ValueError(f"{name} must be a contiguous float32 {list(shape)} tensor")
        o = abi.reparam_opts(**opts)
        if g_translation is not None:
            abi.pt_render_backward_reparam(self.handle, desc, p, o, grad_image.contiguous(), g_translation, rays,
                                           stream)
        if g_vertices is not None:
            abi.pt_render_backward_reparam_vertices(self.handle, desc, p, o, grad_image.contiguous(), g_vertices,
                                                    rays, stream)

    def jvp_reparam(self, st: RenderSettings, dir_translation=None, cams=None, albedo=None, textures=None,
                    roughness=None, env=None, seed=None, rays=None, with_image=True, dir_vertices=None, **opts):
        """Forward-mode reparameterized derivative: (image or None, image_dot),
        image_dot = d image / d eps with every shape moved by eps *
        dir_translation[shape] ([n_shapes, 3], pt_render_jvp_reparam) or every
        triangle corner by eps * dir_vertices[tri][corner] ([n_tris, 3, 3],
        pt_render_jvp_reparam_vertices).  opts: pt_reparam_opts fields."""
        cams = list(cams) if cams is not None else self.cameras
        rows, cols = st.rows_cols()
        dev = self.albedo.device
        if (dir_translation is None) == (dir_vertices is None):
            raise ValueError("give exactly one of dir_translation and dir_vertices")
        vert = dir_vertices is not None
        shape = (self.scene.n_tris, 3, 3) if vert else (self.n_shapes, 3)
        d = torch.as_tensor(dir_vertices if vert else dir_translation, dtype=torch.float32, device=dev).contiguous()
        if tuple(d.shape) != shape:
            raise ValueError(f"the direction must be {list(shape)}")
        img = torch.empty((len(cams), rows, cols, 3), device=dev, dtype=torch.float32) if with_image else None
        dot = torch.empty((len(cams), rows, cols, 3), device=dev, dtype=torch.float32)
        p = abi.params_struct(self.albedo if albedo is None else albedo,
                              self.textures if textures is None else textures,
                              self.roughness if roughness is None else roughness, env)
        desc = self._desc(cams, st, seed=seed)
        fn = abi.pt_render_jvp_reparam_vertices if vert else abi.pt_render_jvp_reparam
        fn(self.handle, desc, p, abi.reparam_opts(**opts), d, img, dot, rays, torch.cuda.current_stream(dev).cuda_stream)
        return img, dot

    # ------------------------------------------------------------------ wavefront variant
    def wavefront_forward(self, st: RenderSettings, calls: int = abi.PT_WF_TRACED, wave_paths: int = 0, cams=None,
                          albedo=None, textures=None, roughness=None, out=None, per_sample=False, env=None):
        """pt_wavefront_forward: the same image as forward(), one kernel per stage."""
        cams = list(cams) if cams is not None else self.cameras
        rows, cols = st.rows_cols()
        dev = self.albedo.device
        img = out if out is not None else torch.empty((len(cams), rows, cols, 3), device=dev, dtype=torch.float32)
        dL = dh = None
        if per_sample:
            dL = torch.empty((len(cams), rows, cols, st.spp, 3), device=dev, dtype=torch.float32)
            dh = torch.empty((len(cams), rows, cols, st.spp), device=dev, dtype=torch.int32)
        p = abi.params_struct(self.albedo if albedo is None else albedo,
                              self.textures if textures is None else textures,
                              self.roughness if roughness is None else roughness, env)
        desc = self._desc(cams, st, dbg_L=dL, dbg_hash=dh)
        abi.pt_wavefront_forward(self.handle, desc, p, abi.pt_wavefront_opts(calls, wave_paths), img,
                                 torch.cuda.current_stream(dev).cuda_stream)
        return (img, dL, dh) if per_sample else img

    def wavefront_backward(self, st: RenderSettings, grad_image, calls: int = abi.PT_WF_TRACED, wave_paths: int = 0,
                           cams=None, albedo=None, textures=None, roughness=None, g_albedo=None, g_textures=None,
                           g_roughness=None, seed=None, env=None, g_env=None):
        """pt_wavefront_backward: the same gradients as backward(), one kernel per stage."""
        cams = list(cams) if cams is not None else self.cameras
        p = abi.params_struct(self.albedo if albedo is None else albedo,
                              self.textures if textures is None else textures,
                              self.roughness if roughness is None else roughness, env)
        g = abi.grads_struct(g_albedo, g_textures or (), g_roughness, g_env)
        desc = self._desc(cams, st, seed=seed)
        abi.pt_wavefront_backward(self.handle, desc, p, abi.pt_wavefront_opts(calls, wave_paths),
                                  grad_image.contiguous(), g, torch.cuda.current_stream(grad_image.device).cuda_stream)

    def jvp(self, st: RenderSettings, t_albedo=None, t_textures=None, t_roughness=None, cams=None, albedo=None,
            textures=None, roughness=None, t_env=None, env=None):
        """(image, image_dot): the render and its derivative along the parameter
        direction (t_albedo, t_textures, t_roughness); None members are zero."""
        cams = list(cams) if cams is not None else self.cameras
        rows, cols = st.rows_cols()
        dev = self.albedo.device
        img = torch.empty((len(cams), rows, cols, 3), device=dev, dtype=torch.float32)
        dot = torch.empty_like(img)
        textures = self.textures if textures is None else textures
        p = abi.params_struct(self.albedo if albedo is None else albedo, textures,
                              self.roughness if roughness is None else roughness, env)
        tt = list(t_textures) if t_textures is not None else []
        t = abi.params_struct(t_albedo, [], t_roughness, t_env.contiguous() if t_env is not None else None)
        for i, x in enumerate(tt):
            if x is not None:
                t.tex[i] = abi._ptr(x.contiguous())
                t.tex_w[i] = int(x.shape[1])
                t.tex_h[i] = int(x.shape[0])
        t.n_tex = len(tt)
        desc = self._desc(cams, st)
        abi.pt_render_jvp(self.handle, desc, p, t, img, dot, torch.cuda.current_stream(dev).cuda_stream)
        return img, dot

    def status(self) -> int:
        return abi.pt_last_device_status(self.handle, torch.cuda.current_stream().cuda_stream)

    def trace(self, origins: torch.Tensor, directions: torch.Tensor, tmax: torch.Tensor = None,
              any_hit: bool = False):
        """Ray queries through the path tracer's traversal (pt_trace_rays): closest hit
        (or any hit before tmax) of each ray.  origins, directions: [n, 3] on this
        device.  Returns (t [n], prim [n] int32: input triangle index or -1, uv [n, 2])."""
        rays = torch.cat([origins, directions], 1).to(device=self.device, dtype=torch.float32).contiguous()
        n = rays.shape[0]
        t = torch.empty(n, device=self.device)
        prim = torch.empty(n, dtype=torch.int32, device=self.device)
        uv = torch.empty((n, 2), device=self.device)
        tm = None if tmax is None else tmax.to(device=self.device, dtype=torch.float32).contiguous()
        abi.pt_trace_rays(self.handle, rays, n, t, prim, tmax=tm, uv=uv, any_hit=any_hit,
                          stream=torch.cuda.current_stream(self.device).cuda_stream)
        return t, prim, uv


class Checkpoints:
    """Owner of a pt_ckpt buffer (reverse mode with one checkpoint per path vertex)."""

    def __init__(self, max_samples: int, max_depth: int):
        self.handle = abi.pt_ckpt_create(max_samples, max_depth)

    @property
    def nbytes(self) -> int:
        return abi.pt_ckpt_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            abi.pt_ckpt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ckpt_forward(dscene: DeviceScene, st: RenderSettings, ck: Checkpoints, cams=None, out=None, env=None):
    """pt_ckpt_forward: the image, storing a checkpoint per path vertex in `ck`."""
    cams = list(cams) if cams is not None else dscene.cameras
    rows, cols = st.rows_cols()
    dev = dscene.albedo.device
    img = out if out is not None else torch.empty((len(cams), rows, cols, 3), device=dev, dtype=torch.float32)
    p = abi.params_struct(dscene.albedo, dscene.textures, dscene.roughness, env)
    abi.pt_ckpt_forward(dscene.handle, dscene._desc(cams, st), p, ck.handle, img,
                        torch.cuda.current_stream(dev).cuda_stream)
    return img


def ckpt_backward(dscene: DeviceScene, st: RenderSettings, ck: Checkpoints, grad_image, cams=None, g_albedo=None,
                  g_textures=None, g_roughness=None, g_env=None, env=None):
    """pt_ckpt_backward: gradients from the checkpoints of the last ckpt_forward."""
    cams = list(cams) if cams is not None else dscene.cameras
    p = abi.params_struct(dscene.albedo, dscene.textures, dscene.roughness, env)
    g = abi.grads_struct(g_albedo, g_textures or (), g_roughness, g_env)
    abi.pt_ckpt_backward(dscene.handle, dscene._desc(cams, st), p, ck.handle, grad_image.contiguous(), g,
                         torch.cuda.current_stream(grad_image.device).cuda_stream)


class RenderFn(torch.autograd.Function):
    """image = render(albedo, roughness, env, texture_0..k); backward = path replay
    backpropagation; forward-mode (torch.autograd.forward_ad) = pt_render_jvp.

    env may be None (the scene's environment map, not differentiated).  The
    backward seed is ``settings.backward_seed`` if given (decorrelated, as the
    paper's three-phase PRB step does), else the forward seed (correlated).
    """

    @staticmethod
    def forward(ctx, dscene: DeviceScene, st: RenderSettings, albedo, roughness, env, *textures):
        ctx.dscene = dscene
        ctx.st = st
        ctx.has_env = env is not None
        ctx.save_for_backward(albedo, roughness, *( [env] if env is not None else [] ), *textures)
        ctx.primal = (albedo.detach().contiguous(), roughness.detach().contiguous(),
                      env.detach().contiguous() if env is not None else None,
                      [t.detach().contiguous() for t in textures])
        a, r, e, tx = ctx.primal
        return dscene.forward(st, albedo=a, roughness=r, textures=tx, env=e)

    @staticmethod
    def jvp(ctx, _scene, _st, t_albedo, t_roughness, t_env, *t_textures):
        """The image tangent along the input tangents, from one pt_render_jvp pass."""
        a, r, e, tx = ctx.primal
        _, dot = ctx.dscene.jvp(ctx.st, t_albedo=t_albedo, t_roughness=t_roughness,
                                t_textures=[t.contiguous() if t is not None else None for t in t_textures],
                                t_env=t_env if ctx.has_env else None,
                                albedo=a, roughness=r, textures=tx, env=e)
        return dot

    @staticmethod
    def backward(ctx, grad_img):
        saved = ctx.saved_tensors
        albedo, roughness = saved[0], saved[1]
        env = saved[2] if ctx.has_env else None
        textures = saved[3:] if ctx.has_env else saved[2:]
        ga = torch.zeros_like(albedo) if ctx.needs_input_grad[2] else None
        gr = torch.zeros_like(roughness) if ctx.needs_input_grad[3] else None
        ge = torch.zeros_like(env) if ctx.has_env and ctx.needs_input_grad[4] else None
        gt = [torch.zeros_like(t) if ctx.needs_input_grad[5 + i] else None for i, t in enumerate(textures)]
        st = ctx.st
        seed = st.backward_seed if st.backward_seed is not None else st.seed
        a, r, e, tx = ctx.primal
        ctx.dscene.backward(st, grad_img.contiguous(), albedo=a, roughness=r, textures=tx, env=e, g_albedo=ga,
                            g_textures=gt if any(g is not None for g in gt) else None, g_roughness=gr, g_env=ge,
                            seed=seed)
        return (None, None, ga, gr, ge, *gt)


def render(dscene: DeviceScene, st: RenderSettings, albedo, roughness, textures: Sequence[torch.Tensor], env=None):
    return RenderFn.apply(dscene, st, albedo, roughness, env, *textures)


class TranslateFn(torch.autograd.Function):
    """image = render of `scene` with every shape moved by translations[shape]
    ([n_shapes, 3]) and every camera by camera_offset ([3]); backward =
    reparameterized PRB (pt_render_backward_reparam, Sec. 4.7), the gradient with
    respect to the translations through visibility.  Moving the cameras is moving
    every shape the opposite way (the environment lies at infinity), so the camera
    offset's gradient is minus the sum of the shapes'.  The moved geometry is
    uploaded (scene and BVH built) on every call."""

    @staticmethod
    def forward(ctx, scene: S.Scene, st: RenderSettings, layout: int, opts: dict, translations, camera_offset):
        ref = translations if translations is not None else camera_offset
        sc = scene
        if translations is not None:
            sc = sc.translated(translations.detach().to("cpu", torch.float64).numpy())
        if camera_offset is not None:
            sc = sc.camera_moved(camera_offset.detach().to("cpu", torch.float64).numpy())
        ds = DeviceScene(sc, layout=layout, device=ref.device)
        ctx.ds, ctx.st, ctx.opts = ds, st, opts
        return ds.forward(st)

    @staticmethod
    def backward(ctx, grad_img):
        ds, st = ctx.ds, ctx.st
        g = torch.zeros((ds.n_shapes, 3), device=grad_img.device, dtype=torch.float32)
        seed = st.backward_seed if st.backward_seed is not None else st.seed
        ds.backward_reparam(st, grad_img.contiguous(), g, seed=seed, **ctx.opts)
        ds.close()  # pt_scene_destroy frees device memory, which waits for the launch
        ctx.ds = None
        g_cam = -g.sum(dim=0) if ctx.needs_input_grad[5] else None
        return None, None, None, None, (g if ctx.needs_input_grad[4] else None), g_cam


def render_translated(scene: S.Scene, st: RenderSettings, translations=None, layout: int = abi.PT_BVH_BINARY,
                      camera_offset=None, **reparam_opts):
    """Differentiable render with respect to one translation per shape ([n_shapes,
    3]) and / or one translation of the cameras ([3]); at least one is given."""
    if translations is None and camera_offset is None:
        raise ValueError("render_translated: give translations, camera_offset or both")
    return TranslateFn.apply(scene, st, layout, reparam_opts, translations, camera_offset)


class VerticesFn(torch.autograd.Function):
    """image = render of `scene` with its triangle corners at `vertices` ([n_tris,
    3, 3], absolute positions); backward = reparameterized PRB with every corner as
    a parameter (pt_render_backward_reparam_vertices).  The geometry is uploaded on
    every call; compose with torch for any parametrisation of the vertices."""

    @staticmethod
    def forward(ctx, scene: S.Scene, st: RenderSettings, layout: int, opts: dict, vertices):
        import copy
        moved = copy.copy(scene)
        moved.vertices = np.ascontiguousarray(vertices.detach().to("cpu", torch.float32).numpy())
        ds = DeviceScene(moved, layout=layout, device=vertices.device)
        ctx.ds, ctx.st, ctx.opts = ds, st, opts
        return ds.forward(st)

    @staticmethod
    def backward(ctx, grad_img):
        ds, st = ctx.ds, ctx.st
        g = torch.zeros((ds.scene.n_tris, 3, 3), device=grad_img.device, dtype=torch.float32)
        seed = st.backward_seed if st.backward_seed is not None else st.seed
        ds.backward_reparam(st, grad_img.contiguous(), g_vertices=g, seed=seed, **ctx.opts)
        ds.close()
        ctx.ds = None
        return None, None, None, None, g


def render_vertices(scene: S.Scene, st: RenderSettings, vertices, layout: int = abi.PT_BVH_BINARY,
                    **reparam_opts):
    """Differentiable render with respect to every triangle corner's position."""
    return VerticesFn.apply(scene, st, layout, reparam_opts, vertices)


def save_pfm(path: str, image) -> None:
    """Write an RGB float image ([rows, cols, 3], row 0 = top; tensor or array) as
    a little-endian Portable Float Map."""
    img = image.detach().cpu().numpy() if isinstance(image, torch.Tensor) else np.asarray(image)
    img = np.ascontiguousarray(img, dtype="<f4").reshape(img.shape[-3], img.shape[-2], 3)
    with open(path, "wb") as f:
        f.write(b"PF\n%d %d\n-1.0\n" % (img.shape[1], img.shape[0]))
        f.write(np.ascontiguousarray(img[::-1]).tobytes())  # PFM stores the bottom row first


def load_pfm(path: str) -> np.ndarray:
    """Read a colour Portable Float Map into [rows, cols, 3] float32, row 0 = top."""
    with open(path, "rb") as f:
        if f.readline().strip() != b"PF":
            raise ValueError("not a colour PFM file")
        w, h = (int(x) for x in f.readline().split())
        scale = float(f.readline())
        data = np.frombuffer(f.read(), dtype="<f4" if scale < 0 else ">f4", count=w * h * 3)
    return np.ascontiguousarray(data.reshape(h, w, 3)[::-1], dtype=np.float32)


class RadianceCache:
    """Owner of a pt_cache (MLP weights, Adam state, query/record buffers)."""

    def __init__(self, box_lo, box_hi, batch=65536, max_queries=0, max_records=0, max_paths=0, lr=5e-3,
                 init_weights=None, seed=0, **adam):
        self.handle = abi.pt_cache_create(box_lo, box_hi, batch, max_queries, max_records, max_paths, lr,
                                          init_weights=init_weights, seed=seed, **adam)

    def weights(self):
        return abi.pt_cache_get_weights(self.handle)

    def average(self):
        """The averaged weights queries use when the cache was created with ema > 0."""
        return abi.pt_cache_get_average(self.handle)

    def set_average(self, w):
        abi.pt_cache_set_average(self.handle, w)

    def set_weights(self, w):
        abi.pt_cache_set_weights(self.handle, w)

    def query(self, raw, out=None):
        n = raw.shape[0]
        out = out if out is not None else torch.empty((n, 3), device=raw.device, dtype=torch.float32)
        abi.pt_cache_query(self.handle, raw.contiguous(), out, n, torch.cuda.current_stream(raw.device).cuda_stream)
        return out

    def train_records(self, raw, target, steps=1):
        abi.pt_cache_train_records(self.handle, raw.contiguous(), target.contiguous(), raw.shape[0], steps,
                                   torch.cuda.current_stream(raw.device).cuda_stream)

    def train(self, dscene: "DeviceScene", st: RenderSettings, steps=1, cams=None) -> int:
        cams = list(cams) if cams is not None else dscene.cameras
        p = abi.params_struct(dscene.albedo, dscene.textures, dscene.roughness)
        desc = dscene._desc(cams, st)
        desc.cache = None
        return abi.pt_cache_train(self.handle, dscene.handle, desc, p, steps,
                                  torch.cuda.current_stream(dscene.albedo.device).cuda_stream)

    def last_loss(self) -> float:
        return abi.pt_cache_last_loss(self.handle, torch.cuda.current_stream().cuda_stream)

    def read_records(self, cap):
        return abi.pt_cache_read_records(self.handle, cap)

    # ---- checkpoint / resume of training: weights, Adam moments and step in one file
    _MAGIC = b"PTGBNRC1"

    def save(self, path):
        w, m, v, step = abi.pt_cache_get_state(self.handle)
        with open(path, "wb") as f:
            f.write(self._MAGIC)
            f.write(np.array([abi.PT_CACHE_N_PARAMS, step], np.int64).tobytes())
            for a in (w, m, v):
                f.write(a.astype("<f4").tobytes())

    def load(self, path):
        with open(path, "rb") as f:
            if f.read(8) != self._MAGIC:
                raise ValueError(f"{path}: not a radiance-cache checkpoint")
            n, step = np.frombuffer(f.read(16), np.int64)
            if n != abi.PT_CACHE_N_PARAMS:
                raise ValueError(f"{path}: {n} parameters, expected {abi.PT_CACHE_N_PARAMS}")
            w, m, v = (np.frombuffer(f.read(4 * n), "<f4").astype(np.float32) for _ in range(3))
        abi.pt_cache_set_state(self.handle, w, m, v, int(step))

    def close(self):
        if getattr(self, "handle", None):
            abi.pt_cache_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
