"""Batched persistent rendering: many cameras over several scenes in one launch.

``Batch`` builds the job table (through ``pt_batch_create``), runs it with one
persistent launch (``pt_batch_run``) or replays it from a captured CUDA graph,
and ``autotune`` picks tile size, lanes per pixel and CTAs per SM by timing the
candidates on the actual jobs, remembering the choice in a JSON file keyed by
the GPU and a signature of the jobs.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass
from typing import List, Optional

import torch

from . import abi
from . import scenes as S


@dataclass
class Job:
    dscene: "object"             # render.DeviceScene
    camera: S.Camera
    spp: int
    max_depth: int = 8
    rr_depth: int = 3
    seed: int = 1
    backward_seed: int = 2
    target: Optional[torch.Tensor] = None   # [H,W,3] device; None = forward only
    g_textures: Optional[list] = None
    g_roughness: Optional[torch.Tensor] = None
    g_albedo: Optional[torch.Tensor] = None
    g_env: Optional[torch.Tensor] = None     # environment-radiance gradient [env_h, env_w, 4]

    def __post_init__(self):
        dev = self.dscene.albedo.device
        h, w = self.camera.height, self.camera.width
        self.image = torch.zeros((h, w, 3), device=dev)

    def struct(self) -> abi.pt_job:
        j = abi.pt_job()
        ds = self.dscene
        j.scene = ds.handle
        j.camera = abi.camera_struct(self.camera)
        j.width, j.height, j.spp = self.camera.width, self.camera.height, self.spp
        j.max_depth, j.rr_depth, j.nee = self.max_depth, self.rr_depth, 1
        j.seed, j.backward_seed = self.seed, self.backward_seed
        j.params = abi.params_struct(ds.albedo, ds.textures, ds.roughness)
        j.grads = abi.grads_struct(self.g_albedo, self.g_textures or (), self.g_roughness, self.g_env)
        j.image = self.image.data_ptr()
        j.target = self.target.data_ptr() if self.target is not None else None
        return j


class Batch:
    def __init__(self, jobs: List[Job], tile=4, lanes_per_pixel=4, ctas_per_sm=4, block_size=128):
        self.jobs = jobs
        self.opts = abi.pt_batch_opts(tile, lanes_per_pixel, ctas_per_sm, block_size)
        self.handle = abi.pt_batch_create([j.struct() for j in jobs], self.opts)
        self.graph = None

    @property
    def n_items(self) -> int:
        return abi.pt_batch_info(self.handle)

    def run(self):
        abi.pt_batch_run(self.handle, torch.cuda.current_stream().cuda_stream)

    def capture(self):
        """Capture pt_batch_run into a CUDA graph (it allocates nothing and never syncs)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            abi.pt_batch_run(self.handle, s.cuda_stream)  # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            abi.pt_batch_run(self.handle, torch.cuda.current_stream().cuda_stream)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def close(self):
        if getattr(self, "handle", None):
            abi.pt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _cache_path():
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "ptgb", "autotune.json")


def jobs_signature(jobs: List[Job]) -> str:
    h = hashlib.sha1()
    for j in jobs:
        h.update(f"{j.dscene.scene.n_tris}:{j.camera.width}x{j.camera.height}:{j.spp}:{j.max_depth}:"
                 f"{j.target is not None};".encode())
    return h.hexdigest()[:16]


def time_batch(b: Batch, reps=2) -> float:
    b.run()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, e = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        b.run()
        e.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(e))
    return min(ts)


def autotune(jobs: List[Job], candidates=None, use_cache=True, reset_grads=None) -> dict:
    """Time each candidate (tile, lanes_per_pixel, ctas_per_sm) on the real jobs; keep the fastest."""
    key = f"{torch.cuda.get_device_name()}|{jobs_signature(jobs)}"
    path = _cache_path()
    table = {}
    if use_cache and os.path.exists(path):
        try:
            table = json.load(open(path))
        except Exception:
            table = {}
        if key in table:
            return table[key]
    if candidates is None:
        candidates = [(t, l, c) for t in (2, 4, 8) for l in (2, 4, 8) for c in (4,)]
    results = []
    for (t, l, c) in candidates:
        b = Batch(jobs, tile=t, lanes_per_pixel=l, ctas_per_sm=c)
        ms = time_batch(b, reps=1)
        b.close()
        if reset_grads:
            reset_grads()
        results.append({"tile": t, "lanes_per_pixel": l, "ctas_per_sm": c, "ms": ms})
    best = min(results, key=lambda r: r["ms"])
    best = dict(best, candidates=results)
    if use_cache:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        table[key] = best
        tmp = path + f".tmp{os.getpid()}"
        json.dump(table, open(tmp, "w"), indent=1)
        os.replace(tmp, path)
    return best
