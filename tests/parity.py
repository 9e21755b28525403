"""Comparison helpers for GPU-vs-oracle parity tests."""
import numpy as np

REL_TOL = 1e-4          # per-pixel relative error bound
PIXEL_FRACTION = 0.999  # fraction of pixels that must meet it
GRAD_COSINE = 0.9999    # gradient cosine similarity bound


def rel_ok(gpu, ref, rel=REL_TOL, tau_frac=1e-3):
    """|g - o| <= rel * max(|o|, tau), tau = tau_frac * mean|o| (near-black pixels)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    tau = tau_frac * max(np.abs(ref).mean(), 1e-30)
    return np.abs(gpu - ref) <= rel * np.maximum(np.abs(ref), tau)


def pixel_ok_fraction(gpu_img, ref_img, rel=REL_TOL):
    ok = rel_ok(gpu_img, ref_img, rel).all(axis=-1)
    return ok.mean(), ok


def cosine(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    if na == 0 and nb == 0:
        return 1.0
    return float(a @ b / (na * nb))


SAMPLE_REL_TOL = 1e-3  # one FP32 path vs FP64: grazing cosines and tiny NEE terms lose a few more digits


def sample_report(gpu_L, gpu_hash, ref_L, ref_hash, gpu_img=None, ref_img=None):
    """Per-sample comparison: samples whose decision fingerprints agree must match
    within SAMPLE_REL_TOL; the rest are path-divergence outliers (counted).  With
    images, pixels are split into clean ones (all samples agree in their decisions,
    judged against the 1e-4 per-pixel bound) and divergent ones (reported)."""
    same = np.asarray(gpu_hash, np.uint32) == np.asarray(ref_hash, np.uint32)
    ok = rel_ok(gpu_L, ref_L, SAMPLE_REL_TOL).all(axis=-1)
    rep = {
        "n": int(same.size),
        "divergent": int((~same).sum()),
        "matched_bad": int((same & ~ok).sum()),
        "divergent_fraction": float((~same).mean()),
    }
    if gpu_img is not None:
        clean = same.all(axis=-1)
        pix_ok = rel_ok(gpu_img, ref_img).all(axis=-1)
        rep["pixels"] = int(clean.size)
        rep["divergent_pixels"] = int((~clean).sum())
        rep["clean_pixel_fraction_ok"] = float(pix_ok[clean].mean()) if clean.any() else 1.0
        rep["all_pixel_fraction_ok"] = float(pix_ok.mean())
    return rep
