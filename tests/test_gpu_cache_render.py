"""Cache-terminated rendering, its adjoint and online training records vs the FP64 oracle."""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

from parity import PIXEL_FRACTION, cosine, pixel_ok_fraction, rel_ok

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BOX = ((-1.0, 0.0, -1.0), (1.0, 2.0, 1.0))


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_01284_gb300 import abi, render
    abi.load()
    return render


def _settings(R, scene, **kw):
    cam = scene.cameras[0]
    base = dict(width=cam.width, height=cam.height, spp=4, max_depth=4, seed=7)
    base.update(kw)
    return R.RenderSettings(**base)


@pytest.mark.parametrize("bounce", [1, 2])
def test_zero_cache_equals_truncated_paths(R, oracle_mod, bounce):
    """A cache that predicts 0 turns the estimator into the path tracer cut at the
    termination vertex, i.e. max_depth = bounce (the Cornell box has no delta BSDFs)."""
    sc = S.cornell()
    ds = R.DeviceScene(sc)
    cache = R.RadianceCache(*BOX, batch=64, max_queries=64 * 64 * 4, init_weights=np.zeros(S.MLP_N_PARAMS))
    st = _settings(R, sc, cache=cache.handle, cache_bounce=bounce)
    img = ds.forward(st)[0].cpu().numpy()
    plain = ds.forward(_settings(R, sc, max_depth=bounce))[0].cpu().numpy()
    assert np.allclose(img, plain, rtol=1e-6, atol=0)
    osc = oracle_mod.OracleScene(sc)
    ref = oracle_mod.render(osc, oracle_mod.render_in(sc.cameras[0], 4, bounce, 7))
    frac, _ = pixel_ok_fraction(img, ref)
    assert frac >= PIXEL_FRACTION


@pytest.mark.parametrize("bounce", [1, 2])
def test_cache_render_matches_oracle(R, oracle_mod, bounce):
    sc = S.cornell()
    # non-negative weights of mean ~1/64 keep every activation and output positive
    # and of order one, so relative errors are well conditioned (no ReLU/clamp flips)
    W = np.abs(S.mlp_init_weights(31)) * 0.1
    ds = R.DeviceScene(sc)
    cache = R.RadianceCache(*BOX, batch=64, max_queries=64 * 64 * 4, init_weights=W)
    img = ds.forward(_settings(R, sc, cache=cache.handle, cache_bounce=bounce))[0].cpu().numpy()
    osc = oracle_mod.OracleScene(sc)
    ref = oracle_mod.render_cached(osc, oracle_mod.render_in(sc.cameras[0], 4, 4, 7), W, *BOX, bounce)
    # The network sees BF16-rounded features of FP32 (GPU) vs FP64 (oracle) hit
    # points: a 1e-7 relative position difference moves sin(32 pi x) by ~1e-5, which
    # flips the BF16 rounding (2^-9 relative) of a feature in ~1 % of cases, i.e.
    # in a large share of the 64-feature queries.  Bound: the MLP output moves by
    # about one BF16 step of its inputs, so 1e-2 relative per pixel.
    frac, ok = pixel_ok_fraction(img, ref, rel=1e-2)
    err = np.abs(img - ref) / (np.abs(ref) + 1e-3 * np.abs(ref).mean())
    print(f"bounce {bounce}: pixels within 1e-2: {frac:.5f}, within 1e-4: {pixel_ok_fraction(img, ref)[0]:.4f}, "
          f"max rel err {err.max():.2e}")
    assert frac >= PIXEL_FRACTION
    assert err.max() < 0.2


def test_cache_adjoint_matches_oracle(R, oracle_mod):
    """Albedo gradient of the cache-terminated estimator (cache radiance detached)."""
    sc = S.cornell()
    W = S.mlp_init_weights(32) * 0.5
    ds = R.DeviceScene(sc)
    cache = R.RadianceCache(*BOX, batch=64, max_queries=64 * 64 * 4, init_weights=W)
    st = _settings(R, sc, cache=cache.handle, cache_bounce=2)
    osc = oracle_mod.OracleScene(sc)
    r = oracle_mod.render_in(sc.cameras[0], 4, 4, 7)
    I = oracle_mod.render_cached(osc, r, W, *BOX, 2)
    gi = 2 * (I - 0.3) / I.size
    g = torch.zeros_like(ds.albedo)
    ds.backward(st, torch.as_tensor(gi[None], dtype=torch.float32, device="cuda"), g_albedo=g)
    torch.cuda.synchronize()
    sel = [(0, a, c, 0) for a in range(5) for c in range(3)]
    ref = oracle_mod.grad_dual_cached(osc, r, W, *BOX, 2, gi, sel)
    got = g.cpu().numpy().ravel()
    c = cosine(got, ref)
    print("cache adjoint cosine", c, "max rel", np.abs(got - ref).max() / np.abs(ref).max())
    assert c >= 0.9999
    assert np.abs(got - ref).max() < 2e-3 * np.abs(ref).max()


def test_training_records_match_oracle(R, oracle_mod):
    sc = S.cornell(width=32, height=32)
    ds = R.DeviceScene(sc)
    cache = R.RadianceCache(*BOX, batch=256, max_records=100000, max_paths=32 * 32 * 2, init_weights=S.mlp_init_weights(5))
    st = _settings(R, sc, spp=2, max_depth=4, seed=9)
    n = cache.train(ds, st, steps=0)
    raw, tgt, meta = cache.read_records(n)
    osc = oracle_mod.OracleScene(sc)
    oraw, otgt, ometa = oracle_mod.train_records(osc, oracle_mod.render_in(sc.cameras[0], 2, 4, 9), 100000)
    assert abs(n - len(oraw)) <= max(2, len(oraw) // 1000)
    key = lambda m: m[:, 0].astype(np.int64) * 16 + m[:, 1]
    gi, oi = np.argsort(key(meta)), np.argsort(key(ometa))
    gk, ok_ = key(meta)[gi], key(ometa)[oi]
    common, ga, oa = np.intersect1d(gk, ok_, return_indices=True)
    assert len(common) >= 0.999 * len(ok_)
    gr, orw = raw[gi][ga], oraw[oi][oa]
    gt, ot = tgt[gi][ga], otgt[oi][oa]
    assert np.mean(np.all(np.abs(gr - orw) < 1e-4, axis=1)) > 0.999
    good = rel_ok(gt, ot, rel=1e-3).all(axis=1)
    print("records", n, "oracle", len(oraw), "targets within 1e-3:", good.mean())
    assert good.mean() > 0.995


def test_trained_cache_lowers_error_at_equal_spp(R):
    """Online training on the renderer's own paths, then a cache-terminated render has
    lower MSE than plain path tracing at the same spp (vs a 1024-spp plain reference)."""
    sc = S.cornell(width=128, height=128)
    ds = R.DeviceScene(sc)
    ref = ds.forward(_settings(R, sc, spp=1024, max_depth=4, seed=1))[0]
    cache = R.RadianceCache(*BOX, batch=16384, max_queries=128 * 128 * 4, max_records=400000,
                            max_paths=128 * 128, lr=5e-3, init_weights=S.mlp_init_weights(7))
    for it in range(60):
        cache.train(ds, _settings(R, sc, spp=1, max_depth=4, seed=1000 + it), steps=4)
    plain = ds.forward(_settings(R, sc, spp=4, max_depth=4, seed=77))[0]
    cached = ds.forward(_settings(R, sc, spp=4, max_depth=4, seed=77, cache=cache.handle, cache_bounce=1))[0]
    # pixels that do not see the light: its edge pixels carry anti-aliasing variance
    # (radiance 15) that is the same for both estimators
    m = (ref.amax(dim=-1, keepdim=True) < 1.0).float()
    mse_plain = float((((plain - ref) ** 2) * m).sum() / (3 * m.sum()))
    mse_cache = float((((cached - ref) ** 2) * m).sum() / (3 * m.sum()))
    print(f"loss {cache.last_loss():.4f}  MSE (indirect pixels) plain {mse_plain:.6f} cache {mse_cache:.6f}")
    assert mse_cache < 0.5 * mse_plain
