"""GPU parity of the radiance-cache MLP kernels (BF16 tensor cores) vs the FP64 oracle."""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

from parity import cosine

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BOX = ((-1.0, 0.0, -1.0), (1.0, 2.0, 1.0))


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_01284_gb300 import abi
    abi.load()
    return abi


def _rel_err(a, b):
    scale = np.abs(b).mean()
    return np.abs(a - b) / (np.abs(b) + 0.05 * scale)


# Octave of each encoded feature: position octave k at features 12 a + 2 k (+1),
# direction and normal octaves 0 and 1, none for roughness and the constants.
OCTAVE = np.zeros(64)
OCTAVE[:36] = np.tile(np.repeat(np.arange(6), 2), 3)
OCTAVE[36:60] = np.tile(np.repeat(np.arange(2), 2), 6)


def _bf16(v):
    """Values of the BF16 roundings (to FP32 nearest, then BF16 nearest even)."""
    f = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    b = (((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def _unique_records(raw, oracle_enc, box=BOX):
    """Records whose 64 BF16 features the kernel and the oracle decide alike.

    Each feature is a quantised code chosen by floating point: the kernel rounds an
    FP32 sin / cos of an FP32 coordinate (within 2^k * 4 * 2^-24 of the exact pair of
    that coordinate at octave k), the oracle an FP64 one.  Where the FP64 value lies
    within the two sides' difference (2^k * (pi + 1) * 4 * 2^-24: the FP32 rounding of
    the coordinate amplified by the octave, plus the kernel's bound) of a BF16
    rounding boundary, both codes are correct, and the network's output differs by
    what one step of that feature makes of it.  The FP64 features here only locate
    those boundaries; they are checked against the oracle's rounded features first.
    The test records lie inside the box (no clamping)."""
    lo, hi = np.asarray(box[0], np.float64), np.asarray(box[1], np.float64)
    raw = raw.astype(np.float64)
    x = (raw[:, :3] - lo) / (hi - lo)
    xd = 0.5 * (raw[:, 3:9] + 1.0)
    v = np.empty((raw.shape[0], 64))
    for a in range(3):
        for k in range(6):
            v[:, 12 * a + 2 * k] = np.sin(2.0 ** k * np.pi * x[:, a])
            v[:, 12 * a + 2 * k + 1] = np.cos(2.0 ** k * np.pi * x[:, a])
    for a in range(6):
        for k in range(2):
            v[:, 36 + 4 * a + 2 * k] = np.sin(2.0 ** k * np.pi * xd[:, a])
            v[:, 37 + 4 * a + 2 * k] = np.cos(2.0 ** k * np.pi * xd[:, a])
    v[:, 60] = raw[:, 9]
    v[:, 61:] = 1.0
    m = 2.0 ** OCTAVE * (np.pi + 1) * 4 * 2.0 ** -24
    either_way = _bf16(v - m) != _bf16(v + m)
    assert np.all((_bf16(v) == oracle_enc) | either_way)
    return ~either_way.any(1)


def _check_outputs(got, ref, unique, tag=""):
    """All records: finite, median error of a BF16 network.  Records with unique
    features: the 99th percentile at FP32 accumulation-order level (measured near
    3e-7).  The others: bounded by a few feature steps."""
    err = _rel_err(got, ref)
    print(f"{tag} median rel err {np.median(err):.2e}; unique-feature records {unique.mean():.2f}, "
          f"p99 {np.quantile(err[unique], 0.99) if unique.any() else 0:.2e}; "
          f"others max {err[~unique].max() if (~unique).any() else 0:.2e}")
    assert np.all(np.isfinite(got))
    assert np.median(err) < 2e-3
    if unique.any():
        assert np.quantile(err[unique], 0.99) < 1e-4
    if (~unique).any():
        assert err[~unique].max() < 0.5


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("n", [1, 17, 127, 128, 129, 5000])
def test_inference_matches_oracle(abi, oracle_mod, n, engine):
    """Ragged sizes (1, 17 = one mma.sync warp tile + 1 row, 127/128/129 around one
    tcgen05 tile, 5000) through the C ABI, both inference engines."""
    raw, _ = S.random_cache_records(n, 11)
    W = S.mlp_init_weights(12)
    h = abi.pt_cache_create(*BOX, batch=64, init_weights=W)
    try:
        abi.pt_cache_set_engine(h, engine)
        d_raw = torch.as_tensor(raw, device="cuda")
        d_out = torch.full((n, 3), float("nan"), device="cuda")
        abi.pt_cache_query(h, d_raw, d_out, n)
        torch.cuda.synchronize()
        assert abi.pt_cache_status(h) == abi.PT_OK
        got = d_out.cpu().numpy().astype(np.float64)
    finally:
        abi.pt_cache_destroy(h)
    enc = oracle_mod.nrc_encode(raw, *BOX)
    ref = oracle_mod.mlp_forward(W.astype(np.float64), enc)
    _check_outputs(got, ref, _unique_records(raw, enc), f"n={n}")


def test_gradient_and_loss_match_oracle(abi, oracle_mod):
    """One optimisation step with beta1 = beta2 = 0, lr = eps = 1e6 turns Adam into
    w1 = w0 - g * 1e6 / (|g| + 1e6), exposing the kernels' weight gradient."""
    n = 4096
    raw, tgt = S.random_cache_records(n, 13)
    W0 = S.mlp_init_weights(14)
    h = abi.pt_cache_create(*BOX, batch=n, lr=1e6, beta1=0.0, beta2=0.0, eps=1e6, init_weights=W0)
    try:
        d_raw = torch.as_tensor(raw, device="cuda")
        d_t = torch.as_tensor(tgt, device="cuda")
        abi.pt_cache_train_records(h, d_raw, d_t, n, 1)
        loss_gpu = abi.pt_cache_last_loss(h)
        W1 = abi.pt_cache_get_weights(h)
    finally:
        abi.pt_cache_destroy(h)
    g_gpu = (W0.astype(np.float64) - W1.astype(np.float64))
    enc = oracle_mod.nrc_encode(raw, *BOX)
    loss_ref, g_ref, _ = oracle_mod.mlp_loss_grad(W0.astype(np.float64), enc, tgt)
    g_gpu = g_gpu * (np.abs(g_ref) + 1e6) / 1e6
    c = cosine(g_gpu, g_ref)
    print(f"loss gpu {loss_gpu:.6f} oracle {loss_ref:.6f}; gradient cosine {c:.6f}")
    assert abs(loss_gpu - loss_ref) < 1e-2 * loss_ref
    assert c > 0.999
    for l in range(6):
        sl = slice(l * 4096, (l + 1) * 4096) if l < 5 else slice(5 * 4096, None)
        assert cosine(g_gpu[sl], g_ref[sl]) > 0.995, l


def test_training_converges_like_oracle(abi, oracle_mod):
    n = 1024
    raw, tgt = S.random_cache_records(n, 15)
    W0 = S.mlp_init_weights(16)
    h = abi.pt_cache_create(*BOX, batch=n, lr=5e-3, init_weights=W0)
    losses = []
    try:
        d_raw = torch.as_tensor(raw, device="cuda")
        d_t = torch.as_tensor(tgt, device="cuda")
        for _ in range(40):
            abi.pt_cache_train_records(h, d_raw, d_t, n, 1)
            losses.append(abi.pt_cache_last_loss(h))
    finally:
        abi.pt_cache_destroy(h)
    enc = oracle_mod.nrc_encode(raw, *BOX)
    W = W0.astype(np.float64)
    m, v = np.zeros_like(W), np.zeros_like(W)
    ref = []
    for t in range(1, 41):
        loss, g, _ = oracle_mod.mlp_loss_grad(W, enc, tgt)
        ref.append(loss)
        oracle_mod.mlp_adam(W, g, m, v, t, lr=5e-3)
    print("gpu", losses[0], losses[-1], "oracle", ref[0], ref[-1])
    assert abs(losses[0] - ref[0]) < 1e-2 * ref[0]
    assert losses[-1] < 0.5 * losses[0]
    assert losses[-1] < 1.5 * ref[-1] + 1e-3


def test_engines_agree_on_large_batch(abi):
    """tcgen05 and mma.sync inference on 300,001 queries (2,344 MMA tiles + a ragged
    one): the same BF16 rounding points, FP32 accumulation in a different order."""
    n = 300_001
    raw, _ = S.random_cache_records(n, 21)
    W = S.mlp_init_weights(13)
    h = abi.pt_cache_create(*BOX, batch=64, init_weights=W)
    try:
        d_raw = torch.as_tensor(raw, device="cuda")
        out = []
        for engine in (abi.PT_CACHE_TCGEN05, abi.PT_CACHE_MMA_SYNC):
            abi.pt_cache_set_engine(h, engine)
            d_out = torch.full((n, 3), float("nan"), device="cuda")
            abi.pt_cache_query(h, d_raw, d_out, n)
            torch.cuda.synchronize()
            assert abi.pt_cache_status(h) == abi.PT_OK
            out.append(d_out.cpu().numpy().astype(np.float64))
    finally:
        abi.pt_cache_destroy(h)
    a, b = out
    assert np.all(np.isfinite(a))
    err = _rel_err(a, b)
    print(f"tcgen05 vs mma.sync: median {np.median(err):.2e} p99.9 {np.quantile(err, 0.999):.2e} max {err.max():.2e}")
    assert np.median(err) < 1e-6  # same features and rounding points; FP32 accumulation order may differ
    assert np.quantile(err, 0.999) < 1e-4


def test_training_engines_agree(abi):
    """One optimisation step (Adam turned into w - g * 1e6 / (|g| + 1e6)) with the
    tcgen05 and the mma.sync forward/backward kernels from the same weights on a
    ragged batch of 5,000 records: the same loss and weight gradients."""
    n = 5000
    raw, tgt = S.random_cache_records(n, 23)
    W0 = S.mlp_init_weights(24)
    res = []
    for engine in (abi.PT_CACHE_TCGEN05, abi.PT_CACHE_MMA_SYNC):
        h = abi.pt_cache_create(*BOX, batch=5056, lr=1e6, beta1=0.0, beta2=0.0, eps=1e6, init_weights=W0)
        try:
            abi.pt_cache_set_engine(h, engine)
            abi.pt_cache_train_records(h, torch.as_tensor(raw, device="cuda"), torch.as_tensor(tgt, device="cuda"),
                                       n, 1)
            assert abi.pt_cache_status(h) == abi.PT_OK
            res.append((abi.pt_cache_last_loss(h), W0.astype(np.float64) - abi.pt_cache_get_weights(h)))
        finally:
            abi.pt_cache_destroy(h)
    (l_tc, g_tc), (l_mma, g_mma) = res
    c = cosine(g_tc, g_mma)
    print(f"loss tcgen05 {l_tc:.7f} mma.sync {l_mma:.7f}; update cosine {c:.9f}")
    assert abs(l_tc - l_mma) <= 1e-5 * abs(l_mma)
    assert c > 0.99999


def test_bounded_wait_timeout_is_reported(abi, oracle_mod):
    """Failure injection without a GPU fault: with a wait limit of 0 polls every
    tcgen05 kernel gives up on its first MMA step, reports PT_ERR_TIMEOUT through
    the status word, lets the MMA in flight finish and frees its tensor memory; the
    next calls with the default limit are correct (the context is intact)."""
    n = 1000
    raw, tgt = S.random_cache_records(n, 31)
    W = S.mlp_init_weights(32)
    h = abi.pt_cache_create(*BOX, batch=1024, init_weights=W)
    try:
        d_raw = torch.as_tensor(raw, device="cuda")
        d_t = torch.as_tensor(tgt, device="cuda")
        abi.pt_cache_set_wait_limit(h, 0)
        out = torch.full((n, 3), float("nan"), device="cuda")
        abi.pt_cache_query(h, d_raw, out, n)
        assert abi.pt_cache_status(h) == abi.PT_ERR_TIMEOUT
        assert torch.isnan(out).all()  # nothing written past the failed step
        abi.pt_cache_train_records(h, d_raw, d_t, n, 1)
        assert abi.pt_cache_status(h) == abi.PT_ERR_TIMEOUT
        # back to the default: correct results, status clear
        abi.pt_cache_set_wait_limit(h, abi.PT_CACHE_WAIT_LIMIT_DEFAULT)
        abi.pt_cache_set_weights(h, W)
        out = torch.full((n, 3), float("nan"), device="cuda")
        abi.pt_cache_query(h, d_raw, out, n)
        assert abi.pt_cache_status(h) == abi.PT_OK
        got = out.cpu().numpy().astype(np.float64)
    finally:
        abi.pt_cache_destroy(h)
    ref = oracle_mod.mlp_forward(W.astype(np.float64), oracle_mod.nrc_encode(raw, *BOX))
    err = _rel_err(got, ref)
    assert np.median(err) < 2e-3


def test_training_checkpoint_resume(abi, tmp_path):
    """Save after 3 Adam steps, reload into a fresh cache, 3 more steps: the same as
    6 uninterrupted steps (weights, moments and the step count are restored; the
    split-K gradient sums are atomics, so equal up to FP32 summation order)."""
    from paper_2202_01284_gb300.render import RadianceCache
    n = 2048
    raw, tgt = S.random_cache_records(n, 41)
    W0 = S.mlp_init_weights(42)
    d_raw, d_t = torch.as_tensor(raw, device="cuda"), torch.as_tensor(tgt, device="cuda")

    def steps(c, k):
        for _ in range(k):
            c.train_records(d_raw, d_t, steps=1)
        torch.cuda.synchronize()
    a = RadianceCache(*BOX, batch=n, lr=5e-3, init_weights=W0)
    steps(a, 6)
    want = a.weights()
    a.close()
    b = RadianceCache(*BOX, batch=n, lr=5e-3, init_weights=W0)
    steps(b, 3)
    b.save(tmp_path / "cache.bin")
    b.close()
    c = RadianceCache(*BOX, batch=n, lr=5e-3, init_weights=S.mlp_init_weights(7))
    c.load(tmp_path / "cache.bin")
    assert abi.pt_cache_get_state(c.handle)[3] == 3
    steps(c, 3)
    got = c.weights()
    assert abi.pt_cache_get_state(c.handle)[3] == 6
    c.close()
    assert np.allclose(got, want, rtol=1e-4, atol=1e-6), np.abs(got - want).max()


@pytest.mark.parametrize("engine", [0, 1])
def test_averaged_weights_follow_the_recurrence_and_serve_queries(abi, oracle_mod, engine):
    """With ema = 0.8, after every Adam step the average is A = 0.8 A + 0.2 W (A
    starting at the initial weights), and queries evaluate the network with A, not W."""
    from paper_2202_01284_gb300.render import RadianceCache
    n = 2048
    raw, tgt = S.random_cache_records(n, 51)
    W0 = S.mlp_init_weights(52)
    d_raw, d_t = torch.as_tensor(raw, device="cuda"), torch.as_tensor(tgt, device="cuda")
    c = RadianceCache(*BOX, batch=n, lr=5e-3, init_weights=W0, ema=0.8)
    try:
        abi.pt_cache_set_engine(c.handle, engine)
        A = W0.astype(np.float64)
        assert np.array_equal(c.average(), W0)
        for _ in range(5):
            c.train_records(d_raw, d_t, steps=1)
            torch.cuda.synchronize()
            A = 0.8 * A + 0.2 * c.weights().astype(np.float64)
        got_A = c.average().astype(np.float64)
        assert np.allclose(got_A, A, rtol=1e-5, atol=1e-7), np.abs(got_A - A).max()
        assert np.abs(got_A - c.weights()).max() > 1e-4           # the average lags the weights
        q = c.query(torch.as_tensor(raw[:300], device="cuda")).cpu().numpy().astype(np.float64)
        assert abi.pt_cache_status(c.handle) == abi.PT_OK
    finally:
        c.close()
    enc = oracle_mod.nrc_encode(raw[:300], *BOX)
    _check_outputs(q, oracle_mod.mlp_forward(got_A, enc), _unique_records(raw[:300], enc))
    with pytest.raises(abi.PtError):
        RadianceCache(*BOX, batch=64, ema=1.0)
