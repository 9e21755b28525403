"""The radiance cache's input encoding on the GPU (pt_cache_encode) against the exact
sin / cos of the same FP32 inputs.

The BF16 feature is a rounding decision, so both sides take it from the same input:
the test forms the FP32 normalised coordinate x exactly as the kernel does ((raw - lo)
* (1 / (hi - lo)) in FP32, (w + 1) / 2 for unit vectors; 2^(k+1) x is exact), then
evaluates sin / cos(pi 2^k x) in FP64 after an exact reduction of the argument mod 2,
and rounds that to BF16 (nearest, ties to even).  Octave 0 of each coordinate is a
reduction and polynomial pair within a few FP32 ulp: its features must equal that
rounding, except where the exact value lies within 4 ulp of the midpoint between two
BF16 neighbours.  Octave d > 0 comes from d double-angle steps, whose error bound is
absolute (2^d * 4 * 2^-24, Euclidean, for the pair): its features must be the BF16
rounding of some value within that bound of the exact one.  Against the FP64 oracle's
encoding (FP64 normalisation of the input) the features agree to BF16 rounding plus
the FP32 input rounding amplified by the octave, plus that bound."""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

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


def _gpu_features(abi, raw, box=BOX):
    n = raw.shape[0]
    h = abi.pt_cache_create(*box, batch=64)
    try:
        d_raw = torch.as_tensor(np.ascontiguousarray(raw, np.float32), device="cuda")
        d_f = torch.full((max(n, 1), 64), -1, dtype=torch.int16, device="cuda")
        abi.pt_cache_encode(h, d_raw, d_f, n)
        torch.cuda.synchronize()
        return d_f[:n].cpu().numpy().view(np.uint16)
    finally:
        abi.pt_cache_destroy(h)


def _bf16_value(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _bf16_rne(v):
    """BF16 bits of float64 values: to FP32 (nearest), then to BF16 (nearest even)."""
    f = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    rounded = (f + 0x7FFF + ((f >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def _exact_inputs(raw, box=BOX):
    """The FP32 coordinates the kernel encodes, per feature word (sin, cos argument
    t = 2^(k+1) x, so that the pair is sin / cos(pi t / 2))."""
    raw = raw.astype(np.float32)
    lo = np.asarray(box[0], np.float32)
    inv = np.float32(1.0) / (np.asarray(box[1], np.float32) - lo)
    t = np.zeros((raw.shape[0], 30), np.float64)
    with np.errstate(invalid="ignore", over="ignore"):
        xp = np.clip((raw[:, :3] - lo) * inv, np.float32(-32768), np.float32(32768))
        xp[np.isnan(raw[:, :3])] = np.nan
        for a in range(3):
            for k in range(6):
                t[:, 6 * a + k] = xp[:, a].astype(np.float64) * 2.0 ** (k + 1)
        xd = np.float32(0.5) * (raw[:, 3:9] + np.float32(1.0))
        xd = np.clip(xd, np.float32(-32768), np.float32(32768))
        for a in range(6):
            t[:, 18 + 2 * a] = xd[:, a].astype(np.float64) * 2.0
            t[:, 19 + 2 * a] = xd[:, a].astype(np.float64) * 4.0
    return t


def _exact_pairs(t):
    """sin / cos(pi t / 2) in FP64 with an exact reduction: period 4 in t, then the
    nearest integer q (a quarter turn each), so that multiples of 1/2 turn give exact
    zeros and ones (pi itself is not exact in FP64)."""
    r = np.fmod(t, 4.0)
    q = np.rint(r)
    a = 0.5 * np.pi * (r - q)
    su, cu = np.sin(a), np.cos(a)
    qi = np.mod(np.nan_to_num(q), 4).astype(int)
    s = np.choose(qi, [su, cu, -su, -cu])
    c = np.choose(qi, [cu, -su, -cu, su])
    return s, c


# Doubling steps behind each of the 64 features: position octave k (0..5), direction
# and normal octave 0 or 1, none for roughness and the constant features.
DOUBLINGS = np.zeros(64, int)
DOUBLINGS[:36] = np.tile(np.repeat(np.arange(6), 2), 3)
DOUBLINGS[36:60] = np.tile(np.repeat(np.arange(2), 2), 6)


def _check(got_bits, exact, ulps=4.0):
    """Return (features that differ from the correctly rounded BF16, those of them
    outside the error model, those of octave 0 or constant).  A feature fits the model
    when it is the BF16 rounding of a value within E of the exact one: E = `ulps` FP32
    ulp of the exact value where no doubling step is involved, 2^d * 4 * 2^-24 after d
    steps."""
    want = _bf16_rne(exact)
    g = _bf16_value(got_bits)
    w = _bf16_value(want)
    both_nan = np.isnan(g) & np.isnan(w)
    differ = (g != w) & ~both_nan
    d = np.broadcast_to(DOUBLINGS[: exact.shape[1]], exact.shape)
    with np.errstate(invalid="ignore"):
        rel = ulps * np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
        tol = np.where(d > 0, 2.0 ** d * 4 * 2.0 ** -24, rel)
        lo = _bf16_value(_bf16_rne(exact - tol))
        hi = _bf16_value(_bf16_rne(exact + tol))
        inside = (g >= lo) & (g <= hi)
    bad = differ & ~inside
    return int(differ.sum()), int(bad.sum()), int((differ & (d == 0)).sum())


def _compare(raw, got):
    t = _exact_inputs(raw)
    s, c = _exact_pairs(t)
    exact = np.empty((raw.shape[0], 64))
    exact[:, 0:60:2] = s
    exact[:, 1:60:2] = c
    exact[:, 60] = raw[:, 9].astype(np.float32)
    exact[:, 61:] = 1.0
    return _check(got, exact), exact


@pytest.mark.parametrize("n", [1, 255, 256, 257, 200_003])
def test_encoding_is_the_correctly_rounded_bf16_of_the_fp32_inputs(abi, n):
    raw, _ = S.random_cache_records(n, 5, *BOX)
    got = _gpu_features(abi, raw)
    (n_diff, n_bad, n_diff0), _ = _compare(raw, got)
    print(f"n={n}: {n_diff} of {got.size} features differ from the correctly rounded BF16 "
          f"({n_diff0} without doubling steps), {n_bad} outside the error model")
    assert n_bad == 0
    assert n_diff0 <= max(2, 2e-4 * got.size)
    assert n_diff <= max(2, 2e-3 * got.size)


def test_quadrant_boundaries_signs_and_clamp(abi):
    """Arguments on and next to multiples of 1/2 (every quadrant switch of every
    octave), points outside the box (negative x, far outside: clamped to 2^15 box
    extents), unit vectors with components exactly +-1 and 0, and a NaN position."""
    rng = np.random.default_rng(8)
    lo = np.asarray(BOX[0], np.float32)
    ext = np.asarray(BOX[1], np.float32) - lo
    grid = (np.arange(-128, 129) / 64.0).astype(np.float32)         # x on multiples of 1/64
    xs = np.concatenate([grid, np.nextafter(grid, np.float32(10)), np.nextafter(grid, np.float32(-10)),
                         np.asarray([-3.5, 5.25, 1e4, -3e4, 1e6, -1e9], np.float32)])
    n = xs.size
    raw = np.zeros((n, 10), np.float32)
    raw[:, :3] = lo + xs[:, None] * ext                              # the same x on every axis
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d[:6] = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]
    raw[:, 3:6] = d
    raw[:, 6:9] = -d
    raw[:, 9] = rng.uniform(0, 1, n)
    raw = np.concatenate([raw, raw[:1]])
    raw[-1, 1] = np.nan
    got = _gpu_features(abi, raw)
    (n_diff, n_bad, _), exact = _compare(raw[:-1], got[:-1])
    print(f"boundary set: {n_diff} differ from the correctly rounded BF16, {n_bad} outside the error model")
    assert n_bad == 0
    # far outside the box the coordinate is clamped: sin / cos of 2^k pi 2^15 = (0, 1)
    far = np.where(np.abs(xs) >= 32768)[0]
    assert np.all(_bf16_value(got[far, 0:36:2]) == 0.0) and np.all(_bf16_value(got[far, 1:36:2]) == 1.0)
    # NaN in y: the y octaves are NaN, the x and z octaves and the rest are finite
    nan_row = _bf16_value(got[-1])
    assert np.all(np.isnan(nan_row[12:24])) and np.all(np.isfinite(np.delete(nan_row, np.arange(12, 24))))
    assert np.all(nan_row[61:] == 1.0)


def test_matches_the_oracle_encoding_within_input_rounding(abi, oracle_mod):
    """Against the FP64 oracle (FP64 normalisation, no FP32 rounding of the input; its
    features are BF16-rounded too): the two roundings differ by at most one BF16 step
    (2^-7 relative at most) plus the FP32 input rounding amplified by the octave
    (2^k pi |dx|) and the doubling steps' bound (2^k * 4 * 2^-24)."""
    raw, _ = S.random_cache_records(4096, 9, *BOX)
    got = _bf16_value(_gpu_features(abi, raw))
    ref = oracle_mod.nrc_encode(raw, *BOX)
    k = DOUBLINGS.astype(float)
    bound = 2.0 ** -7 * np.maximum(np.abs(ref), np.abs(got)) + 2.0 ** k * (np.pi + 1) * 4 * 2.0 ** -24 + 1e-30
    err = np.abs(got - ref)
    print(f"max |gpu - oracle| / bound: {(err / bound).max():.3f}")
    assert np.all(err <= bound)


def test_encode_argument_checks(abi):
    h = abi.pt_cache_create(*BOX, batch=64)
    try:
        raw = torch.zeros((4, 10), device="cuda")
        f = torch.zeros((5, 64), dtype=torch.int16, device="cuda")
        abi.pt_cache_encode(h, raw, f, 0)                            # empty: nothing to do
        with pytest.raises(abi.PtError):
            abi.pt_cache_encode(h, raw, f, -1)
        with pytest.raises(abi.PtError):
            abi.pt_cache_encode(h, raw, f.view(-1)[1:], 4)          # not 16-byte aligned
    finally:
        abi.pt_cache_destroy(h)
