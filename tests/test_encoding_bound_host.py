"""Host check of the error bound behind the radiance cache's higher octaves.

The kernels form octave k + 1 of the frequency encoding from octave k by the
double-angle step (sin 2a, cos 2a) = (2 s c, c^2 - s^2), in FP32: s' = (s + s) c and
c' = fma(c, c, -(s s)).  In that form the step's Jacobian is twice a rotation, so an
error already in the pair grows by exactly a factor 2 per octave, and each step adds at
most 2^-25 to s and 2^-24 to c of rounding; from a start within 2^-23 per component the
pair stays within 2^k * 4 * 2^-24 (Euclidean) of the exact one after k steps.  This test
runs the same FP32 operations in numpy (one rounding per operation, the FMA through
float64, where c*c is exact) from the correctly rounded FP32 pair of octave 0 and
checks the bound over five octaves against FP64 values of the same FP32 argument; it
also checks that the 1 - 2 s^2 form, whose Jacobian is not a scaled rotation, exceeds
it, which is why the kernels use c^2 - s^2."""
import numpy as np

F32 = np.float32


def _step(s, c):
    s2 = ((s + s).astype(F32) * c).astype(F32)
    ss = (s * s).astype(F32)
    c2 = (c.astype(np.float64) * c.astype(np.float64) - ss.astype(np.float64)).astype(F32)
    return s2, c2


def _step_one_minus(s, c):
    t = (s + s).astype(F32)
    s2 = (t * c).astype(F32)
    c2 = (1.0 - t.astype(np.float64) * s.astype(np.float64)).astype(F32)
    return s2, c2


def _exact(x, k):
    """sin / cos(2^k pi x) in FP64 after an exact reduction: t = 2^(k+1) x modulo 4
    (quarter turns), q its nearest integer, then the pair of the remainder rotated by q
    quarter turns, so that multiples of a quarter turn give exact zeros and ones."""
    t = np.fmod(np.ldexp(x.astype(np.float64), k + 1), 4.0)
    q = np.rint(t)
    a = 0.5 * np.pi * (t - q)
    su, cu = np.sin(a), np.cos(a)
    qi = np.mod(q, 4).astype(int)
    return np.choose(qi, [su, cu, -su, -cu]), np.choose(qi, [cu, -su, -cu, su])


def _worst(step, x):
    s0, c0 = _exact(x, 0)
    s, c = s0.astype(F32), c0.astype(F32)
    worst = []
    for k in range(1, 6):
        s, c = step(s, c)
        es, ec = _exact(x, k)
        worst.append(np.hypot(s - es, c - ec).max() / (2.0 ** k * 4 * 2.0 ** -24))
    return worst


def test_double_angle_octaves_stay_within_the_stated_bound():
    rng = np.random.default_rng(2202)
    x = np.concatenate([rng.uniform(0, 1, 400_000), rng.uniform(-3, 3, 100_000),
                        np.arange(0, 4097) / 4096.0]).astype(F32)
    worst = _worst(_step, x)
    print("max error / bound per octave:", [f"{w:.3f}" for w in worst])
    assert max(worst) <= 1.0
    assert max(worst) > 0.1          # the bound is not vacuous


def test_one_minus_two_s_squared_form_breaks_the_bound():
    rng = np.random.default_rng(1284)
    x = rng.uniform(0, 1, 400_000).astype(F32)
    worst = _worst(_step_one_minus, x)
    print("1 - 2 s^2 form, max error / bound per octave:", [f"{w:.3f}" for w in worst])
    assert max(worst) > 1.0


def test_exact_quarter_turns_stay_exact():
    """At multiples of 1/2 turn every octave's pair is exact (0 and +-1 are fixed
    points of the step), as the clamped far-outside coordinates need."""
    x = (np.arange(-64, 65) / 2.0).astype(F32)
    s0, c0 = _exact(x, 0)
    s, c = s0.astype(F32), c0.astype(F32)
    for k in range(1, 6):
        s, c = _step(s, c)
        es, ec = _exact(x, k)
        assert np.array_equal(s.astype(np.float64), np.round(es)) and np.array_equal(c.astype(np.float64), np.round(ec))
