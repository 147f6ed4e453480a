"""The compensated FP32 evaluation of a soft core's Cayley coefficient
b = 1/(1 + i theta), theta = th0 + K/sqrt(R), as the FP32 kernels perform it
(rsqrt estimate plus one Newton step, TwoSum, the FMA split of 1 + theta^2, a
refined reciprocal), emulated step by step in NumPy float32.

The emulation rounds every operation to FP32 (an FMA is formed in float64,
where the product of two floats is exact, and rounded once more to float32),
and the hardware estimates (reciprocal square root, reciprocal) are replaced
by FP32 values with a random relative error of up to 2^-22, about the
accuracy of the approximate instructions.  The claim checked: b_hi + b_lo has
a relative error of ~1e-13 and |2b - 1| = 1 to ~2e-13, for shallow and deep
cores (|theta| up to ~10), so the FP32 coefficients neither bias the phase of
a value nor break the conservation of E (Sect. 2, the Cayley form of Eqs.
ss1-ss4).
"""
import numpy as np
import pytest

f32 = np.float32


def fl(x):
    return np.asarray(x, dtype=np.float64).astype(f32)


def add(a, b):
    return fl(np.float64(a) + np.float64(b))


def sub(a, b):
    return fl(np.float64(a) - np.float64(b))


def mul(a, b):
    return fl(np.float64(a) * np.float64(b))


def fma(a, b, c):
    return fl(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    e = add(sub(a, sub(s, bb)), sub(b, bb))
    return s, e


def b_fp32(Rh, Rl, t0h, t0l, Kh, Kl, rng):
    """The kernels' sequence for one value; estimates perturbed by <= 2^-22."""
    y0 = fl(1.0 / np.sqrt(np.float64(Rh)) * (1.0 + rng.uniform(-2.0 ** -22, 2.0 ** -22)))
    ph = mul(y0, y0)
    pl = fma(y0, y0, -ph)
    e = fma(-Rh, ph, f32(1.0))
    e = fma(-Rh, pl, e)
    e = fma(-Rl, ph, e)
    yl = mul(mul(f32(0.5), y0), e)
    th = mul(Kh, y0)
    tl = fma(Kh, y0, -th)
    tl = fma(Kh, yl, tl)
    tl = fma(Kl, y0, tl)
    ah, ae = two_sum(t0h, th)
    al = add(ae, add(t0l, tl))
    dh = fma(ah, ah, f32(1.0))
    dl = fma(ah, ah, sub(f32(1.0), dh))
    dl = fma(add(ah, ah), al, dl)
    r0 = fl(1.0 / np.float64(dh) * (1.0 + rng.uniform(-2.0 ** -22, 2.0 ** -22)))
    g = fma(-dh, r0, f32(1.0))
    g = fma(-dl, r0, g)
    rl = mul(r0, g)
    mh = mul(ah, r0)
    ml = fma(ah, r0, -mh)
    ml = fma(ah, rl, ml)
    ml = fma(al, r0, ml)
    return complex(np.float64(r0) + np.float64(rl), -(np.float64(mh) + np.float64(ml)))


def split(x):
    h = f32(x)
    return h, f32(x - np.float64(h))


@pytest.mark.parametrize("deep,Z,a,m,V0", [(False, 1.0, 1.0, 1.0, 0.0), (False, 0.8, 1.3, -1.0, 0.4),
                                           (True, 4.0, 0.5, 1.0, 0.0), (True, 30.0, 0.3, -1.0, -0.5)])
def test_softcore_b_accuracy(deep, Z, a, m, V0):
    rng = np.random.default_rng(7)
    dt = 0.9 / np.sqrt(3.0)
    # R as the kernels form it: hi parts exact sums (multiples of 2^-2 here), lo small
    Rvals = np.concatenate([a * a + np.array([0.0, 0.25, 0.5, 1.0, 2.25]),
                            a * a + 0.25 * rng.integers(0, 4 * 3 * 256 ** 2, 400)])
    t0h, t0l = split(dt * (m + V0) / 2.0)
    Kh, Kl = split(-dt * Z / 2.0)
    worst_b = worst_u = 0.0
    worst_theta = 0.0
    for R in Rvals:
        Rh, Rl = split(R)
        theta = dt * (m + V0) / 2.0 - dt * Z / 2.0 / np.sqrt(np.float64(Rh) + np.float64(Rl))
        worst_theta = max(worst_theta, abs(theta))
        exact = 1.0 / (1.0 + 1j * theta)
        got = b_fp32(Rh, Rl, t0h, t0l, Kh, Kl, rng)
        worst_b = max(worst_b, abs(got - exact) / abs(exact))
        worst_u = max(worst_u, abs(abs(2.0 * got - 1.0) - 1.0))
    assert (worst_theta > 1.0) == deep
    assert worst_b < 2e-13, worst_b
    assert worst_u < 4e-13, worst_u


def test_fma_split_of_one_plus_theta_squared():
    """dh = fl(1 + ah^2) >= 1 is a multiple of its own ulp and so is 1, hence
    1 - dh is exact and fma(ah, ah, 1 - dh) is the rounding error of dh,
    rounded once: dh + dl carries 1 + theta^2 to ~2^-48 for any theta, and
    dropping dl leaves the plain FP32 error (~2^-24)."""
    rng = np.random.default_rng(3)
    thetas = np.concatenate([rng.uniform(-1, 1, 300), rng.uniform(-20, 20, 300), [0.0, 1.0, -1.0, 1e-4]])
    worst = worst_plain = 0.0
    for theta in thetas:
        ah, al = split(theta)
        dh = fma(ah, ah, f32(1.0))
        assert sub(f32(1.0), dh) == np.float64(1.0) - np.float64(dh)  # exact
        dl = fma(ah, ah, sub(f32(1.0), dh))
        dl = fma(add(ah, ah), al, dl)
        exact = 1.0 + theta * theta
        worst = max(worst, abs(np.float64(dh) + np.float64(dl) - exact) / exact)
        worst_plain = max(worst_plain, abs(np.float64(dh) - exact) / exact)
    assert worst < 1e-13, worst
    assert worst_plain > 1e-9
