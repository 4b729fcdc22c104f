"""The procedural-alpha decision without a sine (no GPU needed).

The kernels decide sin(a) * sin(b) > 0 from the signs of the two sines: with
k = rint(a / pi) and r = a - k pi reduced by three fused multiply-adds over a
three-part float32 split of pi (Cody and Waite's additive reduction),
sign(sin a) = (-1)^k sign(r).  This file reads the constants from the device
header and emulates those float32 operations exactly with rationals, then
checks the sign against the true sine:
  - the split: the first part has at most 8 significant bits (so k times it is
    exact for the arguments covered), the parts sum to pi within 2e-19, and
    1/pi is the float32 rounding of 1/pi;
  - every float32 next to a multiple of pi for |x| < 2^16 (the hardest
    inputs: the sine is smallest there), and a sample of them up to 2^22;
  - random float32 arguments across the range, zeros and tiny values.
The true sign comes from pi to 90 digits (Machin's formula in integers).
"""
import math
import os
import random
import re
from fractions import Fraction as F

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1912_12786_gb300", "csrc", "vsr_device.cuh")


def _arctan_inv(x, digits):
    s, t, x2, k = 0, 10 ** digits // x, x * x, 0
    while t:
        s += t // (2 * k + 1) if k % 2 == 0 else -(t // (2 * k + 1))
        t //= x2
        k += 1
    return s


PI = F(16 * _arctan_inv(5, 90) - 4 * _arctan_inv(239, 90), 10 ** 90)


def _const(name):
    src = open(HEADER).read()
    m = re.search(r"constexpr float " + name + r"\s*=\s*([0-9a-fA-Fx.p+-]+)f;", src)
    assert m, name
    return F(float.fromhex(m.group(1)))


def rnd32(q: F) -> F:
    """Nearest float32 (ties to even) of a rational, normal or subnormal."""
    if q == 0:
        return F(0)
    sgn, a = (-1 if q < 0 else 1), abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while F(2) ** e > a:
        e -= 1
    while F(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)
    scale = F(2) ** (23 - e)
    m = a * scale
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > F(1, 2) or (rem == F(1, 2) and fl % 2 == 1):
        fl += 1
    return sgn * F(fl) / scale


def rint(q: F) -> F:
    fl = q.numerator // q.denominator
    rem = q - fl
    if rem > F(1, 2) or (rem == F(1, 2) and fl % 2):
        fl += 1
    return F(fl)


INV, A, B, C = (_const(n) for n in ("kInvPi", "kPiA", "kPiB", "kPiC"))


def sign_kernel(x: F) -> int:
    """The kernel's sin_sign, each float32 operation rounded exactly once."""
    k = rint(rnd32(x * INV))
    r = rnd32(x - k * A)
    r = rnd32(r - k * B)
    r = rnd32(r - k * C)
    s = (r > 0) - (r < 0)
    return -s if int(k) % 2 else s


def sign_true(x: F) -> int:
    if x == 0:
        return 0
    k = math.floor(x / PI)
    return 1 if k % 2 == 0 else -1


def test_split_of_pi():
    assert A == F(201, 64) and A.numerator.bit_length() == 8  # 8 significant bits
    assert abs(A + B + C - PI) < F(2, 10 ** 19)
    assert rnd32(1 / PI) == INV
    assert rnd32(PI - A) == B and rnd32(PI - A - B) == C


def _neighbours(k):
    x0 = rnd32(k * PI)
    ulp = F(2) ** (math.floor(math.log2(float(x0))) - 23)
    return (x0 - ulp, x0, x0 + ulp)


def test_floats_next_to_multiples_of_pi_below_2_16():
    for k in range(1, int(2 ** 16 / math.pi) + 2):
        for x in _neighbours(k):
            assert sign_kernel(x) == sign_true(x), (k, float(x))
    rng = random.Random(3)
    for k in rng.sample(range(1, int(2 ** 16 / math.pi)), 300):
        for x in _neighbours(k):
            assert sign_kernel(-x) == sign_true(-x), (k, float(x))


def test_floats_next_to_multiples_of_pi_up_to_2_22():
    rng = random.Random(4)
    for k in rng.sample(range(20_000, int(2 ** 22 / math.pi)), 1500):
        for x in _neighbours(k):
            assert sign_kernel(x) == sign_true(x), (k, float(x))


def test_random_arguments_zeros_and_tiny_values():
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(-40.0, 40.0, 2000),
                         rng.uniform(-2.0 ** 22, 2.0 ** 22, 1000),
                         2.0 ** rng.uniform(-140, 21, 1000)]).astype(np.float32)
    for x in xs:
        q = F(float(x))
        assert sign_kernel(q) == sign_true(q), float(x)
    for x in (0.0, -0.0, 1e-45, -1e-45, 1e-38, float(np.float32(math.pi)),
              float(np.float32(2 * math.pi))):
        q = F(x)
        assert sign_kernel(q) == sign_true(q), x


def test_product_decision_matches_sines_on_the_texture_domain():
    """accept = sign(sin(f u)) * sign(sin(f v)) > 0 equals the float64 sine
    product's sign at f = 40 on uv in [0, 1] (float32 arguments)."""
    rng = np.random.default_rng(6)
    uv = rng.uniform(0.0, 1.0, (2000, 2)).astype(np.float32)
    args = (np.float32(40.0) * uv).astype(np.float32)
    for a, b in args:
        want = math.sin(float(a)) * math.sin(float(b)) > 0
        got = sign_kernel(F(float(a))) * sign_kernel(F(float(b))) > 0
        assert got == want, (a, b)
