"""Pins of the oracle's random-number generator, exponential and decisions.

* Philox4x32-10 is compared word for word with an independent implementation
  (Triton's, executed on the CPU by its interpreter).
* pt_exp's constants are compared with their mathematical definitions rounded
  correctly to float32, and its values with the double-precision exponential.
* The heat-bath decision and the swap test are counted exhaustively over all
  2^23 uniforms and compared with the closed forms 1/(1+exp(-beta H)) and
  min(1, exp(x)).
"""
import json
import math
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _rn_f32(q: Fraction) -> float:
    """Round a rational to the nearest float32 (ties to even), exactly."""
    if q == 0:
        return 0.0
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = math.floor(math.log2(q.numerator) - math.log2(q.denominator))
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    scaled = q / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    m = math.floor(scaled)
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return sign * float(Fraction(m) * Fraction(2) ** (e - 23))


def _ln2_fraction(digits=60) -> Fraction:
    import mpmath

    mpmath.mp.dps = digits
    return Fraction(str(mpmath.log(2)))


def test_philox_matches_triton_reference():
    pytest.importorskip("triton")
    proc = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox.py")],
                          capture_output=True, text=True, timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr[-300:])
    cases = json.loads(proc.stdout.strip().splitlines()[-1])
    assert len(cases) >= 32
    for ctr, key, words in cases:
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == words, (ctr, key)


def test_philox_is_counter_based_and_balanced():
    # different counters or keys give different words; bits are balanced
    key = [7, 0]
    words = np.array([oracle.philox4x32_10([i, 0, 0, 0], key) for i in range(4096)])
    assert len({tuple(w) for w in words}) == 4096
    bits = np.unpackbits(words.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.005
    assert not np.array_equal(oracle.philox4x32_10([1, 2, 3, 4], [7, 0]),
                              oracle.philox4x32_10([1, 2, 3, 4], [8, 0]))


def test_pt_exp_constants_are_their_definitions():
    c = oracle.pt_exp_constants().astype(np.float64)
    ln2 = _ln2_fraction()
    log2e = 1 / ln2
    assert c[0] == _rn_f32(log2e)
    ln2_f = _rn_f32(ln2)
    bits = np.array([ln2_f], dtype=np.float32).view(np.uint32)[0]
    hi = float(np.array([bits & np.uint32(0xFFFFF000)], dtype=np.uint32).view(np.float32)[0])
    assert c[1] == hi
    assert c[2] == _rn_f32(ln2 - Fraction(hi))
    for n in range(8):
        assert c[3 + n] == _rn_f32(Fraction(1, math.factorial(n))), n


def _ulp32(y: float) -> float:
    y = abs(y)
    if y < 2.0 ** -126:
        return 2.0 ** -149
    return 2.0 ** (math.floor(math.log2(y)) - 23)


def test_pt_exp_accuracy_and_range():
    rng = np.random.default_rng(5)
    xs = np.concatenate([
        np.linspace(-103.9, 88.7, 40001, dtype=np.float32),
        rng.uniform(-103.9, 88.7, 20000).astype(np.float32),
        rng.uniform(-1, 1, 5000).astype(np.float32),
    ])
    worst = 0.0
    for x in xs:
        y = oracle.pt_exp(float(x))
        ref = math.exp(float(x))
        err = abs(y - ref) / _ulp32(ref)
        worst = max(worst, err)
    assert worst <= 3.0, worst
    assert oracle.pt_exp(0.0) == 1.0
    assert oracle.pt_exp(89.0) == math.inf
    assert oracle.pt_exp(-104.5) == 0.0
    # monotone non-decreasing on a sorted grid (the decisions rely on it)
    grid = np.linspace(-103.9, 88.7, 20001, dtype=np.float32)
    ys = np.array([oracle.pt_exp(float(x)) for x in grid])
    assert np.all(np.diff(ys) >= 0)


def _sigmoid(z: float) -> float:
    if z >= 0:
        return 1.0 / (1.0 + math.exp(-z))
    e = math.exp(z)
    return e / (1.0 + e)


@pytest.mark.parametrize("beta,H", [
    (1.0e-5, 0), (1.0e-5, 30000), (1.0e-5, -30000), (3.2e-5, 131068), (3.2e-5, -262136),
    (1.57e-6, 98301), (0.25, 7), (0.25, -7), (2.0, 40), (2.0, -50), (1.0, 1),
])
def test_heatbath_matches_sigmoid(beta, H):
    count = oracle.heatbath_count(beta, H)
    p_real = count / 2.0**23
    b32 = float(np.float32(beta))
    p_ref = _sigmoid(b32 * H)
    assert abs(p_real - p_ref) <= 2e-6, (p_real, p_ref)
    if H == 0:
        # d = 2 exactly; u = (m+1) 2^-23 < 1/2 for m = 0 .. 2^22 - 2
        assert count == 2**22 - 1
    if H > 0:
        assert count > 2**22 - 1  # the field favours +1 when E(+1) < E(-1)


@pytest.mark.parametrize("x", [0.0, 1.5, -1e-7, -0.01, -0.69314718, -1.0, -5.0, -16.0, -40.0])
def test_swap_acceptance_matches_metropolis(x):
    count = oracle.swap_count(x)
    p_real = count / 2.0**23
    p_ref = min(1.0, math.exp(float(np.float32(x))))
    assert abs(p_real - p_ref) <= 2e-7 + 2**-23, (p_real, p_ref)
    if x >= 0:
        assert count == 2**23


def test_pswap_always_accepts_when_lower_penalty_is_more_feasible():
    facts = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))
    case = facts["pswap_always_accepts_when_dg_positive"]
    # Eq. 2: exponent beta * dP * dg with dP > 0, dg > 0 -> always accepted
    x = float(np.float32(3.1e-5) * np.float32(case["dP"] * case["dg"]))
    assert oracle.swap_count(x) == 2**23
    # the reverse move (dg < 0) is accepted with probability exp(-beta dP |dg|) < 1
    x_rev = float(np.float32(3.1e-5) * np.float32(-case["dP"] * case["dg"] * 100))
    assert oracle.swap_count(x_rev) < 2**23
