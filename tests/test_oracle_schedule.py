"""Pins of the oracle's adaptive ladder schedule (Algorithm 2).

1. A worked example: a stub population sampler with hand-chosen populations
   walks every branch of the schedule (the first column's stop at sigma_min,
   the sigma_min floor in later columns, rows without a penalty proposal, the
   feasibility break, even and odd medians).  The expected ladders are the
   exact rationals worked out by hand below, rounded to float32 / int.
2. The schedule's purpose (Section "Ground-state optimization under
   constraints"): with learning rates alpha = 2 erfc^-1(1/2) ~ 0.954, adjacent
   replicas swap with probability ~ 1/2.  For Gaussian energy distributions of
   width sigma a beta step d gives a swap rate erfc(d sigma / 2) (a textbook
   property of replica exchange), and the schedule sets d sigma = alpha; the
   same holds for the penalty steps with beta sigma_g in place of sigma.  The
   realised rates of a 2D-PT run on the resulting ladders must sit near 1/2.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest
from scipy.special import erfcinv

import oracle
from oracle.schedule import ScheduleParams, adaptive_schedule, median, oracle_sampler, population_stats
import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def test_population_stats_exact_and_median():
    # populations of two values: std = half the gap, mean of g
    assert population_stats([0, 8], [3, 3]) == (4.0, 0.0, 3.0)
    # one value per chain repeated: zero spread
    assert population_stats([5, 5, 5], [1, 1, 1]) == (0.0, 0.0, 1.0)
    # {1, 2, 3, 4}: variance 5/4 exactly
    s = population_stats([1, 2, 3, 4], [0, 0, 1, 1])
    assert s == (np.sqrt(1.25), 0.5, 0.5)
    # large energies: exact integer sums (no cancellation) keep the spread
    big = 10 ** 12
    assert population_stats([big, big + 2], [0, 0])[0] == 1.0
    assert median([3.0, 1.0, 2.0]) == 2.0 and median([4.0, 1.0, 3.0, 2.0]) == 2.5


# (E population, g population) for sample k, and the (beta, P) it must be drawn at
_STUB = [
    ([0, 8], [0, 2], Fr(1, 2), 8),       # col 1 row 1: sigma_E 4 -> beta 3/4; proposal 8 + 2/(1/2) = 12
    ([0, 10], [0, 4], Fr(3, 4), 8),      # row 2: sigma_E 5 -> beta 19/20; proposal 8 + 2/(3/4 * 2) = 28/3
    ([0, 20], [1, 1], Fr(19, 20), 8),    # row 3: sigma_E 10 -> beta 21/20; sigma_g 0: no proposal
    ([0, 4], [0, 2], Fr(21, 20), 8),     # row 4: sigma_E 2 <= 3: stop, I = 4; P(2) = rint(median(12, 28/3)) = 11
    ([0, 4], [0, 2], Fr(1, 2), 11),      # col 2 row 1: sigma_E 2 floored to 3 -> 5/6; proposal 11 + 4 = 15
    ([0, 8], [0, 8], Fr(5, 6), 11),      # row 2: sigma_E 4 -> 13/12; proposal 11 + 2/(5/6 * 4) = 58/5
    ([0, 16], [0, 2], Fr(13, 12), 11),   # row 3: sigma_E 8 -> 29/24; proposal 11 + 24/13 = 167/13
    ([0, 2], [3, 3], Fr(29, 24), 11),    # row 4 (last): mean_g 3: go on; P(3) = rint(median(15, 58/5, 167/13)) = 13
    ([0, 7], [0, 2], Fr(1, 2), 13),      # col 3 row 1: sigma_E 7/2 -> 11/14
    ([0, 6], [0, 2], Fr(11, 14), 13),    # row 2: sigma_E 3 -> 47/42
    ([0, 40], [0, 2], Fr(47, 42), 13),   # row 3: sigma_E 20 -> 491/420
    ([0, 2], [0, 0], Fr(491, 420), 13),  # row 4: mean_g 0 < 1/2: stop, J = 3
]


def test_worked_example_walks_every_branch():
    calls = []

    def stub(beta, P, k):
        E, g, b_expect, P_expect = _STUB[k]
        assert P == P_expect, (k, P)
        assert beta == np.float32(float(b_expect)), (k, beta, b_expect)
        calls.append(k)
        return np.array(E, np.int64), np.array(g, np.int64)

    prm = ScheduleParams(beta0=0.5, P0=8, max_rows=5, max_cols=4, sigma_min=3.0, alpha_beta=1.0,
                         alpha_P=2.0, n_chain=2, mcs=1, seed=0)
    beta, P, k = adaptive_schedule(stub, prm)
    assert calls == list(range(12)) and k == 12
    assert list(P) == [8, 11, 13]
    # row medians over the three columns:
    #   row 1: 1/2; row 2: (3/4, 5/6, 11/14) -> 11/14; row 3: (19/20, 13/12, 47/42) -> 13/12;
    #   row 4: (21/20, 29/24, 491/420) -> 491/420
    expect = [Fr(1, 2), Fr(11, 14), Fr(13, 12), Fr(491, 420)]
    assert list(beta) == [np.float32(float(x)) for x in expect]


def test_caps_bound_rows_and_columns():
    def stub(beta, P, k):  # always wide populations, never feasible
        return np.array([0, 100], np.int64), np.array([1, 3], np.int64)

    prm = ScheduleParams(beta0=0.1, P0=4, max_rows=3, max_cols=2, sigma_min=1.0, alpha_beta=1.0,
                         alpha_P=1.0, n_chain=2, mcs=1, seed=0)
    beta, P, k = adaptive_schedule(stub, prm)
    assert beta.size == 3 and P.size == 2 and k == 6
    assert np.all(np.diff(beta) > 0) and P[1] > P[0]


def _attempts(n_events, J, I, pswap):
    """Per lower-pair index (column j for P-swaps, row i for beta-swaps): how many
    events of Algorithm 1 tried that pair."""
    cnt = np.zeros(J if pswap else I, np.int64)
    for n in range(1, n_events + 1):
        is_p = ((n - 1) // 2) % 2 == 0
        if is_p != pswap:
            continue
        start = 1 if n % 2 == 0 else 0
        last = (J if pswap else I) - 1
        cnt[start:last:2] += 1
    return cnt


def test_schedule_gives_swap_rates_near_one_half():
    inst = synth.wishart_planted(16, 0.5, 11)
    oinst = oracle.OracleInstance(oracle.sparsify(inst.Jq, "max_edges", 3))
    alpha = float(2 * erfcinv(0.5))
    prm = ScheduleParams(beta0=0.2 / inst.scale, P0=int(0.5 * 32767), max_rows=8, max_cols=6,
                         sigma_min=2.0 * 32767 / 8, alpha_beta=alpha, alpha_P=alpha, n_chain=128,
                         mcs=200, seed=99)
    beta, P, k = adaptive_schedule(oracle_sampler(oinst, prm), prm)
    I, J = beta.size, P.size
    assert I >= 3 and J >= 2 and np.all(np.diff(beta) > 0) and np.all(np.diff(P) > 0)
    runs, events, interval = 8, 400, 5
    orc = oracle.OracleRun(oinst, beta, P, list(range(runs)), 5)
    orc.run(events * interval, interval)
    att_B = _attempts(events, J, I, pswap=False)
    att_P = _attempts(events, J, I, pswap=True)
    acc_B = orc.acc_B.reshape(runs, I, J)[:, :-1, :].sum(axis=(0, 2)) / (runs * J * att_B[:-1])
    acc_P = orc.acc_P.reshape(runs, I, J)[:, :, :-1].sum(axis=(0, 1)) / (runs * I * att_P[:-1])
    assert 0.4 < acc_B.mean() < 0.6, acc_B
    assert 0.4 < acc_P.mean() < 0.7, acc_P
