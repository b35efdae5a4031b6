"""Checkpoint schedule of the discrete adjoint (host logic, no device).

envar_revolve_plan runs the schedule dry and checks it: every step reversed once, in the order
n-1 .. 0, each from its own forward state, slots within range.  Its cost (forward steps beyond the
initial sweep) is pinned here to an exhaustive minimisation over every checkpoint placement of
the same recursive scheme, and to the closed cases (one slot per state: no recomputation; no free
slot: n(n-1)/2) and Griewank's repetition bound."""
import functools
from math import comb

import pytest

from paper_2605_23812_gb300 import build as pkg_build
from paper_2605_23812_gb300 import capi


@pytest.fixture(scope="module", autouse=True)
def so():
    pkg_build.build()


@functools.lru_cache(None)
def _inner(n, c):
    # forward steps to reverse n steps from a restored state, c free slots: choose the first
    # checkpoint k steps ahead, reverse the right part with c-1 slots, then the left part with c
    if n <= 1:
        return 0
    if c == 0:
        return n * (n - 1) // 2
    return min(k + _inner(n - k, c - 1) + _inner(k, c) for k in range(1, n))


@functools.lru_cache(None)
def _spine(n, c):
    # same, for the first descent, whose advances are the initial forward sweep
    if n <= 1:
        return 0
    if c == 0:
        return n * (n - 1) // 2
    return min(_spine(n - k, c - 1) + _inner(k, c) for k in range(1, n))


@pytest.mark.parametrize("S", [1, 2, 3, 4, 6])
def test_schedule_is_optimal_for_its_scheme(S):
    for n in range(1, 48):
        got = capi.revolve_plan(n, S)["recompute"]
        assert got == _spine(n, min(S, n) - 1), (n, S)


@pytest.mark.parametrize("n", [1, 2, 7, 100, 1000])
def test_closed_cases(n):
    assert capi.revolve_plan(n, n)["recompute"] == 0
    assert capi.revolve_plan(n, n + 5)["recompute"] == 0
    assert capi.revolve_plan(n, 1)["recompute"] == n * (n - 1) // 2


@pytest.mark.parametrize("n,S", [(10000, 64), (10000, 16), (30000, 64), (2145, 64), (2146, 64)])
def test_repetition_bound(n, S):
    # with s snapshots each step is advanced at most r times, r the least with C(s + r, s) >= n;
    # the initial sweep is one of them
    r = 0
    while comb(S + r, S) < n:
        r += 1
    plan = capi.revolve_plan(n, S)
    assert 0 <= plan["recompute"] <= (r - 1) * n
    assert plan["stores"] <= n - 1


def test_rejects_bad_arguments():
    with pytest.raises(capi.EnvarError):
        capi.revolve_plan(0, 4)
    with pytest.raises(capi.EnvarError):
        capi.revolve_plan(10, 0)
