"""The full-size checker itself, on the CPU: it accepts the oracle's stable
sort and rejects a swapped pair, an unstable order of equal keys, a changed
byte and a duplicated record."""
import numpy as np
import pytest
import torch

import oracle
import recgen
from stable_check import check_stable_sort


@pytest.fixture(scope="module")
def case():
    n = 20_000
    host = recgen.generate_cpu(n, recgen.KeySpec("zipf", s=1.3, dup=0.2, seed=21))
    return n, host, oracle.stable_sort(host)


def test_accepts_stable_sort(case):
    n, host, out = case
    check_stable_sort(torch.from_numpy(host), torch.from_numpy(out.copy()), n, chunk=3000)


def _planted(out, n, how):
    o = out.copy().reshape(n, 100)
    keys = [bytes(o[i, :10]) for i in range(n)]
    if how == "swap":
        i = next(i for i in range(n - 1) if keys[i] != keys[i + 1])
        o[[i, i + 1]] = o[[i + 1, i]]
    elif how == "unstable":
        i = next(i for i in range(n - 1) if keys[i] == keys[i + 1])
        o[[i, i + 1]] = o[[i + 1, i]]
    elif how == "byte":
        o[n // 2, 60] ^= 1
    elif how == "duplicate":
        i = next(i for i in range(n - 1) if keys[i] == keys[i + 1])
        o[i + 1] = o[i]
    return o.reshape(-1)


@pytest.mark.parametrize("how", ["swap", "unstable", "byte", "duplicate"])
def test_rejects_planted_faults(case, how):
    n, host, out = case
    with pytest.raises(AssertionError):
        check_stable_sort(torch.from_numpy(host), torch.from_numpy(_planted(out, n, how)), n, chunk=3000)
