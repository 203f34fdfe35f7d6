"""Pins of the oracle's Philox4x32-10 against an independent library routine.

Triton ships a Philox4x32 implementation (``tl.philox``, 10 rounds by
default) that runs on the CPU through its interpreter. Agreement on counters
and keys that exercise every word pins the round function, the multipliers,
the key schedule and the word order of ``oracle.philox``.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle.philox import philox4x32, philox_for_groups

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = [
    [0, 0, 0, 0, 0],
    [0xFFFFFFFFFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF],
    [0x299F31D0A4093822, 0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
    [1, 0, 0, 0, 0],
    [1, 12345, 0, 0, 0],
    [48, 0x7FFFFFFF, 3, 0, 0],
    [0x100000001, 7, 0x1, 0, 0],
    [2**32 + 5, 0xDEADBEEF, 0xCAFEBABE, 0x1234, 0x5678],
]


def _triton_words(cases):
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, os.path.join(HERE, "triton_philox_ref.py")],
                          input=json.dumps({"cases": cases}), capture_output=True,
                          text=True, env=env, timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr.strip().splitlines()[-1])
    return json.loads(proc.stdout)


def _oracle_words(case):
    seed, c0, c1, c2, c3 = case
    r = philox4x32(c0, c1, c2, c3, seed & 0xFFFFFFFF, seed >> 32)
    return [int(x) for x in r]


def test_philox_matches_triton_library():
    ref = _triton_words(CASES)
    for case, want in zip(CASES, ref):
        assert _oracle_words(case) == want, (case, [hex(x) for x in want])


def test_group_counter_layout():
    """philox_for_groups puts the 64-bit group index in (c0, c1) and the seed in the key."""
    seed = 0x0000000500000007
    groups = np.array([0, 1, 2**32 + 3, 2**40 + 9], dtype=np.uint64)
    got = philox_for_groups(seed, groups)
    for g, row in zip(groups, got):
        want = _oracle_words([seed, int(g) & 0xFFFFFFFF, int(g) >> 32, 0, 0])
        assert [int(x) for x in row] == want


def test_rounds_matter():
    """Fewer rounds give different words (guards against a loop that stops early)."""
    a = [int(x) for x in philox4x32(1, 2, 3, 4, 5, 6, rounds=10)]
    b = [int(x) for x in philox4x32(1, 2, 3, 4, 5, 6, rounds=9)]
    assert a != b


def test_word_bits_uniform():
    """Each output bit is set with probability 1/2 (5 sigma over 2^18 draws)."""
    w = philox_for_groups(3, np.arange(1 << 16, dtype=np.uint64)).reshape(-1)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.float64)
    frac = bits.mean(axis=0)
    sigma = 0.5 / np.sqrt(w.size)
    assert np.all(np.abs(frac - 0.5) < 5 * sigma)
