"""Pins of the oracle's random numbers and index draws (Section 4.1).

The oracle's Philox4x64-10 is checked against numpy.random.Philox, an
independent implementation of the same published generator; the index draw
is checked against a pure-Python twin built on numpy's generator and
Python's arbitrary-precision integers.
"""
import numpy as np
import pytest

import oracle


def numpy_philox_block(counter, key):
    """One block from numpy's Philox: numpy increments the counter before use."""
    c = [int(v) for v in counter]
    # step the 256-bit counter back by one so numpy's pre-increment lands on it
    for i in range(4):
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = 2**64 - 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(c, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


@pytest.mark.parametrize("counter,key", [
    ([1, 0, 0, 0], [5, 7]),
    ([0, 0, 0, 0], [0, 0]),
    ([123456789, 42, 3, 1], [2**64 - 1, 99]),
    ([2**64 - 1, 7, 2, 0], [1906, 1687]),   # counter word 0 at its maximum
    ([0, 2**64 - 1, 1, 0], [1, 2]),         # numpy's decrement borrows across words
    ([77, 2**63, 4, 1], [31337, 0]),
])
def test_philox_matches_numpy(counter, key):
    ours = [int(v) for v in oracle.philox4x64(counter, key)]
    assert ours == numpy_philox_block(counter, key)


def test_philox_many_counters_match_numpy():
    rng = np.random.default_rng(0)
    for _ in range(50):
        counter = [int(v) for v in rng.integers(0, 2**63, 4, dtype=np.uint64)]
        counter[0] += 1  # keep word 0 nonzero for a simple numpy step-back
        key = [int(v) for v in rng.integers(0, 2**63, 2, dtype=np.uint64)]
        assert [int(v) for v in oracle.philox4x64(counter, key)] == numpy_philox_block(counter, key)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 20, 31, 100, 6186, 100_000, 2**40 + 3])
def test_randi_partitions_words_into_n_intervals(n):
    """randi(n) splits [0, 2^64) into n runs of consecutive words, value v
    starting at the first word W with W * n >= v * 2^64."""
    values = range(n) if n <= 100 else [0, 1, n // 2, n - 2, n - 1]
    for v in values:
        start = -(-v * 2**64 // n)  # ceil(v 2^64 / n)
        assert oracle.randi(start, n) == v
        if start > 0:
            assert oracle.randi(start - 1, n) == v - 1
    assert oracle.randi(2**64 - 1, n) == n - 1
    assert oracle.randi(0, n) == 0


def python_draw(dims, seed, problem, stream, tag, j):
    """Independent twin of the draw: numpy's Philox words, Python big-int multiply-high."""
    idx = []
    for k, n in enumerate(dims):
        w = numpy_philox_block([j, stream, tag, k // 4], [seed, problem])[k % 4]
        idx.append((w * n) >> 64)
    return idx


@pytest.mark.parametrize("dims", [(20, 30, 40), (100, 100, 100, 100), (3, 5, 7, 11, 13), (2,) * 8])
def test_draw_multi_index_matches_python_twin(dims):
    for j in [0, 1, 2, 999, 2**40]:
        for tag in [oracle.TAG_UNIFORM, oracle.TAG_ZERO_CANDIDATE, oracle.TAG_SEMI_ZERO]:
            got = oracle.draw_multi_index(dims, 1687, 3, 11, tag, j).tolist()
            assert got == python_draw(dims, 1687, 3, 11, tag, j)


def test_draw_nonzero_matches_python_twin():
    for nnz in [1, 5, 5_330_673, 10**8]:
        for j in [0, 5, 77777]:
            w = numpy_philox_block([j, 9, oracle.TAG_NONZERO, 0], [42, 0])[0]
            assert oracle.draw_nonzero(nnz, 42, 0, 9, j) == (w * nnz) >> 64


def test_draws_are_uniform():
    """Counts of each mode index over many draws stay within 5 binomial sigma of s/n_k."""
    dims = (7, 5, 3)
    s = 20000
    counts = [np.zeros(n) for n in dims]
    for j in range(s):
        ix = oracle.draw_multi_index(dims, 5, 0, 0, oracle.TAG_UNIFORM, j)
        for k in range(3):
            counts[k][ix[k]] += 1
    for k, n in enumerate(dims):
        mean = s / n
        sd = np.sqrt(s * (1 / n) * (1 - 1 / n))
        assert np.all(np.abs(counts[k] - mean) < 5 * sd)


def test_linear_key_is_row_major():
    dims = (4, 5, 6)
    ref = np.arange(np.prod(dims)).reshape(dims)
    for ix in [(0, 0, 0), (3, 4, 5), (1, 2, 3), (2, 0, 5)]:
        assert oracle.linear_key(dims, ix) == ref[ix]

