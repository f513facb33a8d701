"""Pins of the oracle's Huffman stage (Sec. 2.1 step 3, Sec. 3.3).

* When no length limit binds, the total coded length sum f_i l_i equals the
  minimum-redundancy cost of an independent heap-based Huffman construction
  (that cost is unique even though tie-breaks are not).
* Kraft sum is exactly 1 for two or more live symbols, lengths are
  non-increasing in frequency, and never exceed the limit.
* With a binding limit the code stays complete and costs at least the optimum.
* The coded payload of a real container decodes back to the quantization
  codes (decode o encode = identity).
"""
import heapq

import numpy as np
import pytest

from paper_2509_01626_gb300 import synth


def heap_cost(freq):
    h = [int(f) for f in freq if f > 0]
    if len(h) == 1:
        return h[0]
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a = heapq.heappop(h)
        b = heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def check_code(freq, lens, limit, complete=True):
    live = freq > 0
    assert (lens[~live] == 0).all()
    assert (lens[live] >= 1).all() and lens.max() <= limit
    kraft = sum(2.0 ** -int(l) for l in lens[live])
    assert kraft <= 1.0
    if live.sum() >= 2 and complete:
        assert kraft == 1.0
    order = np.argsort(-freq[live], kind="stable")
    fl = freq[live][order]
    ll = lens[live][order]
    for i in range(len(fl) - 1):
        if fl[i] > fl[i + 1]:
            assert ll[i] <= ll[i + 1]


@pytest.mark.parametrize("seed", range(20))
def test_optimal_when_limit_not_binding(ora, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 300))
    freq = np.zeros(2048, dtype=np.uint64)
    syms = rng.choice(2048, size=n, replace=False)
    freq[syms] = rng.integers(1, 200, size=n)
    lens = ora.huffman_lengths(freq, 24)
    check_code(freq, lens, 24)
    assert int((freq * lens).sum()) == heap_cost(freq)


def test_textbook_example(ora):
    # frequencies 45,13,12,16,9,5 -> optimal lengths 1,3,3,3,4,4 (cost 224)
    freq = np.array([45, 13, 12, 16, 9, 5], dtype=np.uint64)
    lens = ora.huffman_lengths(freq, 12)
    assert int((freq * lens).sum()) == 224 == heap_cost(freq)
    assert lens[0] == 1 and sorted(lens.tolist()) == [1, 3, 3, 3, 4, 4]


@pytest.mark.parametrize("seed", range(10))
def test_length_limit(ora, seed):
    rng = np.random.default_rng(100 + seed)
    # geometric frequencies make an unbounded Huffman tree deeper than 12
    n = int(rng.integers(20, 60))
    freq = np.zeros(2048, dtype=np.uint64)
    freq[:n] = (2.0 ** np.linspace(40, 0, n)).astype(np.uint64) + 1
    lens = ora.huffman_lengths(freq, 12)
    check_code(freq, lens, 12, complete=False)
    assert int((freq * lens).sum()) >= heap_cost(freq)
    assert lens.max() == 12
    # geometric frequencies are the worst case for any limit; the repair stays
    # within 5% of the unlimited optimum
    assert int((freq * lens).sum()) <= 1.05 * heap_cost(freq)


def test_single_and_empty(ora):
    f = np.zeros(16, dtype=np.uint64)
    assert (ora.huffman_lengths(f, 12) == 0).all()
    f[5] = 77
    l = ora.huffman_lengths(f, 12)
    assert l[5] == 1 and l.sum() == 1


@pytest.mark.parametrize("eb", [1e-2, 1e-4])
def test_payload_decodes_to_codes(ora, eb):
    x = synth.sinusoids((40, 36, 44), 9)
    codes, soff, recon, ebs = ora.quantize(x, eb)
    c = ora.compress(x, eb)
    dec, soff2 = ora.decode_streams(c)
    assert np.array_equal(soff, soff2)
    assert np.array_equal(codes, dec)


def test_length_limit_many_rare_symbols(ora):
    """A dominant symbol and a long tail of singletons (the shape of
    quantization codes): the limit binds and the code stays valid."""
    freq = np.zeros(2048, dtype=np.uint64)
    freq[1024] = 10 ** 8
    freq[1023] = freq[1025] = 10 ** 6
    freq[1000:1020] = 1
    freq[1:200] = 1
    lens = ora.huffman_lengths(freq, 12)
    check_code(freq, lens, 12, complete=False)
    assert lens[1024] == 1
