"""Pins of the oracle's quantizer (oracle/quantize.py), CPU only: the class of
every node against its definition by brute force, the hand-worked quantized
Fig. 2 example, the quantizer's error bound, exact multiples and ties,
symmetry and saturation."""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "quantize_1d.txt")


def _golden():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    return [np.array([float(x) for x in r]) for r in rows]


@pytest.mark.parametrize("shape,L", [((5,), 2), ((9, 5), 2), ((9, 17, 5), 2), ((17, 9), 3), ((33,), 5),
                                     ((9, 9, 9), 0)])
def test_node_classes_brute_force(shape, L):
    cls = oracle.node_classes(shape, L)
    for idx in itertools.product(*[range(n) for n in shape]):
        want = next(l for l in range(L + 1) if all(i % (1 << (L - l)) == 0 for i in idx))
        assert cls[idx] == want
    # class l holds |N_l| - |N_{l-1}| nodes
    sizes = [int(np.prod([(n - 1) // (1 << (L - l)) + 1 for n in shape])) for l in range(L + 1)]
    for l in range(L + 1):
        assert int((cls == l).sum()) == sizes[l] - (sizes[l - 1] if l else 0)


def test_golden_worked_example():
    c, classes, q1, q2, d2 = _golden()
    assert np.array_equal(oracle.node_classes((5,), 2), classes.astype(np.int32))
    for dt in (np.float64, np.float32):
        cc = c.astype(dt)
        assert np.array_equal(oracle.quantize(cc, [1, 1, 1], 2), q1.astype(np.int32))
        q = oracle.quantize(cc, [0.5, 1, 2], 2)
        assert np.array_equal(q, q2.astype(np.int32))
        assert np.array_equal(oracle.dequantize(q, [0.5, 1, 2], 2, dt), d2.astype(dt))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_error_bound_half_a_bin(dt):
    rng = np.random.default_rng(3)
    shape, L = (17, 33, 9), 3
    c = rng.normal(0, 1, shape).astype(dt)
    bins = [0.3, 0.07, 0.01, 0.002]
    d = oracle.dequantize(oracle.quantize(c, bins, L), bins, L, dt)
    b = np.asarray(bins)[oracle.node_classes(shape, L)]
    eps = np.finfo(dt).eps
    assert np.all(np.abs(c.astype(np.float64) - d.astype(np.float64)) <= b * (0.5 + 4 * eps) + 4 * eps * np.abs(c))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_exact_multiples_ties_and_symmetry(dt):
    shape, L = (9, 9), 3
    rng = np.random.default_rng(4)
    k = rng.integers(-1000, 1000, shape)
    bins = [2.0 ** -j for j in (0, 2, 3, 5)]                  # powers of two: k bin and (k + 1/2) bin exact
    b = np.asarray(bins)[oracle.node_classes(shape, L)]
    c = (k * b).astype(dt)
    q = oracle.quantize(c, bins, L)
    assert np.array_equal(q, k.astype(np.int32))
    assert np.array_equal(oracle.dequantize(q, bins, L, dt), c)
    ties = ((k + 0.5 * np.sign(k + 0.1)) * b).astype(dt)     # halfway points, away from zero
    want = (k + np.sign(k + 0.1)).astype(np.int32)
    assert np.array_equal(oracle.quantize(ties, bins, L), want)
    assert np.array_equal(oracle.quantize(-c, bins, L), -q)


def test_saturation():
    c = np.array([1e12, -1e12, 1.0, -3e9, 2.0 ** 31], dtype=np.float64)
    q = oracle.quantize(c, [1.0, 1.0, 1.0], 2)
    assert list(q) == [2 ** 31 - 1, -(2 ** 31 - 1), 1, -(2 ** 31 - 1), 2 ** 31 - 1]


def test_bins_validated():
    with pytest.raises(ValueError):
        oracle.quantize(np.zeros(5), [1.0, 1.0], 2)
    with pytest.raises(ValueError):
        oracle.quantize(np.zeros(5), [1.0, 0.0, 1.0], 2)
