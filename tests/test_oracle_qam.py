"""Pins for the oracle's alphabet, decisions and Gray (de)mapping (CPU only)."""

import itertools

import numpy as np
import pytest

from oracle import qam
from synth.channel import modulate


@pytest.mark.parametrize("m", [2, 4, 6, 8])
def test_gray_map_is_a_bijection_with_single_bit_neighbours(m):
    L = qam.n_levels(m)
    li, lq = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    bits = qam.levels_to_bits(li.ravel(), lq.ravel(), m)
    words = {tuple(b) for b in bits}
    assert len(words) == L * L == 2**m                      # bijection onto all m-bit words
    back_i, back_q = qam.bits_to_levels(bits, m)
    assert np.array_equal(back_i, li.ravel()) and np.array_equal(back_q, lq.ravel())
    table = {(int(a), int(b)): bits[i] for i, (a, b) in enumerate(zip(li.ravel(), lq.ravel()))}
    for (a, b), w in table.items():                         # nearest neighbours differ in one bit
        for da, db in ((1, 0), (0, 1)):
            if (a + da, b + db) in table:
                assert int(np.sum(w != table[(a + da, b + db)])) == 1


@pytest.mark.parametrize("m", [2, 4, 6])
def test_decision_is_the_exhaustive_nearest_point(m):
    rng = np.random.default_rng(5)
    z = (rng.normal(size=4000) + 1j * rng.normal(size=4000)) * 0.9
    pts = qam.alphabet(m)
    brute = pts[np.argmin(np.abs(z[:, None] - pts[None, :]), axis=1)]
    assert np.allclose(qam.decide(z, m), brute, atol=0, rtol=0)


@pytest.mark.parametrize("m", [2, 4, 6])
def test_alphabet_has_unit_energy_and_qpsk_sign_rule(m):
    assert np.mean(np.abs(qam.alphabet(m)) ** 2) == pytest.approx(1.0, rel=1e-14)
    if m == 2:
        s = qam.levels_to_symbols(*qam.bits_to_levels(np.array([[0, 1], [1, 0]]), 2), 2)
        assert s[0].real < 0 < s[0].imag and s[1].imag < 0 < s[1].real


@pytest.mark.parametrize("m", [2, 4, 6])
def test_transmitter_and_demapper_agree(m):
    """The generator's mapper (synth) and the oracle's demapper are written apart; they must be inverse."""
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2, size=(3, 200 * m), dtype=np.uint8)
    s = modulate(bits, m)
    li, lq = qam.decide_levels(s, m)
    assert np.array_equal(qam.levels_to_bits(li, lq, m).reshape(3, -1), bits)


def test_cma_radius_closed_forms():
    # E|s|^4 / E|s|^2 for unit-energy square QAM: QPSK 1, 16QAM 1.32, 64QAM 29/21
    assert qam.cma_radius(2) == pytest.approx(1.0, rel=1e-14)
    assert qam.cma_radius(4) == pytest.approx(1.32, rel=1e-14)
    assert qam.cma_radius(6) == pytest.approx(29.0 / 21.0, rel=1e-14)


def test_word_packing_layout():
    bits = np.zeros(70, np.uint8)
    bits[[0, 31, 32, 69]] = 1
    w = qam.pack_words(bits)
    assert w.tolist() == [0x80000001, 0x1, 0x20]
    assert np.array_equal(qam.unpack_words(w, 70), bits)
    for n in itertools.chain(range(1, 40), [95, 96, 97]):
        b = np.random.default_rng(n).integers(0, 2, n, dtype=np.uint8)
        assert np.array_equal(qam.unpack_words(qam.pack_words(b), n), b)
