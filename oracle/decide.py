"""A6 ambiguity resolution, Gray hard demapping, BER / EVM counting, FP64.

TEST INFRASTRUCTURE (see the package docstring).

Paper anchor: decided symbols are demapped to bits on the GPU and the quality
is reported as a Q-factor derived from the BER of each 21 ms section
(Sec. II-D Step 6, Sec. V-D). The paper does not describe how a blind
receiver is aligned with the transmitted bits; reading taken here:

* sync window = the first ``sync_len`` counted symbols; for each output
  polarisation q pick (tx pol p, quarter turn r, delay d), d in
  [-max_delay, max_delay], maximising #{n : dec(z_q[n] j^r) == s_p[n + d - lat]}
  (exact comparison of level indices); ties go to the lexicographically
  smallest (p, r, d). ``lat`` is the receiver's fixed symbol latency (0 for a
  single frame);
* counted window [E, N - E); bits of output q, symbol n are compared with the
  reference bits of pol p at symbol n + d - lat; popcount of the XOR;
* EVM = sqrt(sum |z_q[n] j^r - s| ^2 / sum |s|^2) over the counted window;
* output bits: dec(z_q[n] j^{r_q}) demapped for every n in [0, N), packed
  32 per word (bit i -> word i // 32, bit i % 32), in output-polarisation order.
"""

from __future__ import annotations

import numpy as np

from . import qam

QUARTER = np.array([1.0, 1j, -1.0, -1j])  # j^r


def ref_levels(ref_words: np.ndarray, n_sym: int, m: int):
    bits = qam.unpack_words(ref_words, n_sym * m).reshape(ref_words.shape[0], n_sym, m)
    return qam.bits_to_levels(bits, m)


def resolve(z, ref_words, m, n_ref, lo, hi, max_delay, lat=0):
    """Returns per q a tuple (p, r, d, matches) and the window length."""
    tli, tlq = ref_levels(ref_words, n_ref, m)
    n = np.arange(lo, hi)
    best = []
    for q in range(2):
        cand = None
        for p in range(2):
            for r in range(4):
                li, lq = qam.decide_levels(z[q, lo:hi] * QUARTER[r], m)
                for d in range(-max_delay, max_delay + 1):
                    t = n + d - lat
                    ok = (t >= 0) & (t < n_ref)
                    tc = np.clip(t, 0, n_ref - 1)
                    match = int(np.sum(ok & (li == tli[p, tc]) & (lq == tlq[p, tc])))
                    if cand is None or match > cand[3]:
                        cand = (p, r, d, match)
        best.append(cand)
    return best, max(hi - lo, 0)


def demap_output(z, sync, m):
    """Output bits uint8 [2, N*m] after applying each output's quarter turn."""
    out = []
    for q in range(2):
        r = sync[q][1] if sync is not None else 0
        li, lq = qam.decide_levels(z[q] * QUARTER[r], m)
        out.append(qam.levels_to_bits(li, lq, m).reshape(-1))
    return np.stack(out)


def count(z, sync, ref_words, m, n_ref, lo, hi, lat=0):
    """Bit errors, symbol errors, counted bits/symbols, EVM numerator/denominator."""
    tli, tlq = ref_levels(ref_words, n_ref, m)
    res = dict(bits=0, bit_errors=0, symbols=0, symbol_errors=0, evm_num=0.0, evm_den=0.0)
    if hi <= lo:
        return res
    n = np.arange(lo, hi)
    for q in range(2):
        p, r, d = sync[q][:3]
        t = n + d - lat
        zr = z[q, lo:hi] * QUARTER[r]
        li, lq = qam.decide_levels(zr, m)
        got = qam.levels_to_bits(li, lq, m)
        want = qam.levels_to_bits(tli[p, t], tlq[p, t], m)
        s = qam.levels_to_symbols(tli[p, t], tlq[p, t], m)
        res["bits"] += got.size
        res["bit_errors"] += int(np.sum(got != want))
        res["symbols"] += len(n)
        res["symbol_errors"] += int(np.sum((li != tli[p, t]) | (lq != tlq[p, t])))
        res["evm_num"] += float(np.sum(np.abs(zr - s) ** 2))
        res["evm_den"] += float(np.sum(np.abs(s) ** 2))
    return res
