"""Path numbering and path selection (oracle; test infrastructure only).

Numbering (the paper leaves it open; reading used throughout): cross-cut gates
are ordered by (cycle, smaller qubit, larger qubit). Gate i with r_i terms
(r_i in {1, 2, 4}) owns log2(r_i) bits of the path id; the earliest gate owns
the most significant bits, so a range of path ids is a subtree of the path tree
(Section 2: processes own path prefixes and run all suffixes).

Selection (Eq. 3 and Section 3):
  RANGE    - ids first .. first+count-1 (Eq. 3 takes j = 0 .. f 2^x - 1).
  FRACTION - selection at prefix granularity, as the paper skips whole processes:
             with x the number of path bits and x_s the prefix bits (default
             max(0, x - 7)), K = max(1, floor(f 2^x_s + 1e-9)) prefixes are taken,
             the images of 0..K-1 under a keyed Feistel permutation of [0, 2^x_s),
             and every prefix contributes all 2^(x - x_s) suffixes.
             f_actual = K / 2^x_s.
  LIST     - the given ids.

Feistel permutation of w-bit values (our definition): h = ceil(w/2); a value v
< 2^(2h) is split into L = v >> h and R = v mod 2^h; four rounds
(L, R) <- (R, L xor (F(key, r, R) mod 2^h)), r = 0..3; result (L << h) | R.
Values >= 2^w are mapped again (cycle walking) until they fall below 2^w.
F(key, r, R) = mix(key xor (R + (r + 1) * 0x9E3779B97F4A7C15 mod 2^64)),
mix(z) = the SplitMix64 output function
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
    z ^ (z >> 31)   (all mod 2^64).
"""
import numpy as np

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def mix(z):
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def feistel(v, w, key):
    if w == 0:
        return 0
    h = (w + 1) // 2
    hm = (1 << h) - 1
    while True:
        L, R = v >> h, v & hm
        for r in range(4):
            f = mix(key ^ ((R + (r + 1) * GOLDEN) & M64)) & hm
            L, R = R, L ^ f
        v = (L << h) | R
        if v < (1 << w):
            return v


def digits(path, bits_per_gate):
    """Branch digit of each cross gate for path id `path` (MSB = earliest)."""
    total = sum(bits_per_gate)
    out = []
    shift = total
    for b in bits_per_gate:
        shift -= b
        out.append((path >> shift) & ((1 << b) - 1))
    return out


def select_range(first, count):
    return np.arange(first, first + count, dtype=np.uint64)


def fraction_prefixes(x_bits, f, seed, x_s=None):
    """Sorted selected prefixes and f_actual for FRACTION mode."""
    if x_s is None or x_s < 0:
        x_s = max(0, x_bits - 7)
    K = max(1, int(np.floor(f * (1 << x_s) + 1e-9)))
    K = min(K, 1 << x_s)
    pre = sorted(feistel(i, x_s, seed) for i in range(K))
    return pre, x_s, K / float(1 << x_s)


def select_fraction(x_bits, f, seed, x_s=None):
    pre, x_s, fa = fraction_prefixes(x_bits, f, seed, x_s)
    suf = 1 << (x_bits - x_s)
    ids = [(p << (x_bits - x_s)) | s for p in pre for s in range(suf)]
    return np.array(ids, dtype=np.uint64), fa
