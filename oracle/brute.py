"""TEST INFRASTRUCTURE ONLY - a string-level k-mer counter for tiny inputs.

It counts substrings as Python strings straight from the problem statement
(Section II: frequencies of all length-k strings over {A,C,G,T} in the reads),
with no integer encoding at all: a window counts iff all its characters are
bases; lowercase is read as uppercase; the canonical form of a string is the
lexicographically smaller of it and its reverse complement.  Keys are converted
to integers only at the end (digit value A0 C1 G2 T3, first base most
significant), so that comparing with the C oracle checks that oracle's encoding,
masking and canonicalisation.
"""
from __future__ import annotations

from collections import Counter

_COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}
_DIGIT = {"A": 0, "C": 1, "G": 2, "T": 3}
_UPPER = {"A": "A", "C": "C", "G": "G", "T": "T", "a": "A", "c": "C", "g": "G", "t": "T"}


def revcomp(s: str) -> str:
    return "".join(_COMP[c] for c in reversed(s))


def string_counts(reads: list[bytes], k: int, canonical: bool) -> Counter:
    c: Counter = Counter()
    for r in reads:
        s = r.decode("latin-1")
        for j in range(0, len(s) - k + 1):
            w = s[j:j + k]
            if any(ch not in _UPPER for ch in w):
                continue
            w = "".join(_UPPER[ch] for ch in w)
            if canonical:
                w = min(w, revcomp(w))
            c[w] += 1
    return c


def string_to_int(w: str) -> int:
    v = 0
    for ch in w:
        v = v * 4 + _DIGIT[ch]
    return v


def sorted_histogram(reads: list[bytes], k: int, canonical: bool):
    """[(key_int, count)] ascending by key."""
    c = string_counts(reads, k, canonical)
    return sorted((string_to_int(w), n) for w, n in c.items())
