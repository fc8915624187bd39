"""Small helpers for the tests, written from the problem statement (Section II):
a k-mer key is a k-digit base-4 number (A0 C1 G2 T3, first base most significant).
These work digit by digit on Python integers and share nothing with either the
oracle or the CUDA library."""


def digits(key: int, k: int) -> list[int]:
    out = []
    for _ in range(k):
        out.append(key % 4)
        key //= 4
    return out[::-1]


def rc_key(key: int, k: int) -> int:
    """value of the reverse complement: reverse the digits, map d -> 3 - d"""
    v = 0
    for d in reversed(digits(key, k)):
        v = v * 4 + (3 - d)
    return v


def key_to_str(key: int, k: int) -> str:
    return "".join("ACGT"[d] for d in digits(key, k))


def keys_as_ints(keys) -> list[int]:
    """uint64[n] or uint64[n, 2] (lo, hi) -> python ints"""
    if getattr(keys, "ndim", 1) == 2:
        return [int(lo) | (int(hi) << 64) for lo, hi in keys]
    return [int(x) for x in keys]
