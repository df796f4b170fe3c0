"""Prime-number coding of Linhart and Shamir, as summarised in Sec. 1.3 (Eq. 1-3).

TEST INFRASTRUCTURE ONLY (see the ``oracle`` package docstring).

This is the method the paper starts from, carried out in exact Python
integers so that the precision problem of Sec. 1.3.5 does not arise.  It is an
independent route to the mismatch counts the oracle computes with the Table 3
dictionary, and therefore a pin for it on tiny inputs:

* every letter a_i gets a prime k_i, all primes larger than m (Sec. 1.3);
* ``M`` is the product of the primes; text letter a_i is coded ``e_i = M / k_i``
  (Sec. 1.3.1);
* a class S is coded by the unique ``n_S`` in [0, M) that is 0 modulo k_i for
  every i in S and 1 modulo k_j for every j outside S (Eq. 1), found by the
  Chinese remainder theorem;
* the sum ``sum_j n_{S_j} * e_{t[i+j]}`` (Eq. 2, read as a correlation so that
  p[j] meets t[i+j]) is 0 modulo M exactly at an exact match (Eq. 3).

Mismatch counts come out of the same sum.  Modulo k_a every e_t with t != a
vanishes and ``n_S`` is 0 or 1, so ``sum mod k_a = (M/k_a) * c_a mod k_a``
where c_a counts the pattern positions whose class excludes a while the text
has a.  Because every c_a <= m < k_a, ``c_a = (sum mod k_a) * (M/k_a)^-1 mod
k_a`` exactly, and the window's mismatch count is ``sum_a c_a``.

The character classes below are the "Character class" column of Table 2, kept
as sets of letters; they are deliberately not derived from the oracle's codes.
"""
from __future__ import annotations

ALPHABET = "ACGT"

# Table 2, "Character class" column, as letter sets.  "-" is the empty class
# (it matches nothing: Table 3 row "-" is all ones).
CLASSES = {
    "A": "A", "C": "C", "G": "G", "T": "T",
    "M": "AC", "R": "AG", "W": "AT", "S": "CG", "Y": "CT", "K": "GT",
    "V": "ACG", "H": "ACT", "D": "AGT", "B": "CGT",
    "N": "ACGT", "-": "",
}


def is_prime(x: int) -> bool:
    if x < 2:
        return False
    if x % 2 == 0:
        return x == 2
    d = 3
    while d * d <= x:
        if x % d == 0:
            return False
        d += 2
    return True


def smallest_primes_above(m: int, count: int = 4) -> list[int]:
    """The ``count`` smallest primes strictly greater than m (Sec. 1.3)."""
    out, x = [], m + 1
    while len(out) < count:
        if is_prime(x):
            out.append(x)
        x += 1
    return out


def modulus(primes: list[int]) -> int:
    M = 1
    for q in primes:
        M *= q
    return M


def text_codes(primes: list[int]) -> dict[str, int]:
    """Sec. 1.3.1: letter a_i -> e_i = M / k_i."""
    M = modulus(primes)
    return {a: M // q for a, q in zip(ALPHABET, primes)}


def class_code(letters: str, primes: list[int]) -> int:
    """Eq. 1 solved by the Chinese remainder theorem.

    Returns the unique n_S in [0, M) with n_S = 0 (mod k_i) for letters in the
    class and n_S = 1 (mod k_j) for the others.
    """
    M = modulus(primes)
    n = 0
    for a, q in zip(ALPHABET, primes):
        r = 0 if a in letters else 1
        Mq = M // q
        n += r * Mq * pow(Mq, -1, q)
    return n % M


def pattern_codes(pattern: str, primes: list[int]) -> list[int]:
    return [class_code(CLASSES.get(ch.upper(), ""), primes) for ch in pattern]


def window_sums(text: str, pattern: str, primes: list[int]) -> list[int]:
    """Eq. 2 evaluated directly (no FFT) for windows 0..n-m."""
    e = text_codes(primes)
    ns = pattern_codes(pattern, primes)
    n, m = len(text), len(pattern)
    return [sum(ns[j] * e[text[i + j].upper()] for j in range(m)) for i in range(n - m + 1)]


def exact_locations(text: str, pattern: str, primes: list[int] | None = None) -> list[int]:
    """Eq. 3: 0-based locations whose sum is 0 modulo M."""
    primes = primes or smallest_primes_above(len(pattern))
    M = modulus(primes)
    return [i for i, s in enumerate(window_sums(text, pattern, primes)) if s % M == 0]


def mismatch_counts(text: str, pattern: str, primes: list[int] | None = None) -> list[int]:
    """Per-window mismatch counts decoded from the Eq. 2 sums (needs primes > m)."""
    primes = primes or smallest_primes_above(len(pattern))
    if min(primes) <= len(pattern):
        raise ValueError("count decoding needs every prime larger than m")
    M = modulus(primes)
    out = []
    for s in window_sums(text, pattern, primes):
        total = 0
        for q in primes:
            Mq = M // q
            total += (s % q) * pow(Mq % q, -1, q) % q
        out.append(total)
    return out


def pair_is_match(text_letter: str, pattern_symbol: str, primes: list[int]) -> bool:
    """The per-pair residue test the paper keeps (Sec. 2): e_t * n_S = 0 (mod M)."""
    M = modulus(primes)
    e = text_codes(primes)[text_letter]
    n = class_code(CLASSES.get(pattern_symbol, ""), primes)
    return (e * n) % M == 0
