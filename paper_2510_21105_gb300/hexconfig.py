"""Hexadecimal spin-configuration format (Sec. 3 of arXiv 2510.21105).

The paper publishes its best G63 configuration as a hex string: the digits
expand to one bit per variable, variable 1 first and most significant bit
first within each digit, and a 0 bit means spin -1, a 1 bit spin +1. These
helpers convert between that string and an int8 vector of +-1 spins so that
results of this library can be exported and re-imported in the same form.
"""
from __future__ import annotations

import numpy as np


def decode(hexstr: str, n: int | None = None) -> np.ndarray:
    """Hex string -> int8 spins (+1/-1), variable 1 first. If n is given the
    string must hold at least n bits and any padding bits are dropped."""
    s = "".join(hexstr.split()).lower()
    if not s or any(c not in "0123456789abcdef" for c in s):
        raise ValueError("not a hexadecimal string")
    nib = np.frombuffer(bytes.fromhex(s if len(s) % 2 == 0 else s + "0"), np.uint8)
    bits = np.unpackbits(nib)[: 4 * len(s)]
    if n is not None:
        if n > len(bits):
            raise ValueError(f"{len(bits)} bits cannot hold {n} variables")
        bits = bits[:n]
    return np.where(bits == 1, 1, -1).astype(np.int8)


def encode(x) -> str:
    """int8 spins (+1/-1) -> hex string, zero-padded to a whole digit."""
    x = np.asarray(x)
    if not np.all((x == 1) | (x == -1)):
        raise ValueError("spins must be +1 or -1")
    bits = (x == 1).astype(np.uint8)
    pad = (-len(bits)) % 8
    packed = np.packbits(np.concatenate([bits, np.zeros(pad, np.uint8)]))
    return packed.tobytes().hex()[: (len(bits) + 3) // 4]
