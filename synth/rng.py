"""Counter-based random numbers that give identical values on CPU and GPU.

Every random value is a pure function of (key, counter), so a graph drawn with torch on a GPU is
bit-identical to the same graph drawn on the host. The mixer is the 32-bit "lowbias32" integer
hash (two xor-shift-multiply rounds, constants 0x7feb352d and 0x846ca68b, found by
C. Wellons' hash prospector). Products are formed from 16-bit halves so that int64 tensor
arithmetic never overflows.
"""

import torch

M32 = 0xFFFFFFFF
_C1 = 0x7FEB352D
_C2 = 0x846CA68B


def _mul32_t(x: torch.Tensor, c: int) -> torch.Tensor:
    """(x * c) mod 2^32 for int64 tensors holding values in [0, 2^32)."""
    lo = c & 0xFFFF
    hi = c >> 16
    return (x * lo + (((x * hi) & 0xFFFF) << 16)) & M32


def mix32(x: torch.Tensor) -> torch.Tensor:
    """lowbias32 on an int64 tensor of 32-bit values."""
    x = x ^ (x >> 16)
    x = _mul32_t(x, _C1)
    x = x ^ (x >> 15)
    x = _mul32_t(x, _C2)
    x = x ^ (x >> 16)
    return x


def mix32_int(x: int) -> int:
    """lowbias32 on a Python int (host-side key derivation)."""
    x &= M32
    x ^= x >> 16
    x = (x * _C1) & M32
    x ^= x >> 15
    x = (x * _C2) & M32
    x ^= x >> 16
    return x


def derive_key(seed: int, *purpose: int) -> int:
    """A 32-bit key for one random stream, from the workload seed and a purpose tuple."""
    k = mix32_int((seed & M32) ^ 0x9E3779B9)
    k = mix32_int(k ^ ((seed >> 32) & M32))
    for p in purpose:
        k = mix32_int(k ^ mix32_int((p & M32) + 0x632BE5AB))
    return k


def uniform53(idx: torch.Tensor, key_a: int, key_b: int) -> torch.Tensor:
    """Uniform float64 in [0, 1) with 53 random bits, one per int64 counter in ``idx``."""
    lo = idx & M32
    hi = (idx >> 32) & M32
    w1 = mix32(mix32(lo ^ key_a) ^ hi)
    w2 = mix32(mix32(lo ^ key_b) ^ hi)
    bits = (w1 >> 5) * 67108864 + (w2 >> 6)
    return bits.to(torch.float64) * (1.0 / 9007199254740992.0)


def uniform53_int(i: int, key_a: int, key_b: int) -> float:
    """Host-side scalar twin of :func:`uniform53` (same values)."""
    lo = i & M32
    hi = (i >> 32) & M32
    w1 = mix32_int(mix32_int(lo ^ key_a) ^ hi)
    w2 = mix32_int(mix32_int(lo ^ key_b) ^ hi)
    return ((w1 >> 5) * 67108864 + (w2 >> 6)) * (1.0 / 9007199254740992.0)
