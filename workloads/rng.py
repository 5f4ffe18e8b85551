"""PCG32 random stream (O'Neill 2014, "PCG: A family of simple fast
space-efficient statistically good algorithms", the XSH-RR 64/32 member).

Used to draw the seeded random vectors on which matrix-vector products are
timed and compared.  The stream is generated on the host once and the same
numbers are handed to the oracle and to the GPU library.
"""
import numpy as np

_MULT = 6364136223846793005
_MASK64 = (1 << 64) - 1


class PCG32:
    """PCG-XSH-RR with 64-bit state and 32-bit output (O'Neill's reference
    ``pcg32_random_r`` semantics, re-derived from the published definition)."""

    def __init__(self, seed: int, stream: int = 54):
        self.inc = ((stream << 1) | 1) & _MASK64
        self.state = 0
        self.next_u32()
        self.state = (self.state + (seed & _MASK64)) & _MASK64
        self.next_u32()

    def next_u32(self) -> int:
        old = self.state
        self.state = (old * _MULT + self.inc) & _MASK64
        xorshifted = (((old >> 18) ^ old) >> 27) & 0xFFFFFFFF
        rot = old >> 59
        return ((xorshifted >> rot) | (xorshifted << ((-rot) & 31))) & 0xFFFFFFFF

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) built from two 32-bit draws (53 random bits)."""
        out = np.empty(n, dtype=np.float64)
        for i in range(n):
            hi = self.next_u32() >> 5          # 27 bits
            lo = self.next_u32() >> 6          # 26 bits
            out[i] = (hi * 67108864.0 + lo) / 9007199254740992.0
        return out


def random_complex_vectors(seed: int, count: int, length: int) -> np.ndarray:
    """``count`` complex vectors of ``length`` entries, re and im ~ U(-1, 1).

    For long vectors the PCG32 stream seeds numpy's PCG64 generator (a
    different member of the same family) so that generation stays fast; the
    first draw of the PCG32 stream is the seed, which keeps the whole vector a
    function of ``seed`` alone.
    """
    total = count * length
    if total <= 4096:
        u = PCG32(seed).uniform(2 * total)
    else:
        s = PCG32(seed)
        g = np.random.Generator(np.random.PCG64((s.next_u32() << 32) | s.next_u32()))
        u = g.random(2 * total)
    z = (2.0 * u[0::2] - 1.0) + 1j * (2.0 * u[1::2] - 1.0)
    return z.reshape(count, length)
