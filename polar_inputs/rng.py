"""SplitMix64: the public-domain 64-bit mixing generator (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), written out from
its published definition.  It seeds every synthetic workload so that the CPU
oracle and the GPU library receive bit-identical input arrays.
"""

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """Counter-based SplitMix64 stream.  ``uniform()`` returns a double in [0, 1)
    built from the top 53 bits of each 64-bit output."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_in(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()
