"""Lift heights omega(i) in [1, 2^20] from a counter-based generator.

Test infrastructure only (see oracle/__init__.py).

The paper only asks for a generic lifting function (Sec. 4.1, "for almost all
choices") with rational values; it names no generator.  The reading used here:
SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state advances by the golden-ratio increment
0x9E3779B97F4A7C15 and each output is the state passed through the published
mixing function (xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift 27, multiply
0x94D049BB133111EB, xor-shift 31).

    seed'    = mix(seed XOR attempt * 0xD1B54A32D192ED03)
    omega(i) = 1 + (mix(seed' + (i + 1) * 0x9E3779B97F4A7C15) >> 44),  i = 0 .. N-1

`attempt` counts re-lifts after a tie.  Arithmetic is modulo 2^64.
"""

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
ATTEMPT_MULT = 0xD1B54A32D192ED03


def mix(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def lifts(npts: int, seed: int, attempt: int = 0):
    s = mix((seed ^ (attempt * ATTEMPT_MULT)) & MASK)
    return [1 + (mix((s + (i + 1) * GOLDEN) & MASK) >> 44) for i in range(npts)]
