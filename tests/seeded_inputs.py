"""Seeded synthetic inputs shared by the oracle tests and the GPU tests.

Holds no arithmetic of the method: only random numbers drawn from a stated
generator (SplitMix64, Steele, Lea & Flood 2014) and their standard-normal
transform (Box-Muller), used to perturb circuit angles.
"""
import math

MASK = (1 << 64) - 1


def splitmix64_stream(seed):
    x = seed & MASK
    while True:
        x = (x + 0x9E3779B97F4A7C15) & MASK
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        yield z ^ (z >> 31)


def normals(seed, count):
    """count standard normal deviates (Box-Muller on 53-bit uniforms)."""
    g = splitmix64_stream(seed)
    out = []
    while len(out) < count:
        u1 = ((next(g) >> 11) + 1) / 9007199254740993.0     # (0, 1]
        u2 = (next(g) >> 11) / 9007199254740992.0
        r = math.sqrt(-2.0 * math.log(u1))
        out.append(r * math.cos(2 * math.pi * u2))
        out.append(r * math.sin(2 * math.pi * u2))
    return out[:count]


def mix64(z):
    """SplitMix64's output finaliser applied to z."""
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def ensemble_instance(s):
    """Instance s of the batched ensemble: n uniform in 12..24, depth uniform
    in 10..40, grid with 3 rows (n <= 15) or 4 rows, ceil(n / rows) columns,
    the last rows*cols - n sites of the last row dead."""
    n = 12 + mix64(s) % 13
    depth = 10 + mix64(s ^ 0xD1B54A32D192ED03) % 31
    rows = 3 if n <= 15 else 4
    cols = -(-n // rows)
    dead = [0] * (rows * cols)
    for k in range(rows * cols - n):
        dead[rows * cols - 1 - k] = 1
    return n, depth, rows, cols, dead
