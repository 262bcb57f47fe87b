"""Oracle copy of the counter-based random stream used by the initial conditions.

Test infrastructure only (see ``oracle/__init__``).

Definition (SplitMix64, Steele, Lea & Flood, OOPSLA 2014): the generator's
state advances by gamma = 0x9E3779B97F4A7C15 per draw and each output is the
state passed through the finaliser
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.
Stream position c of a generator started from state 0 therefore outputs
mix((c + 1) * gamma mod 2^64).  A run with seed s reads positions
c = s * 2^40 + i, i = 0, 1, 2, ...

Uniforms: u = (v >> 11) * 2^-53 in [0, 1);  u1 = ((v >> 11) + 1) * 2^-53 in (0, 1].
Normals (Box-Muller): g = sqrt(-2 ln u1(v_a)) * cos(2 pi u(v_b)) (and sin for the pair).
The GPU library implements the same published definition independently.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
SEED_STRIDE = 1 << 40


def splitmix64(counter):
    """Output of SplitMix64 at stream positions ``counter`` (uint64 array)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (c + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def positions(seed, index):
    with np.errstate(over="ignore"):
        return np.uint64(seed) * np.uint64(SEED_STRIDE) + np.asarray(index, dtype=np.uint64)


def uniform01(v):
    """[0, 1) double from a 64-bit draw."""
    return (np.asarray(v, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def uniform01_open0(v):
    """(0, 1] double from a 64-bit draw (safe argument for log)."""
    return ((np.asarray(v, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
