"""Counter-based uniform draws for the initial guess (Section 6 initialisation).

splitmix64 (S. Vigna, public-domain reference generator, 2015) evaluated at a
counter instead of a running state:  z = seed + (c + 1) * GOLDEN (mod 2^64),
then the three-step xor-shift-multiply finaliser.  The 53 high bits give a
double u in [0, 1); the draw used is 2u - 1 in [-1, 1).

Counter layout (one draw per coordinate):
    c = point * 2^32 + stream * 2^31 + j * 2^12 + coord
with stream 0 for x_j (j = 0..N-1) and stream 1 for p_j (j = 1..N);
coord < 4096, j < 2^19.  The CUDA side implements the same published
generator on its own; the two share no code.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_at(seed, counter):
    """splitmix64 output for `counter` (uint64 array) under `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed, point, stream, j, coord):
    """2u - 1 for the broadcast index arrays (point, stream, j, coord)."""
    c = (np.asarray(point, dtype=np.uint64) << np.uint64(32)) \
        + (np.asarray(stream, dtype=np.uint64) << np.uint64(31)) \
        + (np.asarray(j, dtype=np.uint64) << np.uint64(12)) \
        + np.asarray(coord, dtype=np.uint64)
    z = splitmix64_at(seed, c)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0
