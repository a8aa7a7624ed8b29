"""FP64 oracle: Philox-4x32-10 counter-based generator and Box-Muller normals.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The sSVGD noise Xi (Eq. 25) is drawn on the device from a counter-based
generator so that the update is reproducible; this module re-implements the
same generator from its published definition (Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC 2011) so that the oracle can
consume the identical stream.

Philox-4x32 round on counter (x0, x1, x2, x3) with key (k0, k1):
  (hi0, lo0) = M0 * x0,  (hi1, lo1) = M1 * x2       (32 x 32 -> 64-bit products)
  x' = (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0)
with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by
(0x9E3779B9, 0xBB67AE85); 10 rounds.

Normal draws for element (row i, column c) of an [n, d] array at iteration t
under seed s: counter = (c // 4, i, t mod 2^32, t >> 32), key = (s mod 2^32,
s >> 32). The four output words u0..u3 give two Box-Muller pairs,
U = ((u >> 8) + 1/2) 2^-24,  r = sqrt(-2 ln U_a),  angle = 2 pi U_b,
z0 = r cos(angle), z1 = r sin(angle) from (u0, u1) and z2, z3 likewise from
(u2, u3); column c takes z_{c mod 4}.
"""
import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def _mulhilo(m, x):
    p = np.uint64(m) * x.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint64), (p & np.uint64(MASK)).astype(np.uint64)


def philox4x32_10(ctr, key):
    """ctr: 4 arrays of uint32-valued integers (any common shape); key: 2 of them.
    Returns the 4 output words as uint64 arrays holding 32-bit values."""
    x = [np.asarray(c, dtype=np.uint64) & np.uint64(MASK) for c in ctr]
    k0 = np.asarray(key[0], dtype=np.uint64) & np.uint64(MASK)
    k1 = np.asarray(key[1], dtype=np.uint64) & np.uint64(MASK)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
        hi0, lo0 = _mulhilo(M0, x[0])
        hi1, lo1 = _mulhilo(M1, x[2])
        x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
    return x


def _unit(u):
    return ((u >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24


def normal(n, d, seed, it):
    """Standard-normal array [n, d] of the stream described above."""
    seed = int(seed)
    it = int(it)
    nq = (d + 3) // 4
    q = np.arange(nq, dtype=np.uint64)[None, :]
    i = np.arange(n, dtype=np.uint64)[:, None]
    zero = np.zeros((n, nq), dtype=np.uint64)
    ctr = (q + zero, i + zero, zero + np.uint64(it & MASK),
           zero + np.uint64((it >> 32) & MASK))
    key = (np.uint64(seed & MASK), np.uint64((seed >> 32) & MASK))
    u = philox4x32_10(ctr, key)
    z = np.empty((n, nq, 4))
    for pair in (0, 1):
        ua, ub = _unit(u[2 * pair]), _unit(u[2 * pair + 1])
        r = np.sqrt(-2.0 * np.log(ua))
        ang = 2.0 * np.pi * ub
        z[:, :, 2 * pair] = r * np.cos(ang)
        z[:, :, 2 * pair + 1] = r * np.sin(ang)
    return z.reshape(n, nq * 4)[:, :d]
