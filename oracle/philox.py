"""Philox4x32-10 counter-based generator, written from its published definition.

TEST INFRASTRUCTURE. This module belongs to the FP64 CPU oracle: only tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
The CUDA library carries its own, independent implementation.

Definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11, section 3.2): a 4-word counter and a 2-word key; each of the
ten rounds multiplies counter words 0 and 2 by the constants M0, M1, keeps
both 32-bit halves of each 64-bit product, and permutes/xors them with the
other counter words and the key; the key is bumped by the Weyl constants W0,
W1 between rounds.

The paper (vMAP, section 3.3 "Depth Guided Sampling") draws random sample
depths but names no generator; this counter-based one is the reading taken
so that both sides of the parity tests can draw the very same integers.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter, key):
    """Apply Philox4x32 with 10 rounds.

    counter: integer array of shape (..., 4) (values < 2**32).
    key:     integer array of shape (..., 2) or a pair, broadcast against counter.
    Returns a uint32 array of shape (..., 4).
    """
    c = np.asarray(counter, dtype=np.uint64) & MASK32
    k = np.broadcast_to(np.asarray(key, dtype=np.uint64) & MASK32,
                        c.shape[:-1] + (2,)).copy()
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0], k[..., 1]
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(W0)) & MASK32
            k1 = (k1 + np.uint64(W1)) & MASK32
        p0 = M0 * c0            # < 2**64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def seed_key(seed):
    """Split a 64-bit seed into the two key words (low word first)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)


def ray_words(seed, stream, step, rays, n_words):
    """The random words one ray of one object draws in one step.

    Counter layout (a reading of ours; the paper does not fix one):
    (ray index within the object's batch, block index, the object's own step
    count, the object's stream id); key = the 64-bit seed. Word w of a ray is
    lane w % 4 of block w // 4.  Returns uint32 array (len(rays), n_words).
    """
    rays = np.asarray(rays, dtype=np.uint64)
    n_blocks = (n_words + 3) // 4
    ctr = np.zeros((rays.size, n_blocks, 4), dtype=np.uint64)
    ctr[..., 0] = rays[:, None]
    ctr[..., 1] = np.arange(n_blocks, dtype=np.uint64)[None, :]
    ctr[..., 2] = np.uint64(int(step) & 0xFFFFFFFF)
    ctr[..., 3] = np.uint64(int(stream) & 0xFFFFFFFF)
    out = philox4x32_10(ctr, seed_key(seed))
    return out.reshape(rays.size, n_blocks * 4)[:, :n_words]


def word_to_unit(w):
    """Map a 32-bit word to an open-interval uniform in (0, 1).

    u = (2 * (w >> 9) + 1) * 2**-24: an odd multiple of 2**-24, exactly
    representable in float32 and float64, never 0 or 1.
    """
    w = np.asarray(w, dtype=np.uint64)
    return ((w >> np.uint64(9)) * np.uint64(2) + np.uint64(1)).astype(np.float64) * 2.0 ** -24


def word_to_index(w, n):
    """Uniform index in [0, n): the high word of the 64-bit product w * n."""
    w = np.asarray(w, dtype=np.uint64)
    return ((w * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
