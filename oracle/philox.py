"""Philox4x32-10 counter-based generator and the standard-normal draws xi.

Oracle (test infrastructure only).  The method draws the random input
xi^(m,l) independently for every sample m and level l (Sec. 2.2, the
sentence after eq:delta-notation; Algorithm 1, GradientEstimate "draw xi").
The generator is Philox4x32 with 10 rounds as published by Salmon, Moraes,
Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):

* state: four 32-bit counter words and two 32-bit key words;
* one round: multiply counter word 0 by 0xD2511F53 and word 2 by 0xCD9E8D57
  (full 64-bit products), then the new words are
  (hi(w2*M1) ^ c1 ^ k0, lo(w2*M1), hi(w0*M0) ^ c3 ^ k1, lo(w0*M0));
* between rounds the key is bumped by the Weyl constants 0x9E3779B9,
  0xBB67AE85 (mod 2^32).

Draw layout (this build's own convention, shared with the CUDA path only
through this written definition):
  key     = (seed mod 2^32, seed >> 32)
  counter = (mode pair p, sample index mod 2^32, level, iteration)
Output words (w0, w1) give u1, (w2, w3) give u2 by the 53-bit construction
u = ((w_a >> 5) * 2^26 + (w_b >> 6) + 1) * 2^-53, so u in (0, 1].
Box-Muller: r = sqrt(-2 log u1); xi[2p] = r cos(2 pi u2), xi[2p+1] = r sin(2 pi u2).

Pins: known-answer vectors of Philox4x32-10 (tests/test_oracle_philox.py) and
moment tests of the normals.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter, key):
    """Philox4x32-10 block function.

    counter: uint array [..., 4]; key: uint array [..., 2] (broadcastable).
    Returns uint64 array [..., 4] holding the four 32-bit output words.
    """
    c = np.asarray(counter, dtype=np.uint64) & MASK32
    k = np.asarray(key, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = np.broadcast_to(k[..., 0], c0.shape), np.broadcast_to(k[..., 1], c0.shape)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = c0 * M0  # < 2^64: exact in uint64
        p1 = c2 * M1
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1)


def uniform53(w_hi, w_lo):
    """53-bit uniform in (0, 1] from two 32-bit words."""
    m = (np.asarray(w_hi, np.uint64) >> np.uint64(5)) * np.uint64(1 << 26) + (
        np.asarray(w_lo, np.uint64) >> np.uint64(6))
    return (m.astype(np.float64) + 1.0) * 2.0 ** -53


def _pair_uniforms(seed, iteration, level, samples, n_pairs):
    samples = np.asarray(samples, dtype=np.uint64)
    S = samples.shape[0]
    ctr = np.zeros((S, n_pairs, 4), dtype=np.uint64)
    ctr[..., 0] = np.arange(n_pairs, dtype=np.uint64)[None, :]
    ctr[..., 1] = (samples & MASK32)[:, None]
    ctr[..., 2] = np.uint64(level)
    ctr[..., 3] = np.uint64(iteration)
    seed = int(seed)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    w = philox4x32_10(ctr, key)
    return uniform53(w[..., 0], w[..., 1]), uniform53(w[..., 2], w[..., 3])


def uniforms(seed, iteration, level, samples, n_modes, half_width):
    """xi[s, k] ~ U(-half_width, half_width] from the same counters as `normals`:
    mode 2p from the first uniform of pair p, mode 2p+1 from the second."""
    npairs = (n_modes + 1) // 2
    u1, u2 = _pair_uniforms(seed, iteration, level, samples, npairs)
    xi = np.empty((u1.shape[0], 2 * npairs))
    xi[:, 0::2] = -half_width + 2.0 * half_width * u1
    xi[:, 1::2] = -half_width + 2.0 * half_width * u2
    return xi[:, :n_modes]


def normals(seed, iteration, level, samples, n_modes):
    """xi[s, k] ~ N(0, 1) for the given sample indices (array of int).

    Returns float64 [len(samples), n_modes].  n_modes must be even.
    """
    assert n_modes % 2 == 0
    samples = np.asarray(samples, dtype=np.uint64)
    npairs = n_modes // 2
    S = samples.shape[0]
    ctr = np.zeros((S, npairs, 4), dtype=np.uint64)
    ctr[..., 0] = np.arange(npairs, dtype=np.uint64)[None, :]
    ctr[..., 1] = (samples & MASK32)[:, None]
    ctr[..., 2] = np.uint64(level)
    ctr[..., 3] = np.uint64(iteration)
    seed = int(seed)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    w = philox4x32_10(ctr, key)
    u1 = uniform53(w[..., 0], w[..., 1])
    u2 = uniform53(w[..., 2], w[..., 3])
    r = np.sqrt(-2.0 * np.log(u1))
    xi = np.empty((S, n_modes), dtype=np.float64)
    xi[:, 0::2] = r * np.cos(2.0 * np.pi * u2)
    xi[:, 1::2] = r * np.sin(2.0 * np.pi * u2)
    return xi
