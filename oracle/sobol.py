"""Sobol low-discrepancy points in [0, 1)^d, written from their published
definition (test infrastructure: only tests and the benchmark's CPU leg use it).

Sobol (1967) with the direction numbers of Joe & Kuo (2008, "Constructing Sobol
sequences with better two-dimensional projections"): dimension 1 uses
m_k = 1; dimension j > 1 uses a primitive polynomial of degree s with inner
coefficient bits a and initial odd integers m_1..m_s, and

    m_k = 2 a_1 m_{k-1} xor 4 a_2 m_{k-2} xor ... xor 2^(s-1) a_(s-1) m_(k-s+1)
          xor 2^s m_(k-s) xor m_(k-s)                      (k > s),

v_k = m_k / 2^k.  Point n (Gray-code order, Antonov & Saleev 1979) is the xor of
v_k over the set bits k of gray(n) = n xor (n >> 1); the sequence starts at 0.
"""

from __future__ import annotations

import numpy as np

BITS = 32

# (s, a, m_1..m_s) for dimensions 2..5 of the Joe-Kuo table
JOE_KUO = [
    (1, 0, (1,)),
    (2, 1, (1, 3)),
    (3, 1, (1, 3, 1)),
    (3, 2, (1, 1, 1)),
]


def direction_numbers(dim):
    """V[j][k] = m_k << (32 - k), k = 1..32, for dimensions j < dim (uint64 holding 32 bits)."""
    if dim > 1 + len(JOE_KUO):
        raise ValueError("only %d dimensions are tabulated" % (1 + len(JOE_KUO)))
    V = np.zeros((dim, BITS), dtype=np.uint64)
    for k in range(1, BITS + 1):
        V[0, k - 1] = 1 << (BITS - k)
    for j in range(1, dim):
        s, a, m_init = JOE_KUO[j - 1]
        m = [0] + list(m_init)           # 1-based
        for k in range(s + 1, BITS + 1):
            val = m[k - s] ^ (m[k - s] << s)
            for i in range(1, s):
                if (a >> (s - 1 - i)) & 1:
                    val ^= m[k - i] << i
            m.append(val)
        for k in range(1, BITS + 1):
            V[j, k - 1] = m[k] << (BITS - k)
    return V


def sobol_points(n_start, count, dim):
    """Points n_start .. n_start + count - 1 as float64 [count, dim]."""
    V = direction_numbers(dim)
    out = np.zeros((count, dim), dtype=np.float64)
    for r in range(count):
        n = n_start + r
        g = n ^ (n >> 1)
        x = np.zeros(dim, dtype=np.uint64)
        k = 0
        while g:
            if g & 1:
                x ^= V[:, k]
            g >>= 1
            k += 1
        out[r] = x.astype(np.float64) / float(1 << BITS)
    return out
