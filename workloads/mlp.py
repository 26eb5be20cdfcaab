"""Seeded inputs of the learned surrogate: layer widths, initial weights and the
box its inputs are normalised to.  Random numbers the training draws (initial
weights, training points) are made here and passed to both the CUDA library
and the oracle; no arithmetic of the method lives in this module.
"""

from __future__ import annotations

import numpy as np

HIDDEN = 256
N_HIDDEN_LAYERS = 3

# theta box of the scans (|eps| <= 0.3, mu_hat in [0, 3]) as centre / half width
BOX_CENTRE = np.array([0.0, 0.0, 0.0, 0.0, 1.5], dtype=np.float32)
BOX_HALF = np.array([0.3, 0.3, 0.3, 0.3, 1.5], dtype=np.float32)


def layer_shapes(n_out, n_in=5, hidden=HIDDEN, n_hidden=N_HIDDEN_LAYERS):
    """[(out, in), ...] of the four linear layers 5 -> 256 -> 256 -> 256 -> n_out."""
    dims = [n_in] + [hidden] * n_hidden + [n_out]
    return [(dims[k + 1], dims[k]) for k in range(len(dims) - 1)]


def init_weights(n_out, seed=5, hidden=HIDDEN, n_hidden=N_HIDDEN_LAYERS):
    """Normal weights with variance 2 / fan_in (He et al. 2015), zero biases,
    float32.  Returns [(W [out, in], b [out]), ...]."""
    rng = np.random.default_rng(seed)
    params = []
    for out, fan_in in layer_shapes(n_out, hidden=hidden, n_hidden=n_hidden):
        W = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(out, fan_in)).astype(np.float32)
        params.append((W, np.zeros(out, dtype=np.float32)))
    return params


def round_to_bf16(x):
    """Nearest BF16 value of each float32 (round to nearest even), as float32:
    inputs that the tensor cores take without rounding."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)
