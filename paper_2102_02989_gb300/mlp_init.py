"""Seeded initial parameters of the screening network (uniform +-1/sqrt(fan_in),
packed W1, b1, W2, b2, W3, b3, w4, b4 with 64 hidden units per layer)."""
import numpy as np

H = 64


def init_params(F: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, n in ((F, H * F), (F, H), (H, H * H), (H, H), (H, H * H), (H, H), (H, H), (H, 1)):
        s = np.sqrt(1.0 / fan_in)
        parts.append(rng.uniform(-s, s, size=n))
    return np.concatenate(parts).astype(np.float32)
