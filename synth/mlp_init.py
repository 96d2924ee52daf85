"""Seeded initial weights of the learned-initial-value network (random
numbers the training draws, generated once on the host and passed to both
the GPU trainer and the FP64 oracle).  No arithmetic of the method here."""
import numpy as np

from .sky import rng_for

SHAPES = (("W1", (256, 1024)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (4, 256)), ("b3", (4,)))


def mlp_init(seed: int = 0) -> dict:
    """He-normal weights (std sqrt(2 / fan_in)) for the GELU layers, a
    0.1 / sqrt(fan_in) output layer, zero biases."""
    rng = rng_for(5, seed)
    w = {}
    w["W1"] = rng.normal(0.0, np.sqrt(2.0 / 1024), (256, 1024))
    w["b1"] = np.zeros(256)
    w["W2"] = rng.normal(0.0, np.sqrt(2.0 / 256), (256, 256))
    w["b2"] = np.zeros(256)
    w["W3"] = rng.normal(0.0, 0.1 / np.sqrt(256), (4, 256))
    w["b3"] = np.zeros(4)
    return w
