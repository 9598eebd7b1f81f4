"""Inputs for the corrector tests (CPU pins and GPU parity): integer-valued networks whose
every stored value is exact in bfloat16 and every sum exact in float32, so that any
correct evaluation -- in any summation order -- gives the same bits.

Hidden 32 -> 32 layers: output channel o reads two entries, input channel o at one random
tap and input channel (o + 7) mod 32 at another, each +-1; every input channel is then
read by exactly two entries, so forward activations and backward gradients at most double
per layer.  First layer: taps in {-1, 0, 1}, biases in {0, 1}; last layer: sparse taps in
{-1, 0, 1}.  With images in {-1, 0, 1} the activations stay below 2 * 2 * 2 * 2 * 11 and the
pre-activation gradients below 2^4 * 9 for a loss gradient in {-1, 0, 1}.
"""
import numpy as np

C = 32


def int_params(seed: int, channels: int = C):
    rng = np.random.default_rng(seed)
    ps = [(rng.integers(-1, 2, size=(channels, 1, 3, 3)).astype(np.float64),
           rng.integers(0, 2, size=channels).astype(np.float64))]
    for _ in range(4):
        w = np.zeros((channels, channels, 3, 3))
        for o in range(channels):
            ta, tb = rng.integers(0, 9, 2)
            w[o, o, ta // 3, ta % 3] = rng.choice([-1.0, 1.0])
            w[o, (o + 7) % channels, tb // 3, tb % 3] = rng.choice([-1.0, 1.0])
        ps.append((w, rng.integers(-1, 2, size=channels).astype(np.float64)))
    w6 = rng.integers(-1, 2, size=(1, channels, 3, 3)) * (rng.random((1, channels, 3, 3)) < 0.3)
    ps.append((w6.astype(np.float64), np.zeros(1)))
    return ps


def int_images(rng, shape, density: float) -> np.ndarray:
    return (rng.integers(-1, 2, size=shape) * (rng.random(shape) < density)).astype(np.float64)


def flatten(ps) -> np.ndarray:
    """The library's parameter layout: per layer its weights [co][ci][3][3], then biases."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in ps]).astype(np.float32)


def unflatten(flat, channels: int = C, layers: int = 6):
    dims = [1] + [channels] * (layers - 1) + [1]
    out, off = [], 0
    for k in range(layers):
        ci, co = dims[k], dims[k + 1]
        w = np.asarray(flat[off:off + co * ci * 9], np.float64).reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = np.asarray(flat[off:off + co], np.float64)
        off += co
        out.append((w, b))
    return out


def abs_gradient_bound(cnn, ps, cache, gy):
    """Per weight and bias, sum over pixels of |dL/dz| |input|: the backward pass of the
    network with |weights| on |dL/dy| through the same ReLU masks.  Every partial sum of a
    gradient is bounded by it, whatever the order."""
    aps = [(np.abs(w), np.abs(b)) for w, b in ps]
    acache = [np.abs(h) for h in cache]
    grads, _ = cnn.backward(aps, acache, np.abs(gy))
    return grads
