"""The learned corrector's kernels against the oracle CNN, and a training run that shows
the corrector moving fast reconstructions towards direct-FBP ones.

Tolerances: hidden activations and the 32 -> 32 weights are bf16 (8 significant bits) in the
kernels, float64 in the oracle; the residual net(x) and the gradients are compared in
relative L2 norm at 3e-2 (a wrong tap, channel or sign gives O(1) errors).
"""
import numpy as np
import pytest

import phantoms
from oracle import cnn as ocnn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


def unflatten(flat):
    dims = [1] + [32] * 5 + [1]
    out, off = [], 0
    for k in range(6):
        ci, co = dims[k], dims[k + 1]
        w = flat[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = flat[off:off + co]
        off += co
        out.append((w.astype(np.float64), b.astype(np.float64)))
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def smooth_images(rng, B, N):
    x = rng.normal(size=(B, N + 4, N + 4))
    return (x[:, :-4, :-4] + x[:, 2:-2, 2:-2] + x[:, 4:, 4:]) / 3.0


def test_forward_matches_oracle(fbp, torch):
    from paper_2007_06289_gb300 import corrector
    rng = np.random.default_rng(0)
    B, N = 2, 32
    flat = corrector.init_params(seed=1, scale=2.0)
    flat[-289:] *= 10.0                              # a last layer of normal size
    flat[:] += rng.normal(0, 0.02, flat.size).astype(np.float32)   # nonzero biases
    x = smooth_images(rng, B, N).astype(np.float32)
    params = torch.tensor(flat, device="cuda")
    y = corrector.infer(params, torch.tensor(x, device="cuda")).cpu().numpy()
    ps = unflatten(flat)
    for b in range(B):
        want, _ = ocnn.forward(ps, x[b].astype(np.float64))
        assert rel(y[b] - x[b], want - x[b]) <= 3e-2
        assert abs(float(np.mean(y[b] - want))) <= 3e-2 * float(np.abs(want - x[b]).max())


def test_gradients_match_oracle(fbp, torch):
    from paper_2007_06289_gb300 import corrector
    rng = np.random.default_rng(1)
    B, N = 2, 32
    flat = corrector.init_params(seed=2, scale=2.0)
    flat[-289:] *= 10.0
    flat[:] += rng.normal(0, 0.02, flat.size).astype(np.float32)
    x = smooth_images(rng, B, N).astype(np.float32)
    t = (x + 0.3 * smooth_images(rng, B, N)).astype(np.float32)
    params = torch.tensor(flat, device="cuda", requires_grad=True)
    y = corrector.correct(params, torch.tensor(x, device="cuda"))
    loss = torch.mean((y - torch.tensor(t, device="cuda")) ** 2)
    loss.backward()
    got = params.grad.cpu().numpy().astype(np.float64)
    ps = unflatten(flat)
    want = np.zeros_like(got)
    for b in range(B):
        _, grads, _ = ocnn.loss_and_grads(ps, x[b].astype(np.float64), t[b].astype(np.float64))
        flat_g = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])
        want += flat_g / B                           # batch mean of per-image means
    off = 0
    for k, (w, bb) in enumerate(ps):
        n = w.size + bb.size
        assert rel(got[off:off + w.size], want[off:off + w.size]) <= 3e-2, k
        assert rel(got[off + w.size:off + n], want[off + w.size:off + n]) <= 3e-2, k
        off += n


def test_training_reduces_the_error_to_direct_fbp(fbp, torch):
    from paper_2007_06289_gb300 import corrector
    N, S = 64, 16
    K, M = phantoms.geometry_for(N)
    sino = phantoms.phantom_stack_torch(N, S, 500, "cuda", noise_i0=1e5)
    fast = torch.empty(S, N, N, device="cuda")
    direct = torch.empty(S, N, N, device="cuda")
    fbp.fbp_reconstruct(fbp.fbp_plan(N, K, M, S), sino, fast)
    fbp.fbp_direct_reconstruct(fbp.fbp_plan(N, K, M, S), sino, direct)
    torch.cuda.synchronize()
    train, test = slice(0, 12), slice(12, 16)
    params, losses = corrector.train(fast[train], direct[train], steps=400, batch=4, lr=2e-3)
    before = float(torch.sqrt(torch.mean((fast[test] - direct[test]) ** 2)))
    after = float(torch.sqrt(torch.mean((corrector.infer(params, fast[test].contiguous())
                                         - direct[test]) ** 2)))
    assert np.mean(losses[-20:]) < np.mean(losses[:20])
    assert after < 0.9 * before, (before, after)
