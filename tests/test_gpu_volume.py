"""Ragged volumes (slices of mixed sizes in one call) against the float64 oracle and the
one-slice path.

Every image of a volume must match the float64 oracle (sampled pixels of every size group,
N = 256 .. 2048, within 1e-5 of the image range, before and after autotuning) and equal,
bit for bit, the image fbp_reconstruct gives for that slice alone with the same filter:
grouping, pointer tables, per-group streams, graph capture and replay, and the autotuner's
choices change the execution, never the sums.
"""
import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


# (N, K, M): the standard geometry for four sizes, plus a second shape at N = 128
SHAPES = [(64,) + phantoms.geometry_for(64), (128,) + phantoms.geometry_for(128),
          (256,) + phantoms.geometry_for(256), (512,) + phantoms.geometry_for(512),
          (128, 100, 190)]
ORDER = [1, 0, 4, 2, 1, 3, 0, 2, 1, 4, 3, 1]       # item -> shape, shuffled, ragged counts


def make_items(torch, seed=7):
    items = []
    for i, si in enumerate(ORDER):
        N, K, M = SHAPES[si]
        sino = phantoms.phantom_stack_torch(N, 1, seed + i, "cuda", K=K, M=M,
                                            noise_i0=1e5)[0].contiguous()
        img = torch.full((N, N), float("nan"), device="cuda")
        items.append((N, sino, img))
    return items


def one_slice(fbp, torch, N, sino):
    K, M = sino.shape
    plan = fbp.fbp_plan(N, K, M, 1)
    img = torch.empty(plan.img_shape, device="cuda")
    fbp.fbp_reconstruct(plan, sino[None].contiguous(), img)
    torch.cuda.synchronize()
    return img[0]


def test_volume_matches_one_slice_path(fbp, torch):
    items = make_items(torch)
    vol = fbp.fbp_volume_create(items)
    assert vol.info()["groups"] == len(SHAPES)
    counts = {}
    for g in range(len(SHAPES)):
        info = vol.group(g)
        counts[(info["N"], info["K"], info["M"])] = info["items"]
    for si, shp in enumerate(SHAPES):
        assert counts[shp] == ORDER.count(si)
    vol.run()
    torch.cuda.synchronize()
    for N, sino, img in items:
        assert torch.equal(img, one_slice(fbp, torch, N, sino))


def test_volume_graph_replay_follows_the_inputs(fbp, torch):
    items = make_items(torch, seed=30)
    s = torch.cuda.Stream()
    vol = fbp.fbp_volume_create(items, graph=True)
    with pytest.raises(fbp.FbpError):
        vol.run(torch.cuda.default_stream())       # capture needs a created stream
    vol.run(s)                                     # captures, then launches
    s.synchronize()
    first = [img.clone() for _, _, img in items]
    for (N, sino, img), ref in zip(items, first):
        assert torch.equal(ref, one_slice(fbp, torch, N, sino))
    # new data in the same buffers: the replayed graph reads them
    for i, (N, sino, img) in enumerate(items):
        K, M = sino.shape
        sino.copy_(phantoms.phantom_stack_torch(N, 1, 100 + i, "cuda", K=K, M=M)[0])
        img.fill_(float("nan"))
    vol.run(s)
    s.synchronize()
    for N, sino, img in items:
        assert torch.equal(img, one_slice(fbp, torch, N, sino))


def test_volume_autotuner_keeps_the_bits(fbp, torch):
    items = make_items(torch, seed=50)
    vol = fbp.fbp_volume_create(items)
    vol.run()
    torch.cuda.synchronize()
    before = [img.clone() for _, _, img in items]
    choices = vol.tune()
    assert len(choices) == len(SHAPES)
    for g, (k, c) in enumerate(choices):
        info = vol.group(g)
        n = int(np.log2(info["N"]))
        assert info["fuse_k"] == k and info["chunk"] == c
        assert 1 <= c <= info["items"]
        assert (k == n) if n <= 6 else (2 <= k <= 6 and n - k <= 6)
    for _, _, img in items:
        img.fill_(float("nan"))
    vol.run()
    torch.cuda.synchronize()
    for (_, _, img), ref in zip(items, before):
        assert torch.equal(img, ref)


def test_volume_rejects_bad_items(fbp, torch):
    N, K, M = SHAPES[0]
    sino = torch.zeros(K, M, device="cuda")
    img = torch.zeros(N, N, device="cuda")
    with pytest.raises(fbp.FbpError):
        fbp.fbp_volume_create([])
    spare = torch.zeros(K * M + 4, device="cuda")
    with pytest.raises(fbp.FbpError):              # 4 bytes off a 16-byte boundary
        fbp.fbp_volume_create([(N, spare[1:1 + K * M].view(K, M), img)])
    with pytest.raises(ValueError):
        fbp.fbp_volume_create([(N, sino, img[:-1])])


def test_volume_matches_oracle_at_every_size(fbp, torch):
    # the ragged benchmark's sizes (N = 256 .. 2048, standard geometry), shuffled, with
    # repeated sizes; graph capture and replay, then the autotuner's choices
    from paper_2007_06289_gb300 import iir_fit
    sizes = [2048, 256, 1024, 512, 2048, 256, 1024]
    items = []
    for i, N in enumerate(sizes):
        K, M = phantoms.geometry_for(N)
        sino = phantoms.phantom_stack_torch(N, 1, 900 + i, "cuda", K=K, M=M,
                                            noise_i0=1e5)[0].contiguous()
        items.append((N, sino, torch.full((N, N), float("nan"), device="cuda")))
    for N in set(sizes):                           # the volume's filters are the table's
        b, a = fbp.fbp_default_coeffs(N, 3)
        wb, wa = iir_fit.coefficients(N, 3)
        assert np.array_equal(b, wb) and np.array_equal(a, wa)
    rng = np.random.default_rng(17)
    want = []
    for N, sino, _ in items:
        ys, xs = rng.integers(0, N, 32), rng.integers(0, N, 32)
        ys[:4] = [0, N - 1, 0, N - 1]
        xs[:4] = [0, 0, N - 1, N - 1]
        s64 = sino.cpu().numpy().astype(np.float64)
        want.append((ys, xs, oracle.fast_fbp_pixels(s64, N, *iir_fit.coefficients(N, 3), ys, xs)))

    def check(tag):
        for (N, _, img), (ys, xs, w) in zip(items, want):
            got = img.cpu().numpy()
            assert np.isfinite(got).all(), (tag, N)
            err = np.abs(got[ys, xs] - w).max() / (got.max() - got.min())
            assert err <= 1e-5, (tag, N, err)

    st = torch.cuda.Stream()
    vol = fbp.fbp_volume_create(items, order=3, graph=True)
    vol.run(st)
    st.synchronize()
    check("graph")
    choices = vol.tune(st)
    for _, _, img in items:
        img.fill_(float("nan"))
    vol.run(st)
    st.synchronize()
    check(f"tuned {choices}")
