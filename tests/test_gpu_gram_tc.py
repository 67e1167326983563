"""The tensor-core Gram kernel (tcgen05, split-TF32) through the C ABI: G = W^T W for W in the
DOF-major layout the triangular solves write, against an FP64 product of the same FP32
inputs.  The split keeps about 21 bits of each product (error ~2^-21 per term); what is left
is the tensor core's truncating FP32 accumulation over the K steps, spread over four
accumulators (a quarter of K each): about 3e-6 of max|G| at K = 1000-1200 for unit normal W
(1.0e-5 with a single accumulator).  The bound is |G - G_64| <= 1e-5 max|G_64|."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sa():
    from paper_2302_14344_gb300 import subadmm
    subadmm.load()
    return subadmm


def _run(sa, shapes, seed=0, reps=1):
    import torch
    g = torch.Generator().manual_seed(seed)
    Ws, Gs, ref = [], [], []
    for n, cols, ldw in shapes:
        W = torch.randn(n, ldw, generator=g, dtype=torch.float32)
        W[:, cols:] = float("nan")               # columns past `cols` must not be read
        Ws.append(W.cuda())
        Gs.append(torch.full((cols, cols + 3), float("nan"), device="cuda"))
        w64 = W[:, :cols].double()
        ref.append((w64.T @ w64).numpy())
    ms = sa.sim_gram_tc(0, [w.data_ptr() for w in Ws], [s[0] for s in shapes],
                        [s[1] for s in shapes], [s[2] for s in shapes],
                        [x.data_ptr() for x in Gs], [s[1] + 3 for s in shapes], reps=reps)
    torch.cuda.synchronize()
    out = [x[:, : s[1]].cpu().double().numpy() for x, s in zip(Gs, shapes)]
    return out, ref, ms


def _err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("shape", [(1000, 701, 704), (32, 128, 128), (33, 129, 132),
                                   (37, 1, 4), (1200, 257, 260)])
def test_gram_single(sa, shape, capsys):
    (G,), (R,), _ = _run(sa, [shape])
    assert np.all(np.isfinite(G))
    err = _err(G, R)
    with capsys.disabled():
        print(f"\n[tcgen05 Gram, n={shape[0]} cols={shape[1]}] rel err {err:.2e}")
    assert err < 1e-5
    assert np.array_equal(G, G.T)                # mirrored lower triangle


def test_gram_ragged_batch(sa):
    """One launch over jobs of different sizes (the stacked buffer pads rows to 128 and K to
    the longest job with zeros)."""
    shapes = [(1200, 701, 704), (900, 129, 132), (37, 1, 4), (130, 300, 300), (64, 64, 64)]
    Gs, Rs, _ = _run(sa, shapes, seed=3)
    for G, R in zip(Gs, Rs):
        assert np.all(np.isfinite(G))
        assert _err(G, R) < 1e-5


def test_gram_repeated_runs_agree(sa):
    (G1,), (R,), ms = _run(sa, [(1000, 701, 704)], seed=5, reps=3)
    (G2,), _, _ = _run(sa, [(1000, 701, 704)], seed=5, reps=1)
    assert np.array_equal(G1, G2) and ms > 0.0


def test_gram_many_tiles_per_block(sa):
    """More tiles than blocks (the launch has one block per SM): each block runs several tiles
    through its accumulators, nine at most here (64 jobs of the FEM beam's slab shape)."""
    shapes = [(1000, 701, 704)] * 20 + [(1200, 691, 692)] * 44
    Gs, Rs, _ = _run(sa, shapes, seed=11)
    for G, R in zip(Gs, Rs):
        assert np.all(np.isfinite(G))
        assert _err(G, R) < 1e-5
