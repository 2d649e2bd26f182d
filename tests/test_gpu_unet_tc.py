"""GPU tests of the tcgen05 / TMEM convolution path of the learned-guess network: the forward
pass and every parameter gradient agree with the mma.sync path (itself checked against the
FP64 CPU oracle in test_gpu_unet.py) up to the rounding of BF16 outputs; the TMA-fed forward
path (2) reads the same operands in the same reduction order as the gather path (1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def un():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0811_4446_gb300 import build, unet
    build.build()
    return unet


def _inputs(un, B, n, seed):
    rng = np.random.default_rng(seed)
    p = un.init_params(seed)
    p += (0.01 * rng.standard_normal(p.size)).astype(np.float32)
    x = np.zeros((B, n + 1, n + 1, 8), np.float32)
    x[..., :5] = rng.standard_normal((B, n + 1, n + 1, 5)).astype(np.float32)
    t = (0.5 * rng.standard_normal((B, n + 1, n + 1, 3))).astype(np.float32)
    return p, x, t


@pytest.mark.parametrize("B,n", [(2, 32), (3, 64)])
def test_tc_forward_matches_mma_sync(un, B, n):
    p, x, _ = _inputs(un, B, n, 11)
    ys = []
    for path in (0, 1):
        net = un.UNet(B, n)
        net.set_tensor_path(path)
        net.set_params(p)
        ys.append(net.forward(x))
        net.close()
    rel = np.linalg.norm(ys[1] - ys[0]) / np.linalg.norm(ys[0])
    assert rel <= 1e-2, rel


def test_tc_gradients_match_mma_sync(un):
    p, x, t = _inputs(un, 2, 32, 12)
    out = []
    for path in (0, 1):
        net = un.UNet(2, 32)
        net.set_tensor_path(path)
        net.set_params(p)
        out.append(net.loss_grad(x, t))
        net.close()
    (l0, g0), (l1, g1) = out
    assert abs(l1 - l0) <= 1e-2 * abs(l0)
    rel = np.linalg.norm(g1 - g0) / np.linalg.norm(g0)
    assert rel <= 3e-2, rel


@pytest.mark.parametrize("Bmax,B,n", [(2, 2, 32), (3, 2, 64), (1, 1, 128)])
def test_tma_forward_matches_gather(un, Bmax, B, n):
    # Bmax > B: the tensor maps span the allocated batch, the launch only the images given;
    # 33, 65 and 129 node rows leave ragged 16 x 8 tiles on the right and bottom edges.
    p, x, _ = _inputs(un, B, n, 13)
    ys = []
    for path in (1, 2):
        net = un.UNet(Bmax, n)
        net.set_tensor_path(path)
        net.set_params(p)
        ys.append(net.forward(x))
        net.close()
    rel = np.linalg.norm(ys[1] - ys[0]) / np.linalg.norm(ys[0])
    assert rel <= 1e-5, rel


def test_tma_gradients_match_gather(un):
    p, x, t = _inputs(un, 2, 32, 14)
    out = []
    for path in (1, 2):
        net = un.UNet(2, 32)
        net.set_tensor_path(path)
        net.set_params(p)
        out.append(net.loss_grad(x, t))
        net.close()
    (l1, g1), (l2, g2) = out
    assert abs(l2 - l1) <= 1e-5 * abs(l1)
    rel = np.linalg.norm(g2 - g1) / np.linalg.norm(g1)
    assert rel <= 1e-4, rel


@pytest.mark.parametrize("Bmax,B,n", [(2, 2, 32), (3, 2, 64), (1, 1, 128)])
def test_halo_forward_matches_tile_path(un, Bmax, B, n):
    # path 3 sums each output chunk by chunk, each chunk tap by tap (path 2: tap by tap over all
    # channels), so FP32 rounding differs, some BF16 activations round to the neighbouring value
    # and the differences carry through the twelve layers: the bound of the mma.sync comparison
    p, x, _ = _inputs(un, B, n, 15)
    ys = []
    for path in (2, 3):
        net = un.UNet(Bmax, n)
        net.set_tensor_path(path)
        net.set_params(p)
        ys.append(net.forward(x))
        net.close()
    rel = np.linalg.norm(ys[1] - ys[0]) / np.linalg.norm(ys[0])
    assert rel <= 1e-2, rel


@pytest.mark.parametrize("Bmax,B,n", [(2, 2, 8), (1, 1, 16), (2, 2, 32), (4, 3, 64), (1, 1, 128)])
def test_layer_gradients_match_mma_sync(un, Bmax, B, n):
    # Path 3 takes the weight gradient of every 3x3 layer from the TMA-fed tcgen05 kernel
    # (MN-major operands, segments of 64 or 128 pixels: 9 to 129 node rows leave ragged
    # segments, the smallest grids tiles larger than the image; B < Bmax leaves images of the
    # tensor maps unread), the data gradient as a forward convolution of (spread) dY on the halo
    # or tile kernels, each first contribution to an activation gradient overwriting it, and the
    # head's backward on the CUDA cores.
    # Path 0 runs mma.sync everywhere.  The two forwards round BF16 activations differently, so
    # per layer the largest difference is compared with the layer's largest gradient entry.
    from oracle import unet as ou
    p, x, t = _inputs(un, B, n, 16)
    out = []
    for path in (0, 3):
        net = un.UNet(Bmax, n)
        net.set_tensor_path(path)
        net.set_params(p)
        out.append(net.loss_grad(x, t))
        net.close()
    (l0, g0), (l3, g3) = out
    assert abs(l3 - l0) <= 1e-2 * abs(l0)
    off = 0
    for name, k, _, ci, co, _ in ou.LAYERS:
        for size in (k * k * ci * co, co):
            a, b = g3[off:off + size], g0[off:off + size]
            rel = np.abs(a - b).max() / np.abs(b).max()
            assert rel <= 3e-2, (name, size, rel)
            off += size
    assert off == g0.size


def test_graphs_match_launch_by_launch(un):
    """The per-batch-size CUDA graphs (the default) replay the launches of the kernel-by-kernel
    mode: the same forward outputs bit for bit, also when batch sizes alternate on one network
    (one graph each), and the same loss and gradients up to the order of the weight gradient's
    FP32 atomic adds."""
    p, x, t = _inputs(un, 3, 32, 17)
    res = []
    for graphs in (True, False):
        net = un.UNet(3, 32)
        net.set_params(p)
        net.set_graphs(graphs)
        y2 = net.forward(x[:2])
        y3 = net.forward(x)
        y2b = net.forward(x[:2])
        loss, g = net.loss_grad(x[:2], t[:2])
        res.append((y2, y3, y2b, loss, g))
        net.close()
    (a2, a3, a2b, la, ga), (b2, b3, b2b, lb, gb) = res
    assert np.array_equal(a2, b2) and np.array_equal(a3, b3) and np.array_equal(a2b, a2)
    assert np.array_equal(b2b, b2)
    assert abs(la - lb) <= 1e-6 * abs(lb)
    assert np.linalg.norm(ga - gb) <= 1e-5 * np.linalg.norm(gb)
