"""GPU parity of the learned-guess network kernels (BF16 tensor cores, FP32
accumulation) against the FP64 oracle (oracle/cnn.py), with the BF16 storage
rounding of inputs, weights and inter-layer activations/gradients modelled on
the oracle side.  Tolerance 1e-2 relative (BF16 carries 8 significant bits;
FP32 accumulation order differs)."""
import numpy as np
import pytest

from _util import bf16_round, rel
from oracle import cnn as ocnn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03061_gb300 import build
    build.build()


class _Dev:
    """A torch view of a device pointer owned by the library."""

    def __init__(self, ptr, shape, typestr="<f4"):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def _view(ptr, shape):
    return torch.as_tensor(_Dev(ptr, shape), device="cuda")


def _make(depth, cin, cout, seed):
    from paper_1802_03061_gb300 import _binding as B
    net = B.rte_cnn_create(cin, 64, depth, cout, seed)
    rng = np.random.default_rng(seed)
    layers = []
    for l in range(depth):
        d = B.rte_cnn_layer(net, l)
        W = rng.standard_normal((9, d["cin"], d["cout"])) * np.sqrt(2.0 / (9 * d["cin"]))
        b = rng.standard_normal(d["cout"]) * 0.05
        _view(d["w"], W.shape).copy_(torch.from_numpy(W.astype(np.float32)))
        _view(d["b"], b.shape).copy_(torch.from_numpy(b.astype(np.float32)))
        layers.append((bf16_round(W), b.astype(np.float32).astype(np.float64)))
    B.rte_cnn_sync_weights(net)
    torch.cuda.synchronize()
    return net, layers


@pytest.mark.parametrize("cin,cout,H,W", [(16, 16, 5, 150), (32, 32, 3, 64)])
def test_forward_matches_oracle(cin, cout, H, W):
    from paper_1802_03061_gb300 import _binding as B
    net, layers = _make(3, cin, cout, 7)
    Bn = 2
    X = bf16_round(np.random.default_rng(3).standard_normal((Bn, H, W, cin)))
    Xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    y = torch.zeros((Bn, H, W, cout), dtype=torch.float32, device="cuda")
    B.rte_cnn_forward(net, Xd.data_ptr(), Bn, H, W, y.data_ptr())
    torch.cuda.synchronize()
    ref = ocnn.net_forward(X, layers, round_act=bf16_round)[-1]
    assert rel(y.cpu().numpy(), ref) < 1e-2
    B.rte_cnn_destroy(net)


def test_gradients_match_oracle():
    from paper_1802_03061_gb300 import _binding as B
    depth, cin, cout, used = 4, 16, 16, 9
    net, layers = _make(depth, cin, cout, 11)
    Bn, H, W = 2, 6, 140
    rng = np.random.default_rng(4)
    X = bf16_round(rng.standard_normal((Bn, H, W, cin)))
    T = bf16_round(rng.standard_normal((Bn, H, W, cout)))
    Xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    Td = torch.from_numpy(T.astype(np.float32)).to(torch.bfloat16).cuda()
    loss = B.rte_cnn_train_step(net, Xd.data_ptr(), Td.data_ptr(), Bn, H, W, used, 0.0)
    torch.cuda.synchronize()
    ref_loss, grads = ocnn.net_loss_grads(X, T, layers, used, round_act=bf16_round, round_grad=bf16_round)
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    for l in range(depth):
        d = B.rte_cnn_layer(net, l)
        gw = _view(d["gw"], (9, d["cin"], d["cout"])).cpu().numpy()
        gb = _view(d["gb"], (d["cout"],)).cpu().numpy()
        assert rel(gw, grads[l][0]) < 2e-2, l
        assert rel(gb, grads[l][1]) < 2e-2, l
    B.rte_cnn_destroy(net)


def test_training_reduces_loss():
    from paper_1802_03061_gb300 import _binding as B
    net = B.rte_cnn_create(16, 64, 4, 16, 5)
    rng = np.random.default_rng(6)
    Bn, H, W = 4, 16, 128
    X = rng.standard_normal((Bn, H, W, 16)).astype(np.float32)
    # a target that a 3x3 network can represent: a local smoothing of channel 0
    T = np.zeros((Bn, H, W, 16), np.float32)
    T[..., 0] = 0.5 * X[..., 0] + 0.25 * np.roll(X[..., 1], 1, axis=2)
    Xd = torch.from_numpy(X).to(torch.bfloat16).cuda()
    Td = torch.from_numpy(T).to(torch.bfloat16).cuda()
    l0 = B.rte_cnn_train_step(net, Xd.data_ptr(), Td.data_ptr(), Bn, H, W, 1, 0.0)
    for _ in range(200):
        B.rte_cnn_train_step(net, Xd.data_ptr(), Td.data_ptr(), Bn, H, W, 1, 2e-3, want_loss=False)
    l1 = B.rte_cnn_train_step(net, Xd.data_ptr(), Td.data_ptr(), Bn, H, W, 1, 0.0)
    assert l1 < 0.1 * l0
    B.rte_cnn_destroy(net)


def test_weights_file_round_trip(tmp_path):
    """rte_cnn_save / rte_cnn_load: a second network of the same shape loads
    the first one's weights and then computes the same forward output; a file
    of another shape or a truncated file is refused and leaves it unchanged."""
    from paper_1802_03061_gb300 import _binding as B
    net1, _ = _make(4, 16, 16, 3)
    net2, _ = _make(4, 16, 16, 9)
    path = tmp_path / "w.bin"
    B.rte_cnn_save(net1, path)
    X = torch.from_numpy(np.random.default_rng(1).standard_normal((1, 8, 40, 16)).astype(np.float32)).to(
        torch.bfloat16).cuda()

    def fwd(net):
        Y = torch.empty((1, 8, 40, 16), dtype=torch.float32, device="cuda")
        B.rte_cnn_forward(net, X.data_ptr(), 1, 8, 40, Y.data_ptr())
        torch.cuda.synchronize()
        return Y.cpu().numpy()

    y1, y2 = fwd(net1), fwd(net2)
    assert rel(y2, y1) > 1e-2                      # different seeds, different networks
    B.rte_cnn_load(net2, path)
    assert np.array_equal(fwd(net2), y1)
    other, _ = _make(3, 16, 16, 3)                 # another depth
    with pytest.raises(B.RteError):
        B.rte_cnn_load(other, path)
    bad = tmp_path / "short.bin"
    bad.write_bytes(path.read_bytes()[:100])
    with pytest.raises(B.RteError):
        B.rte_cnn_load(net1, bad)
    assert np.array_equal(fwd(net1), y1)
    for n in (net1, net2, other):
        B.rte_cnn_destroy(n)


def test_training_checkpoint_resumes_the_same_trajectory(tmp_path):
    """rte_cnn_save_state / rte_cnn_load_state: a network of another seed that
    loads the checkpoint taken after 3 Adam steps and then takes the same 4
    steps ends with the same weights, bit for bit, as the run that saved it;
    loading the weights alone (fresh moments, step 0) does not.  A weights
    file, a truncated checkpoint and another shape are refused."""
    from paper_1802_03061_gb300 import _binding as B
    rng = np.random.default_rng(11)
    Bn, H, W = 2, 8, 64
    X = torch.from_numpy(rng.standard_normal((Bn, H, W, 16)).astype(np.float32)).to(torch.bfloat16).cuda()
    T = torch.from_numpy(rng.standard_normal((Bn, H, W, 16)).astype(np.float32)).to(torch.bfloat16).cuda()

    def steps(net, k):
        for _ in range(k):
            B.rte_cnn_train_step(net, X.data_ptr(), T.data_ptr(), Bn, H, W, 1, 1e-3, want_loss=False)
        torch.cuda.synchronize()

    def weights(net):
        out = []
        for l in range(3):
            d = B.rte_cnn_layer(net, l)
            out.append(_view(d["w"], (9, d["cin"], d["cout"])).cpu().numpy().copy())
            out.append(_view(d["b"], (d["cout"],)).cpu().numpy().copy())
        return out

    a = B.rte_cnn_create(16, 64, 3, 16, 5)
    steps(a, 3)
    ck, wf = tmp_path / "ck.bin", tmp_path / "w.bin"
    B.rte_cnn_save_state(a, ck)
    B.rte_cnn_save(a, wf)
    steps(a, 4)
    want = weights(a)
    b = B.rte_cnn_create(16, 64, 3, 16, 7)
    B.rte_cnn_load_state(b, ck)
    steps(b, 4)
    assert all(np.array_equal(x, y) for x, y in zip(weights(b), want))
    c = B.rte_cnn_create(16, 64, 3, 16, 7)
    B.rte_cnn_load(c, wf)
    steps(c, 4)
    assert not all(np.array_equal(x, y) for x, y in zip(weights(c), want))
    before = weights(c)
    with pytest.raises(B.RteError):
        B.rte_cnn_load_state(c, wf)                 # a weights file is not a checkpoint
    short = tmp_path / "short.bin"
    short.write_bytes(ck.read_bytes()[:-4])
    with pytest.raises(B.RteError):
        B.rte_cnn_load_state(c, short)
    other = B.rte_cnn_create(16, 64, 4, 16, 7)
    with pytest.raises(B.RteError):
        B.rte_cnn_load_state(other, ck)
    assert all(np.array_equal(x, y) for x, y in zip(weights(c), before))
    for n in (a, b, c, other):
        B.rte_cnn_destroy(n)
