"""Controller network kernels (FP32, GPU) against the FP64 oracle network."""
import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_21200_gb300 import Mlp  # noqa: E402

KEYS = ["W1", "b1", "W2", "b2", "W3", "b3"]


def flat(p):
    return np.concatenate([p[k].reshape(-1) for k in KEYS]).astype(np.float32)


def unflat(v, n_in, n_out, h=128):
    shapes = {"W1": (h, n_in), "b1": (h,), "W2": (h, h), "b2": (h,), "W3": (n_out, h), "b3": (n_out,)}
    out, o = {}, 0
    for k in KEYS:
        n = int(np.prod(shapes[k]))
        out[k] = v[o:o + n].reshape(shapes[k]).astype(np.float64)
        o += n
    return out


def test_forward_and_gradients_match_oracle():
    rng = np.random.default_rng(0)
    p = mlp.init_params(40, 2, rng)
    p = unflat(flat(p), 40, 2)          # exactly the FP32-rounded weights
    net = Mlp(40, 2, flat(p))
    X = rng.standard_normal((64, 40)).astype(np.float32)
    T = rng.standard_normal((64, 2)).astype(np.float32)
    w = np.array([1.0, 0.25])
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    Y = net.forward(Xd).cpu().numpy()
    Yref, _ = mlp.forward(p, X.astype(np.float64))
    assert np.abs(Y - Yref).max() <= 1e-5 * max(1.0, np.abs(Yref).max())
    loss, G = net.grads(Xd, Td, w, want_grad=True)
    gref = mlp.grads(p, X.astype(np.float64), T.astype(np.float64), w)
    assert abs(loss - mlp.loss(p, X.astype(np.float64), T.astype(np.float64), w)) <= 1e-5 * abs(loss)
    G = G.cpu().numpy()
    gr = flat({k: gref[k] for k in KEYS}).astype(np.float64)
    assert np.abs(G - gr).max() <= 1e-4 * np.abs(gr).max()


def test_adam_matches_oracle():
    rng = np.random.default_rng(1)
    p = unflat(flat(mlp.init_params(10, 1, rng)), 10, 1)
    net = Mlp(10, 1, flat(p))
    X = rng.standard_normal((32, 10)).astype(np.float32)
    T = rng.standard_normal((32, 1)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    state = {}
    q = {k: v.copy() for k, v in p.items()}
    for _ in range(5):
        net.grads(Xd, Td)
        net.adam(lr=1e-2)
        mlp.adam_step(q, mlp.grads(q, X.astype(np.float64), T.astype(np.float64)), state, lr=1e-2)
    got = net.get_params().astype(np.float64)
    ref = flat(q).astype(np.float64)
    assert np.abs(got - ref).max() <= 2e-4 * max(1.0, np.abs(ref).max())


def test_network_trains_on_the_gpu():
    rng = np.random.default_rng(2)
    net = Mlp(4, 1, flat(mlp.init_params(4, 1, rng)))
    X = rng.uniform(-1, 1, size=(1024, 4)).astype(np.float32)
    T = (np.sin(2 * X[:, :1]) + X[:, 1:2] ** 2 - 0.5 * X[:, 2:3] * X[:, 3:4]).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    l0, _ = net.grads(Xd, Td)
    for _ in range(1500):
        net.grads(Xd, Td)
        net.adam(lr=3e-3)
    l1, _ = net.grads(Xd, Td)
    assert l1 < l0 / 50, (l0, l1)
