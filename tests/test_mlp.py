"""The surrogate network: CPU float64 oracle pinned to finite differences; GPU forward/backward
kernels against the oracle; BF16 inference; training reduces the loss."""
import numpy as np
import pytest

from oracle import mlp as ref

SHAPE = (17, 32, 3, 2)


def _params(seed, shape=SHAPE):
    n_in, width, hidden, n_out = shape
    rng = np.random.default_rng(seed)
    dims = [n_in] + [width] * hidden + [n_out]
    p = []
    for di, do in zip(dims[:-1], dims[1:]):
        p.append(rng.standard_normal(di * do) * np.sqrt(2.0 / di))
        p.append(0.1 * rng.standard_normal(do))
    return np.concatenate(p)


def test_oracle_gradient_matches_central_differences():
    shape = (5, 7, 3, 2)
    p = _params(1, shape)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((9, 5))
    t = rng.standard_normal((9, 2))
    _, g = ref.loss_and_grad(p, x, t, *shape)
    h = 1e-6
    idx = rng.choice(len(p), 40, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (ref.loss_and_grad(p + e, x, t, *shape)[0] - ref.loss_and_grad(p - e, x, t, *shape)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_oracle_gelu_known_values():
    # GELU(0) = 0, odd part: GELU(z) - GELU(-z) = z, large z -> z
    z = np.array([0.0, 1.0, -1.0, 6.0])
    gz = ref.gelu(z)
    assert gz[0] == 0.0 and abs(gz[1] - gz[2] - 1.0) < 1e-15 and abs(gz[3] - 6.0) < 1e-9
    assert abs(ref.gelu(np.array([1.0]))[0] - 0.8411919906082768) < 1e-12


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no GPU")
    return t


@pytest.mark.gpu
def test_gpu_loss_and_gradients_match_oracle(torch):
    from paper_1702_05167_gb300 import hsc
    p = _params(3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((200, 17))
    t = rng.standard_normal((200, 2))
    net = hsc.MLP(*SHAPE, max_batch=256)
    net.set_params(p.astype(np.float32))
    p32 = net.get_params().astype(np.float64)
    loss, g = net.loss_grad(torch.from_numpy(x.astype(np.float32)).cuda(),
                            torch.from_numpy(t.astype(np.float32)).cuda(), want_grad=True)
    lref, gref = ref.loss_and_grad(p32, x.astype(np.float32).astype(np.float64),
                                   t.astype(np.float32).astype(np.float64), *SHAPE)
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    assert np.abs(g - gref).max() <= 1e-4 * np.abs(gref).max()
    y = torch.empty((200, 2), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(x.astype(np.float32)).cuda(), y)
    yref = ref.forward(p32, x.astype(np.float32).astype(np.float64), *SHAPE)
    assert np.abs(y.cpu().numpy() - yref).max() <= 1e-5 * np.abs(yref).max()
    yb = torch.empty_like(y)
    net.forward(torch.from_numpy(x.astype(np.float32)).cuda(), yb, bf16=True)
    assert np.abs(yb.cpu().numpy() - yref).max() <= 3e-2 * np.abs(yref).max()
    net.close()


@pytest.mark.gpu
def test_gpu_training_reduces_loss(torch):
    from paper_1702_05167_gb300 import hsc
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (1024, 17))
    t = np.column_stack([np.sin(3 * x[:, 0]) + 0.3 * x[:, 1], np.cos(2 * x[:, 0]) * x[:, 2]])
    net = hsc.MLP(17, 64, 3, 2, max_batch=1024)
    net.set_params(_params(6, (17, 64, 3, 2)).astype(np.float32))
    tx = torch.from_numpy(x.astype(np.float32)).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    first = net.loss_grad(tx, tt)
    for _ in range(400):
        net.loss_grad(tx, tt)
        net.adam(3e-3)
    last = net.loss_grad(tx, tt)
    net.close()
    assert last < 0.05 * first, (first, last)
