"""Surrogate MLP kernels against the FP64 reference oracle/mlp_oracle.py:
forward pass, full-batch gradient, Adam updates over shuffled minibatches,
ensemble mean/spread and a training run that must lower the loss."""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu

MASK64 = (1 << 64) - 1


def splitmix64(state):
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): returns (value, state)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31), state


def shuffled(n, state):
    perm = list(range(n))
    for i in range(n - 1, 0, -1):
        r, state = splitmix64(state)
        j = r % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm, state


@pytest.fixture(scope="module")
def lbm():
    from paper_2512_12934_gb300 import lbm as L
    L.load()
    return L


def members_params(E, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(E):
        p = M.init_params(rng)
        for k in ("b1", "b2", "b3", "b4"):  # non-zero biases so their paths are exercised
            p[k] = rng.uniform(-0.1, 0.1, size=p[k].shape)
        out.append(p)
    return out


def f32_params(ps):
    """The float32 values the GPU receives, back in float64 dicts for the oracle."""
    flat = np.stack([M.flatten(p) for p in ps]).astype(np.float32)
    return flat, [M.unflatten(f.astype(np.float64)) for f in flat]


def data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 4)).astype(np.float32)
    x = X.astype(np.float64)
    T = np.stack([np.tanh(x[:, 0] - 0.5 * x[:, 1]) + 0.1 * x[:, 2] * x[:, 3],
                  np.sin(x[:, 1]) * np.cos(0.5 * x[:, 0]) + 0.2 * x[:, 3]], axis=1).astype(np.float32)
    return X, T


@pytest.mark.parametrize("path", ["simt", "tensor"])
@pytest.mark.parametrize("n", [1, 31, 100, 257])
def test_forward_matches_oracle(lbm, n, path):
    E = 3
    flat, ps = f32_params(members_params(E, 11 + n))
    X, _ = data(n, 5 + n)
    net = lbm.MLP(E)
    try:
        net.set_infer_path(path)
        net.set_params(flat)
        assert np.array_equal(net.params(), flat)
        Y = net.forward(X)
    finally:
        net.close()
    for e in range(E):
        ref, _ = M.forward(ps[e], X.astype(np.float64))
        err = np.abs(Y[e] - ref).max() / np.abs(ref).max()
        assert err < 2e-5, (e, err)


@pytest.mark.parametrize("n", [32, 100])
def test_gradient_matches_oracle(lbm, n):
    E = 2
    flat, ps = f32_params(members_params(E, 21 + n))
    X, T = data(n, 7 + n)
    net = lbm.MLP(E)
    try:
        net.set_params(flat)
        g = net.gradient(X, T)
        assert np.array_equal(net.params(), flat)  # a gradient call changes nothing
    finally:
        net.close()
    for e in range(E):
        ref = M.backward(ps[e], X.astype(np.float64), T.astype(np.float64))
        got = M.unflatten(g[e].astype(np.float64))
        for name, _ in M.shapes():
            scale = np.abs(ref[name]).max()
            assert scale > 0, name
            err = np.abs(got[name] - ref[name]).max() / scale
            assert err < 1e-4, (e, name, err)


def test_adam_minibatch_steps_match_oracle(lbm):
    """One epoch over n = 96 rows in minibatches of 40 (a ragged tail of 16
    dropped): two Adam steps on the rows a SplitMix64 Fisher-Yates shuffle
    picks.  Updates whose gradients are far above FP32 noise must agree to
    1e-3 of the learning rate; every update stays within the Adam bound."""
    E, n, batch, lr, seed = 2, 96, 40, 1e-3, 987654321
    flat, ps = f32_params(members_params(E, 31))
    X, T = data(n, 13)
    net = lbm.MLP(E)
    try:
        net.set_params(flat)
        net.train(X, T, epochs=1, batch=batch, lr=lr, shuffle_seed=seed)
        got = net.params().astype(np.float64)
    finally:
        net.close()
    perm, _ = shuffled(n, seed)
    for e in range(E):
        p = flat[e].astype(np.float64)
        m = np.zeros_like(p)
        v = np.zeros_like(p)
        small = np.zeros(p.size, dtype=bool)
        for t, b0 in enumerate(range(0, n - batch + 1, batch), start=1):
            rows = perm[b0:b0 + batch]
            g = M.flatten(M.backward(M.unflatten(p), X[rows].astype(np.float64), T[rows].astype(np.float64)))
            off = 0
            for name, shp in M.shapes():
                k = int(np.prod(shp))
                seg = np.abs(g[off:off + k])
                small[off:off + k] |= seg < 1e-3 * seg.max()
                off += k
            p, m, v = M.adam_step(p, g, m, v, t, lr=lr)
        d = np.abs(got[e] - p)
        assert (~small).mean() > 0.9
        assert d[~small].max() < 1e-3 * lr + 1e-7, d[~small].max()
        assert np.abs(got[e] - flat[e]).max() <= 2 * lr * 1.01


@pytest.mark.parametrize("path", ["simt", "tensor"])
def test_predict_mean_and_spread(lbm, path):
    E, n = 5, 300
    flat, ps = f32_params(members_params(E, 41))
    X, _ = data(n, 17)
    net = lbm.MLP(E)
    try:
        net.set_infer_path(path)
        net.set_params(flat)
        mean, spread = net.predict(X)
    finally:
        net.close()
    Ys = np.stack([M.forward(p, X.astype(np.float64))[0] for p in ps])
    mu = Ys.mean(axis=0)
    sd = Ys.std(axis=0)
    ref_spread = (sd / np.abs(mu)).max(axis=1)
    assert np.abs(mean - mu).max() < 2e-5 * np.abs(mu).max()
    ok = np.abs(mu).min(axis=1) > 1e-2  # spread is ill-conditioned where a mean is ~0
    assert ok.mean() > 0.8
    assert np.allclose(spread[ok], ref_spread[ok], rtol=1e-3, atol=1e-5)


def test_predict_device_pointers(lbm):
    import torch
    E, n = 5, 1000
    flat, _ = f32_params(members_params(E, 51))
    X, _ = data(n, 19)
    net = lbm.MLP(E)
    try:
        net.set_params(flat)
        mean_h, spread_h = net.predict(X)
        Xd = torch.from_numpy(X).cuda()
        md = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        sd = torch.empty(n, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        net.predict_device(Xd.data_ptr(), n, md.data_ptr(), sd.data_ptr())
        assert np.array_equal(md.cpu().numpy(), mean_h)
        assert np.array_equal(sd.cpu().numpy(), spread_h)
    finally:
        net.close()


def test_training_lowers_the_loss(lbm):
    E, n = 5, 2048
    X, T = data(n, 23)
    net = lbm.MLP(E, seed=7)
    try:
        p0 = net.params().astype(np.float64)
        assert not np.array_equal(p0[0], p0[1])  # members start apart
        net.train(X, T, epochs=40, batch=128, lr=2e-3, shuffle_seed=3)
        p1 = net.params().astype(np.float64)
    finally:
        net.close()
    for e in range(E):
        l0 = M.loss(M.unflatten(p0[e]), X.astype(np.float64), T.astype(np.float64))
        l1 = M.loss(M.unflatten(p1[e]), X.astype(np.float64), T.astype(np.float64))
        assert l1 < 0.05 * l0, (e, l0, l1)


def test_tensor_path_agrees_with_simt_path_on_a_large_batch(lbm):
    """65,536 points x 5 members (the size the surrogate is timed on): the
    tcgen05 split-product path and the FP32 path agree to FP32 level, and
    sampled rows match the FP64 oracle."""
    E, n = 5, 65536
    flat, ps = f32_params(members_params(E, 61))
    X, _ = data(n, 29)
    net = lbm.MLP(E)
    try:
        net.set_params(flat)
        net.set_infer_path("simt")
        Ys = net.forward(X)
        net.set_infer_path("tensor")
        Yt = net.forward(X)
    finally:
        net.close()
    scale = np.abs(Ys).max()
    assert np.abs(Yt - Ys).max() <= 2e-5 * scale
    rows = np.random.default_rng(3).choice(n, 64, replace=False)
    for e in range(E):
        ref, _ = M.forward(ps[e], X[rows].astype(np.float64))
        assert np.abs(Yt[e][rows] - ref).max() <= 2e-5 * np.abs(ref).max()


def test_tensor_path_wait_that_runs_out_is_reported(lbm):
    """A one-cycle limit makes the tensor-core kernel's first wait (on its
    weight copy) run out: the call fails with LBM_ERR_TIMEOUT, and with the
    default limit back the ensemble predicts correctly again."""
    E, n = 2, 500
    flat, ps = f32_params(members_params(E, 71))
    X, _ = data(n, 31)
    net = lbm.MLP(E)
    try:
        net.set_params(flat)
        net.set_infer_path("tensor")
        net.set_wait_limit(1)
        with pytest.raises(lbm.LbmError, match="TIMEOUT"):
            net.forward(X)
        net.set_wait_limit(0)
        Y = net.forward(X)
    finally:
        net.close()
    for e in range(E):
        ref, _ = M.forward(ps[e], X.astype(np.float64))
        assert np.abs(Y[e] - ref).max() <= 2e-5 * np.abs(ref).max()
