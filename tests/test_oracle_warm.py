"""Pins for the warm-start oracle (oracle/warm.py): the backpropagated gradient against
central finite differences, GELU's derivative, and the semivariogram of a linear field
against its direct definition."""
import numpy as np

from oracle import warm


def _blob(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    b = np.empty(warm.BLOB)
    b[:warm.NFEAT] = rng.normal(size=warm.NFEAT)
    b[warm.NFEAT:2 * warm.NFEAT] = rng.uniform(0.5, 2.0, warm.NFEAT)
    b[2 * warm.NFEAT:2 * warm.NFEAT + 3] = rng.normal(size=3)
    b[2 * warm.NFEAT + 3:2 * warm.NFEAT + 6] = rng.uniform(0.5, 2.0, 3)
    b[2 * warm.NFEAT + 6:] = rng.normal(scale=scale, size=warm.NPARAM) / 6
    return b


def _batch(seed=1, B=7):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, warm.NFEAT))
    T = np.column_stack([rng.normal(size=(B, 3)), rng.choice([0.5, 1.5, 2.5], B)])
    return X, T


def test_gradient_matches_central_differences():
    b = _blob()
    X, T = _batch()
    loss, g = warm.mlp_loss_grad(b, X, T)
    rng = np.random.default_rng(5)
    off = 2 * warm.NFEAT + 6
    # sample coordinates in every layer's weights and biases
    idx = np.concatenate([rng.choice(warm.NPARAM, 40, replace=False),
                          [0, 5120, 5120 + 127, warm.NPARAM - 1, warm.NPARAM - 7]])
    h = 1e-6
    for i in idx:
        bp, bm = b.copy(), b.copy()
        bp[off + i] += h
        bm[off + i] -= h
        fd = (warm.mlp_loss_grad(bp, X, T)[0] - warm.mlp_loss_grad(bm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_gelu_derivative():
    x = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (warm._gelu(x + h) - warm._gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(warm._gelu_d(x), fd, atol=1e-8)


def test_loss_zero_at_perfect_fit():
    b = _blob(scale=0.0)                     # zero weights: outputs are the biases (0)
    X, T = _batch()
    ym, ys = b[2 * warm.NFEAT:2 * warm.NFEAT + 3], b[2 * warm.NFEAT + 3:2 * warm.NFEAT + 6]
    T[:, :3] = ym                            # standardised targets 0 -> zero regression loss
    loss, _ = warm.mlp_loss_grad(b, X, T)
    assert abs(loss - np.log(3.0)) < 1e-12   # uniform logits: cross-entropy log 3


def test_variogram_of_a_linear_field():
    # d = 1, y = c x:  (y_i - y_j)^2 / 2 = c^2 h^2 / 2, so gamma_k is that mean per bin
    rng = np.random.default_rng(2)
    n = 300
    x = np.sort(rng.random(n))[:, None]
    c = 1.7
    y = c * x[:, 0]
    f = warm.features(x, y, np.array([0, 100, 300]), np.array([0, 0, 50]), max_points=10000)
    var = np.mean((y - y.mean()) ** 2)
    sums, cnts = np.zeros(32), np.zeros(32)
    for i in range(n):
        for j in range(i + 1, n):
            h = abs(x[i, 0] - x[j, 0])
            if 0 < h <= 0.5:
                k = min(int(np.floor(h * 64)), 31)
                sums[k] += 0.5 * (c * h) ** 2
                cnts[k] += 1
    want = np.where(cnts > 0, sums / np.maximum(cnts, 1) / var, 0.0)
    np.testing.assert_allclose(f[:32], want, rtol=1e-12)
    # two blocks of 100 and 200 points: both in the last size class
    np.testing.assert_array_equal(f[33:38], [0, 0, 0, 0, 1])
    # the size classes on a hand-made partition: sizes 1, 4, 5, 8, 9, 12, 13, 16, 17, 40
    sizes = np.array([1, 4, 5, 8, 9, 12, 13, 16, 17, 40])
    bp = np.concatenate([[0], np.cumsum(sizes)])
    xx = rng.random((int(bp[-1]), 1))
    g = warm.features(xx, xx[:, 0], bp, np.zeros(len(bp), np.int64), max_points=10000)
    np.testing.assert_array_equal(g[33:38], [0.2, 0.2, 0.2, 0.2, 0.2])
    # nearest neighbour on a sorted line: the closer of the two adjacent points
    xs = x[:, 0]
    g_nn = d_nn = 0.0
    for i in range(n):
        cand = [j for j in (i - 1, i + 1) if 0 <= j < n]
        j = min(cand, key=lambda jj: ((xs[i] - xs[jj]) ** 2, jj))
        g_nn += 0.5 * (c * (xs[i] - xs[j])) ** 2
        d_nn += abs(xs[i] - xs[j])
    assert abs(f[38] - g_nn / n / var) <= 1e-12 * f[38]
    assert abs(f[39] - 64 * d_nn / n) <= 1e-12 * f[39]


def test_adam_first_step_and_constant_gradient():
    # the bias corrections make the first step (and every step under a constant gradient)
    # move each parameter by lr g / (|g| + eps): a sign step of length lr up to eps
    rng = np.random.default_rng(9)
    th0 = rng.normal(size=50)
    g = rng.normal(size=50) * np.logspace(-6, 2, 50)
    lr, eps = 1e-3, 1e-8
    th, m, v = th0, np.zeros(50), np.zeros(50)
    for t in range(1, 11):
        th, m, v = warm.adam_step(th, g, m, v, t, lr, eps=eps)
        np.testing.assert_allclose(th, th0 - t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)


def test_adam_two_steps_closed_form():
    # two gradients g1, g2: the bias-corrected moments are (b1 g1 + g2) / (1 + b1) and
    # (b2 g1^2 + g2^2) / (1 + b2)
    rng = np.random.default_rng(10)
    th0, g1, g2 = rng.normal(size=(3, 40))
    lr, b1, b2, eps = 2e-3, 0.9, 0.999, 1e-8
    th1, m, v = warm.adam_step(th0, g1, np.zeros(40), np.zeros(40), 1, lr)
    th2, _, _ = warm.adam_step(th1, g2, m, v, 2, lr)
    mhat = (b1 * g1 + g2) / (1 + b1)
    vhat = (b2 * g1 ** 2 + g2 ** 2) / (1 + b2)
    np.testing.assert_allclose(th2, th1 - lr * mhat / (np.sqrt(vhat) + eps), rtol=1e-12, atol=1e-15)


def test_adam_is_invariant_to_gradient_scale():
    # with eps = 0 the trajectory does not change when every gradient is scaled by c > 0
    rng = np.random.default_rng(11)
    th0 = rng.normal(size=30)
    gs = rng.normal(size=(6, 30))
    a = b = th0
    ma = va = mb = vb = np.zeros(30)
    for t, g in enumerate(gs, start=1):
        a, ma, va = warm.adam_step(a, g, ma, va, t, 1e-2, eps=0.0)
        b, mb, vb = warm.adam_step(b, 37.5 * g, mb, vb, t, 1e-2, eps=0.0)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)
