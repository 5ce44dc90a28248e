"""Pins of the FP64 CNN reference (oracle/cnn.py): the convolution against
its definition, gradients against central finite differences, the Adam step
against its closed form, the residual identity, and that training descends."""
import numpy as np

from oracle import cnn as C


def _tiny(seed=1, K=12, ks=5, ch=3, layers=3):
    rng = np.random.default_rng(seed)
    params = C.init_params(seed, channels=ch, ksize=ks, layers=layers)
    params = [(W * 3.0, rng.standard_normal(b.shape) * 0.1) for W, b in params]  # non-trivial last layer
    x = rng.standard_normal((K, 4))
    t = rng.standard_normal((K, 4))
    return params, x, t


def test_conv_matches_definition():
    rng = np.random.default_rng(0)
    K, ks, ci, co = 9, 5, 3, 2
    h = rng.standard_normal((K, ci))
    W = rng.standard_normal((ks, ci, co))
    b = rng.standard_normal(co)
    a = C.conv1d(h, W, b)
    c = (ks - 1) // 2
    for n in range(K):
        for o in range(co):
            v = b[o]
            for k in range(ks):
                m = n + k - c
                if 0 <= m < K:
                    v += sum(h[m, i] * W[k, i, o] for i in range(ci))
            assert abs(a[n, o] - v) < 1e-12


def test_gradients_match_central_differences():
    params, x, t = _tiny()
    J, grads = C.loss_and_grads(params, x, t)
    eps = 1e-6
    worst = 0.0
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + eps
                Jp = C.loss_and_grads(params, x, t)[0]
                arr[idx] = old - eps
                Jm = C.loss_and_grads(params, x, t)[0]
                arr[idx] = old
                fd = (Jp - Jm) / (2 * eps)
                worst = max(worst, abs(fd - g[idx]) / max(1e-3, abs(fd)))
    assert worst < 1e-6


def test_input_gradient_of_conv():
    rng = np.random.default_rng(5)
    h = rng.standard_normal((10, 3))
    W = rng.standard_normal((5, 3, 2))
    b = rng.standard_normal(2)
    da = rng.standard_normal((10, 2))
    dh, dW, db = C.conv1d_backward(h, W, da)
    eps = 1e-6
    for idx in np.ndindex(h.shape):
        hp, hm = h.copy(), h.copy()
        hp[idx] += eps
        hm[idx] -= eps
        fd = (np.sum(C.conv1d(hp, W, b) * da) - np.sum(C.conv1d(hm, W, b) * da)) / (2 * eps)
        assert abs(fd - dh[idx]) < 1e-7 * max(1.0, abs(fd))
    assert np.allclose(db, da.sum(0))


def test_adam_first_step_closed_form():
    params = [(np.array([[[1.0, -2.0]]]), np.array([0.5, 0.0]))]
    grads = [(np.array([[[0.3, -4.0]]]), np.array([-1e-3, 2.0]))]
    opt = C.Adam(params, lr=0.01)
    new = opt.step(params, grads)
    # m_hat = g, v_hat = g^2 after one step: p - lr g / (|g| + eps)
    for (p, g), q in zip(((params[0][0], grads[0][0]), (params[0][1], grads[0][1])), new[0]):
        assert np.allclose(q, p - 0.01 * g / (np.abs(g) + 1e-8), atol=1e-15)


def test_residual_identity_with_zero_last_layer():
    params, x, _ = _tiny()
    params[-1] = (np.zeros_like(params[-1][0]), np.zeros_like(params[-1][1]))
    y, _ = C.forward(params, x)
    assert np.array_equal(y, x)


def test_training_descends_on_a_learnable_target():
    rng = np.random.default_rng(9)
    K = 256
    x = rng.standard_normal((K, 4))
    # target: a fixed 3-tap mixing of the features plus a cubic term, learnable by the net
    t = x + 0.3 * C.conv1d(x, rng.standard_normal((3, 4, 4)) * 0.3, np.zeros(4)) + 0.05 * x ** 3
    params = C.init_params(2, channels=8, ksize=5, layers=3)
    opt = C.Adam(params, lr=3e-3)
    J0 = C.loss_and_grads(params, x, t)[0]
    for _ in range(300):
        J, g = C.loss_and_grads(params, x, t)
        params = opt.step(params, g)
    assert J < 0.1 * J0
