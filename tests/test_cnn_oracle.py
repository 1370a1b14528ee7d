"""CPU pins of the surrogate network oracle (oracle/cnn_oracle.py).

The convolution is checked against scipy's N-d correlation, every gradient
against central finite differences of the oracle's own forward pass, Adam
against its closed-form first step, and the gate on constructed cases.
"""

import numpy as np
import pytest

from oracle import cnn_oracle as N

RNG = np.random.default_rng(2208)


def test_conv3d_matches_scipy_correlate():
    scipy_signal = pytest.importorskip("scipy.signal")
    for stride in (1, 2):
        x = RNG.standard_normal((2, 7, 6, 5))
        w = RNG.standard_normal((27, 2, 3))
        b = RNG.standard_normal(3)
        y = N.conv3d(x, w, b, stride)
        xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
        for o in range(3):
            ref = b[o] + sum(scipy_signal.correlate(xp[c], w[:, c, o].reshape(3, 3, 3), mode="valid")
                             for c in range(2))
            ref = ref[::stride, ::stride, ::stride]
            assert y[o].shape == ref.shape
            assert np.abs(y[o] - ref).max() < 1e-12


def test_output_sizes():
    assert [N.out_size(32, s) for s in (1, 2)] == [32, 16]
    assert N.out_size(16, 2) == 8 and N.out_size(7, 2) == 4
    assert N.n_params() == 27 * 4 * 16 + 16 + 27 * 16 * 32 + 32 + 27 * 32 * 64 + 64 + 27 * 64 * 64 + 64 + \
        64 * 128 + 128 + 128 * 21 + 21


def test_input_channels_and_core_mask():
    lab = np.array([[[0, 1, 2, 3]]], dtype=np.uint8)  # (1, 1, 4): one voxel of each label
    x = N.net_input(lab)
    assert x.shape == (4, 1, 1, 4)
    assert np.array_equal(x[:3, 0, 0], [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]])  # label 3: no phase
    assert np.all(x[3] == 1.0)  # no core given: the whole box is the core
    m = N.core_mask((5, 6, 7), (1, 2, 3, 4, 3, 2))  # x0 1, y0 2, z0 3; 4 x 3 x 2 voxels
    assert m.sum() == 4 * 3 * 2 and m[3:5, 2:5, 1:5].all()
    # a non-cubic box runs through the global pool
    theta = N.init_params(RNG.random(N.n_params()))
    out, cache = N.forward(theta, RNG.integers(0, 3, size=(9, 6, 13)).astype(np.uint8), (2, 1, 2, 9, 4, 5))
    assert out.shape == (21,) and cache["acts"][-1].shape == (64, 3, 2, 4)


def _fd(f, a, idx, h=1e-6):
    a0 = a[idx]
    a[idx] = a0 + h
    fp = f()
    a[idx] = a0 - h
    fm = f()
    a[idx] = a0
    return (fp - fm) / (2 * h)


@pytest.mark.parametrize("stride", [1, 2])
def test_conv3d_backward_finite_differences(stride):
    x = RNG.standard_normal((2, 5, 6, 4))
    w = RNG.standard_normal((27, 2, 3))
    b = RNG.standard_normal(3)
    dy = RNG.standard_normal(N.conv3d(x, w, b, stride).shape)
    dx, dw, db = N.conv3d_backward(x, w, stride, dy)
    L = lambda: float(np.sum(dy * N.conv3d(x, w, b, stride)))
    for _ in range(6):
        i = tuple(RNG.integers(0, s) for s in x.shape)
        assert abs(_fd(L, x, i) - dx[i]) < 1e-6 * (1 + abs(dx[i]))
        j = tuple(RNG.integers(0, s) for s in w.shape)
        assert abs(_fd(L, w, j) - dw[j]) < 1e-6 * (1 + abs(dw[j]))
    k = (1,)
    assert abs(_fd(L, b, k) - db[k]) < 1e-6 * (1 + abs(db[k]))


def test_network_gradient_finite_differences():
    theta = N.init_params(RNG.random(N.n_params()))
    theta += 0.01 * RNG.standard_normal(theta.size)  # nonzero biases
    labs = [RNG.integers(0, 3, size=(8, 8, 8)).astype(np.uint8), RNG.integers(0, 3, size=(6, 9, 7)).astype(np.uint8)]
    cores = [None, (1, 2, 1, 5, 5, 4)]  # a buffered, non-cubic box with its core
    tg = RNG.standard_normal((2, N.NOUT))
    loss, grad, _ = N.batch_loss_and_grad(theta, labs, tg, cores)
    f = lambda: N.batch_loss_and_grad(theta, labs, tg, cores)[0]
    # one coordinate in every layer's weights and biases
    o = 0
    for name, shape in N.layer_shapes():
        n = int(np.prod(shape))
        i = o + int(RNG.integers(0, n))
        g = _fd(f, theta, i, h=1e-5)
        assert abs(g - grad[i]) <= 1e-5 * max(1e-3, abs(g)) + 1e-9, name
        o += n


def test_adam_first_step_closed_form():
    theta = RNG.standard_normal(5)
    g = RNG.standard_normal(5)
    new, m, v = N.adam_step(theta, g, np.zeros(5), np.zeros(5), 1, lr=1e-2, eps=0.0)
    # bias-corrected first moments are g and g^2: the step is lr * sign(g)
    assert np.allclose(new, theta - 1e-2 * np.sign(g), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_second_step_written_out():
    # two steps with gradients g1, g2: m2 = 0.09 g1 + 0.1 g2, v2 = 0.000999 g1^2
    # + 0.001 g2^2, bias corrections 1 - 0.9^2 = 0.19 and 1 - 0.999^2 = 0.001999
    theta = RNG.standard_normal(7)
    g1, g2 = RNG.standard_normal(7), RNG.standard_normal(7)
    t1, m, v = N.adam_step(theta, g1, np.zeros(7), np.zeros(7), 1, lr=3e-3)
    t2, m, v = N.adam_step(t1, g2, m, v, 2, lr=2e-3)
    m2 = 0.09 * g1 + 0.1 * g2
    v2 = 0.000999 * g1 * g1 + 0.001 * g2 * g2
    step2 = 2e-3 * (m2 / 0.19) / (np.sqrt(v2 / 0.001999) + 1e-8)
    assert np.allclose(t2, t1 - step2, rtol=0, atol=1e-15)


def test_cosine_step_size_special_values():
    lr, T = 0.02, 40
    assert N.cosine_step_size(lr, 0, T) == lr
    assert abs(N.cosine_step_size(lr, T // 2, T) - lr / 2) < 1e-18
    assert abs(N.cosine_step_size(lr, T, T)) < 1e-18
    s = np.array([N.cosine_step_size(lr, t, T) for t in range(T + 1)])
    # half a cosine period: decreasing, and symmetric about the midpoint
    assert np.all(np.diff(s) < 0)
    assert np.allclose(s + s[::-1], lr, rtol=0, atol=1e-17)


def test_train_full_batch_first_update_is_the_closed_form_step():
    theta = init_small()
    labels = RNG.integers(0, 3, size=(2, 4, 4, 4)).astype(np.uint8)
    targets = RNG.standard_normal((2, N.NOUT))
    new, losses = N.train_full_batch(theta, labels, targets, 1, 1e-3)
    loss, g, _ = N.batch_loss_and_grad(theta, labels, targets)
    # one update at the full step size: lr g / (|g| + 1e-8) per parameter
    assert losses[0] == loss
    assert np.allclose(new, theta - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # and the loss falls over a few updates on a fixed batch
    _, losses = N.train_full_batch(theta, labels, targets, 6, 1e-2)
    assert losses[-1] < losses[0]


def init_small():
    return N.init_params(np.random.default_rng(5).random(N.n_params()))


def test_init_params_bounds():
    theta = N.init_params(RNG.random(N.n_params()))
    p = N.unflatten(theta)
    for name, shape in N.layer_shapes():
        if name.endswith(".b"):
            assert np.all(p[name] == 0)
        else:
            bound = np.sqrt(6.0 / np.prod(shape[:-1]))
            assert np.abs(p[name]).max() <= bound and np.abs(p[name]).max() > 0.5 * bound


def _iso_c21(K, G):
    lam = K - 2 * G / 3
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[np.arange(3), np.arange(3)] += 2 * G
    C[np.arange(3, 6), np.arange(3, 6)] = G
    return C[np.triu_indices(6)]


def test_gate_cases():
    lab = np.zeros((4, 4, 4), dtype=np.uint8)
    lab[:2] = 1
    ph = [[37.0, 44.0], [21.0, 7.0]]
    KR, KV, GR, GV = N.phase_bounds(lab, ph)
    assert KR < KV and GR < GV
    Km, Gm = 0.5 * (KR + KV), 0.5 * (GR + GV)
    good = [_iso_c21(Km * (1 + 0.001 * i), Gm) for i in range(4)]
    ok, mean = N.gate(good, lab, ph, 0.01)
    assert ok and np.allclose(mean, np.mean(good, axis=0))
    # a member outside the Voigt bound of K
    bad = good[:3] + [_iso_c21(1.01 * KV, Gm)]
    assert not N.gate(bad, lab, ph, 0.5)[0]
    # spread of G above the threshold
    spread = [_iso_c21(Km, Gm * (1 + 0.01 * i)) for i in range(4)]
    assert not N.gate(spread, lab, ph, 0.02)[0] and N.gate(spread, lab, ph, 0.05)[0]
    # indefinite mean (a shear entry below zero) with moduli in bounds
    c = _iso_c21(Km, Gm)
    C = N.c21_to_full(c)
    C[3, 3] = -1.0  # shear trace kept: K and G unchanged
    C[4, 4] += Gm + 1.0
    ci = C[np.triu_indices(6)]
    Kc, Gc = N.moduli_voigt(C)
    assert KR <= Kc <= KV and GR <= Gc <= GV
    assert not N.gate([ci] * 4, lab, ph, 0.01)[0]
