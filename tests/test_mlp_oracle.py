"""The MLP oracle of the learned continuation: gradients against finite differences, pole-model properties."""
import numpy as np

from oracle import mlp_oracle as mo


def _batch(seed=3, B=5, J=7):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, mo.N_IN))
    scale = rng.uniform(0.5, 2.0, size=B)
    z = np.concatenate([1j * rng.uniform(0.01, 5, size=(B, 3)), rng.uniform(0, 10, size=(B, J - 3)) + 1e-3j], axis=1)
    W_ref = -rng.uniform(0.1, 1.0, size=(B, J)) + 0.05j * rng.normal(size=(B, J))
    return x, scale, z, W_ref


def test_gradient_matches_finite_differences():
    theta = mo.init_params(1)
    x, scale, z, W_ref = _batch()
    L, g = mo.loss_and_grad(theta, x, scale, z, W_ref)
    rng = np.random.default_rng(7)
    # every bias and a sample of weights in each layer
    idx, off = [], 0
    for i, o in mo.LAYERS:
        idx += list(off + rng.choice(i * o, size=12, replace=False))
        idx += list(off + i * o + np.arange(min(o, 8)))
        off += i * o + o
    for k in idx:
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (mo.loss(tp, x, scale, z, W_ref) - mo.loss(tm, x, scale, z, W_ref)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, fd, g[k])
    assert abs(L - mo.loss(theta, x, scale, z, W_ref)) < 1e-15


def test_pole_model_is_negative_on_imaginary_axis_and_even():
    Om = np.array([[0.5, 2.0, 7.0] + [1.0] * 5])
    r = np.array([[0.2, 0.1, 0.05] + [0.0] * 5])
    xi = np.geomspace(1e-3, 1e3, 50)[None, :]
    W = mo.model_w(Om, r, np.array([1.3]), 1j * xi)
    assert np.all(W.real <= 0) and np.max(np.abs(W.imag)) < 1e-15
    z = np.array([[0.3 + 1e-3j, 4.0 + 1e-3j]])
    assert np.allclose(mo.model_w(Om, r, np.array([1.0]), z), mo.model_w(Om, r, np.array([1.0]), -z))


def test_gelu_and_softplus_closed_forms():
    a = np.array([-3.0, -0.5, 0.0, 0.7, 4.0])
    assert abs(mo.gelu(np.array([0.0]))[0]) == 0.0
    assert np.allclose(mo.gelu(a) - mo.gelu(-a), a)            # 0.5 a (1 + erf) + 0.5 a (1 - erf) = a
    h = 1e-6
    assert np.allclose((mo.gelu(a + h) - mo.gelu(a - h)) / (2 * h), mo.gelu_prime(a), atol=1e-8)
    assert np.allclose(mo.softplus(np.array([0.0])), np.log(2.0))
    assert np.allclose(mo.softplus(np.array([50.0])), 50.0)
