"""Plain FP64 CPU oracle of the learned continuation of W (pole-residue MLP).

TEST INFRASTRUCTURE ONLY (imported by tests/ and the CPU-baseline leg of bench.py, never by the CUDA library).

The network maps 32 samples of W_nm(i xi_k) (every third node of the imaginary grid, divided by the scale
s = |W_nm(i xi_1)|) through three hidden layers of 256 GELU units to 16 outputs, read as 8 poles
Omega_s = softplus(o_s) + omega_floor and residues r_s = softplus(o_{8+s}).  The model
    W(z) = -s * sum_s r_s 2 Omega_s / (Omega_s^2 - z^2)
is the sum-over-poles form of W behind Eq. sigma_pole (Sec. 2.1): W(i xi) <= 0 by construction.  The loss of one
sample is (1/J) sum_j |W(z_j) - W_ref(z_j)|^2 / (s^2 + |W_ref(z_j)|^2) over its reference points (imaginary nodes
and near-real points, Sec. 3.3): a relative error with the scale as floor, so that the spikes of W next to its
poles do not dominate; averaged over the batch.  Gradients follow the chain rule written out step by step; the
tests pin them against finite differences of the forward pass.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_POLES = 32, 256, 8
N_OUT = 2 * N_POLES
OMEGA_FLOOR = 0.05                      # Ha: the smallest pole position the head can produce
LAYERS = [(N_IN, N_HID), (N_HID, N_HID), (N_HID, N_HID), (N_HID, N_OUT)]
N_PARAMS = sum(i * o + o for i, o in LAYERS)


def unpack(theta):
    """Flat parameter vector -> [(W [in, out], b [out]), ...] (row-major weights, then bias, per layer)."""
    out, off = [], 0
    for i, o in LAYERS:
        W = theta[off:off + i * o].reshape(i, o)
        off += i * o
        b = theta[off:off + o]
        off += o
        out.append((W, b))
    return out


def init_params(seed=0):
    """He-style uniform initialisation (deterministic)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in LAYERS:
        lim = math.sqrt(6.0 / i) * (0.25 if o == N_OUT else 1.0)
        parts.append(rng.uniform(-lim, lim, size=i * o))
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def gelu(a):
    return 0.5 * a * (1.0 + np.vectorize(math.erf)(a / math.sqrt(2.0)))


def gelu_prime(a):
    Phi = 0.5 * (1.0 + np.vectorize(math.erf)(a / math.sqrt(2.0)))
    phi = np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)
    return Phi + a * phi


def softplus(y):
    return np.maximum(y, 0.0) + np.log1p(np.exp(-np.abs(y)))


def sigmoid(y):
    return 1.0 / (1.0 + np.exp(-y))


def forward(theta, x):
    """Returns (o [B, 16], cache of pre-activations and activations)."""
    layers = unpack(theta)
    h = x
    cache = [x]
    for li, (W, b) in enumerate(layers):
        a = h @ W + b
        if li < len(layers) - 1:
            cache.append(a)
            h = gelu(a)
            cache.append(h)
        else:
            h = a
    return h, cache


def poles(o):
    """(Omega [B, 8], r [B, 8]) from the network outputs."""
    return softplus(o[:, :N_POLES]) + OMEGA_FLOOR, softplus(o[:, N_POLES:])


def model_w(Omega, r, scale, z):
    """W(z) = -s sum_s r_s 2 Omega_s / (Omega_s^2 - z^2); z [B, J] complex -> [B, J]."""
    g = 2.0 * Omega[:, None, :] / (Omega[:, None, :] ** 2 - z[:, :, None] ** 2)
    return -scale[:, None] * np.sum(r[:, None, :] * g, axis=2)


def loss(theta, x, scale, z, W_ref):
    o, _ = forward(theta, x)
    Om, r = poles(o)
    e = model_w(Om, r, scale, z) - W_ref
    wgt = 1.0 / (scale[:, None] ** 2 + np.abs(W_ref) ** 2)
    return float(np.mean(np.mean(np.abs(e) ** 2 * wgt, axis=1)))


def loss_and_grad(theta, x, scale, z, W_ref):
    """Loss and its gradient with respect to the flat parameter vector (chain rule, FP64)."""
    B, J = z.shape
    layers = unpack(theta)
    o, cache = forward(theta, x)
    y_om, y_r = o[:, :N_POLES], o[:, N_POLES:]
    Om = softplus(y_om) + OMEGA_FLOOR
    r = softplus(y_r)
    den = Om[:, None, :] ** 2 - z[:, :, None] ** 2              # [B, J, 8]
    g = 2.0 * Om[:, None, :] / den
    dg = -2.0 * (Om[:, None, :] ** 2 + z[:, :, None] ** 2) / den ** 2
    Wm = -scale[:, None] * np.sum(r[:, None, :] * g, axis=2)
    e = Wm - W_ref
    wgt = 1.0 / (scale[:, None] ** 2 + np.abs(W_ref) ** 2)     # [B, J]
    L = float(np.mean(np.mean(np.abs(e) ** 2 * wgt, axis=1)))
    # dL/dp = sum_j (2 / (J B)) wgt_j Re(conj(e_j) dW_j/dp)
    c = (2.0 / (J * B)) * wgt                                   # [B, J]
    dWdr = -scale[:, None, None] * g                            # [B, J, 8]
    dWdOm = -scale[:, None, None] * r[:, None, :] * dg
    d_r = np.sum(c[:, :, None] * np.real(np.conj(e)[:, :, None] * dWdr), axis=1)
    d_Om = np.sum(c[:, :, None] * np.real(np.conj(e)[:, :, None] * dWdOm), axis=1)
    d_o = np.concatenate([d_Om * sigmoid(y_om), d_r * sigmoid(y_r)], axis=1)   # [B, 16]
    grads = [None] * len(layers)
    d_a = d_o
    n_hidden = len(layers) - 1
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        h_in = cache[0] if li == 0 else cache[2 * li]
        grads[li] = (h_in.T @ d_a, np.sum(d_a, axis=0))
        if li > 0:
            a_prev = cache[2 * li - 1]
            d_a = (d_a @ W.T) * gelu_prime(a_prev)
    flat = []
    for gW, gb in grads:
        flat.append(gW.reshape(-1))
        flat.append(gb)
    return L, np.concatenate(flat)


def features(W_imag_nm, every=3, n_in=N_IN):
    """x = W(i xi_{every k}) / s, s = |W(i xi_1)|, for one table [n_imag] per row of W_imag_nm [B, n_imag]."""
    idx = np.arange(n_in) * every
    s = np.abs(W_imag_nm[:, 0])
    return W_imag_nm[:, idx] / s[:, None], s, idx
