"""FP64 reference of the warm-start network (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
import this module; the product path never does.

The network is not part of the paper's method: it predicts the steady state
(rho, T) that the lattice Boltzmann method of Eqs. (1), (2)/(4) and (24)-(25)
relaxes to, so that the method can start close to it.  Architecture (a
4-level U-Net with base width C):

* encoder level l = 0..3 (width C 2^l): two 3x3 convolutions with circular
  padding (the domains are periodic), each followed by ReLU; levels 0..2 keep
  their output as a skip tensor and pass a 2x2 average pool down;
* decoder level l = 2..0: nearest-neighbour 2x upsampling of the level below,
  concatenation [upsampled, skip_l] along channels, two 3x3 conv + ReLU;
* head: 1x1 convolution C -> 2 (normalised rho and T), no activation.

Tensors are NHWC.  A 3x3 convolution is a cross-correlation: output pixel
(y, x) takes input (y + dy, x + dx) (mod H, W) with tap (dy + 1, dx + 1) of
W[cout, 3, 3, cin].  Loss: mean squared error over every output value.
Optimiser: Adam (Kingma & Ba) with bias correction.

Optional rounding emulation (``rnd``): the GPU stores activations and
activation gradients in BF16; passing ``rnd=bf16_round`` rounds exactly the
tensors the GPU rounds, so that both sides take the same ReLU decisions.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------- layout
def architecture(base=32, cin=3, cin_pad=32, levels=4, cout=2):
    """Ordered layer list: (name, cin_stored, cout, ksize, cin_real).

    cin_stored is the channel count of the stored input tensor (the network
    input is padded with zero channels to cin_pad); cin_real is the fan-in
    used by the initialiser."""
    L = []
    c_in = cin_pad
    for l in range(levels):
        w = base << l
        L.append((f"e{l}a", c_in, w, 3, cin if l == 0 else c_in))
        L.append((f"e{l}b", w, w, 3, w))
        c_in = w
    for l in reversed(range(levels - 1)):
        w = base << l
        cat = (base << (l + 1)) + w
        L.append((f"d{l}a", cat, w, 3, cat))
        L.append((f"d{l}b", w, w, 3, w))
    L.append(("head", base, cout, 1, base))
    return L


def param_count(arch):
    return sum(co * k * k * ci + co for _, ci, co, k, _ in arch)


def unpack(flat, arch):
    """Flat vector -> {name: (W [cout, k, k, cin], b [cout])} (views)."""
    P, o = {}, 0
    for name, ci, co, k, _ in arch:
        n = co * k * k * ci
        P[name] = (flat[o:o + n].reshape(co, k, k, ci), flat[o + n:o + n + co])
        o += n + co
    assert o == flat.size
    return P


# ------------------------------------------------------------- rounding
def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (8 significant bits), ties to even."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)                    # a = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)


def _id(a):
    return a


# ------------------------------------------------------------ primitives
TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shifted(x, dy, dx):
    """s[n, y, x] = x[n, (y + dy) mod H, (x + dx) mod W]."""
    return np.roll(x, shift=(-dy, -dx), axis=(1, 2))


def conv3(x, W, b):
    """3x3 circular cross-correlation + bias: y = b + sum_tap shift(x) W_tap^T."""
    y = np.broadcast_to(b, x.shape[:3] + (W.shape[0],)).copy()
    for dy, dx in TAPS:
        y += shifted(x, dy, dx) @ W[:, dy + 1, dx + 1, :].T
    return y


def conv3_dgrad(gy, W):
    """Adjoint of conv3 in x: gx[q] = sum_tap W_tap^T gy[q - off(tap)]."""
    gx = np.zeros(gy.shape[:3] + (W.shape[3],))
    for dy, dx in TAPS:
        gx += shifted(gy @ W[:, dy + 1, dx + 1, :], -dy, -dx)
    return gx


def conv3_wgrad(gy, x):
    """Gradient in W and b: gW[:, tap, :] = sum_p gy[p]^T shift(x)[p]; gb = sum_p gy[p]."""
    co, ci = gy.shape[3], x.shape[3]
    gW = np.zeros((co, 3, 3, ci))
    g2 = gy.reshape(-1, co)
    for dy, dx in TAPS:
        gW[:, dy + 1, dx + 1, :] = g2.T @ shifted(x, dy, dx).reshape(-1, ci)
    return gW, g2.sum(axis=0)


def relu(a):
    return np.maximum(a, 0.0)


def pool2(x):
    """2x2 average pool."""
    n, h, w, c = x.shape
    return x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def pool2_bwd(g):
    """Adjoint of pool2: each input pixel receives a quarter of its window's gradient."""
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) * 0.25


def up2(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_bwd(g):
    """Adjoint of up2: sum over each 2x2 block."""
    n, h, w, c = g.shape
    return g.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


# ------------------------------------------------------------ network
def forward(flat, x, arch, rnd=None, keep=False):
    """Network output y [N, H, W, cout] for input x [N, H, W, cin_stored]."""
    R = rnd or _id
    P = unpack(np.asarray(flat, dtype=np.float64), arch)
    if rnd is not None:
        # the 3x3 weights are stored in BF16; biases and the 1x1 head stay FP32
        P = {k: ((R(W), b) if W.shape[1] == 3 else (W, b)) for k, (W, b) in P.items()}
    levels = sum(1 for n, *_ in arch if n.endswith("a") and n.startswith("e"))
    C = {}
    h = R(np.asarray(x, dtype=np.float64))
    skips = []
    for l in range(levels):
        C[f"e{l}a"] = h
        a = R(relu(conv3(h, *P[f"e{l}a"])))
        C[f"e{l}b"] = a
        s = R(relu(conv3(a, *P[f"e{l}b"])))
        C[f"e{l}b:out"] = s
        C[f"e{l}a:out"] = a
        if l < levels - 1:
            skips.append(s)
            h = R(pool2(s))
        else:
            h = s
    for l in reversed(range(levels - 1)):
        cat = np.concatenate([up2(h), skips[l]], axis=3)
        C[f"d{l}a"] = cat
        c = R(relu(conv3(cat, *P[f"d{l}a"])))
        C[f"d{l}a:out"] = c
        C[f"d{l}b"] = c
        h = R(relu(conv3(c, *P[f"d{l}b"])))
        C[f"d{l}b:out"] = h
    C["head"] = h
    Wh, bh = P["head"]
    y = h @ Wh[:, 0, 0, :].T + bh
    if keep:
        return y, C, P, levels
    return y


def loss_and_grad(flat, x, target, arch, rnd=None, keep=False):
    """(mean squared error, flat gradient) at the given parameters; with
    keep=True also the forward cache and the activation-gradient tensors."""
    R = rnd or _id
    y, C, P, levels = forward(flat, x, arch, rnd=rnd, keep=True)
    diff = y - target
    loss = float(np.mean(diff * diff))
    gy = 2.0 * diff / diff.size
    G = {}
    # head
    h = C["head"]
    Wh, _ = P["head"]
    G["head"] = ((gy.reshape(-1, gy.shape[3]).T @ h.reshape(-1, h.shape[3]))[:, None, None, :],
                 gy.reshape(-1, gy.shape[3]).sum(axis=0))
    g = R((gy @ Wh[:, 0, 0, :]) * (h > 0))
    GT = {"gD0": g}
    cat_grads = {}
    # decoder, finest first
    for l in range(levels - 1):
        # g: gradient at the pre-activation of d{l}b
        G[f"d{l}b"] = conv3_wgrad(g, C[f"d{l}b"])
        g = R(conv3_dgrad(g, P[f"d{l}b"][0]) * (C[f"d{l}a:out"] > 0))
        GT[("gC", l)] = g
        G[f"d{l}a"] = conv3_wgrad(g, C[f"d{l}a"])
        gcat = R(conv3_dgrad(g, P[f"d{l}a"][0]))
        GT[("gCAT", l)] = gcat
        n_up = gcat.shape[3] - C[f"e{l}b:out"].shape[3]
        cat_grads[l] = gcat[..., n_up:]
        below = C[f"d{l + 1}b:out"] if l + 1 < levels - 1 else C[f"e{levels - 1}b:out"]
        g = R(up2_bwd(gcat[..., :n_up]) * (below > 0))
        GT[("gUP", l + 1)] = g
    # bottom level: g is the gradient at the pre-activation of e{L-1}b
    for l in reversed(range(levels)):
        G[f"e{l}b"] = conv3_wgrad(g, C[f"e{l}b"])
        g = R(conv3_dgrad(g, P[f"e{l}b"][0]) * (C[f"e{l}a:out"] > 0))
        GT[("gA", l)] = g
        G[f"e{l}a"] = conv3_wgrad(g, C[f"e{l}a"])
        if l == 0:
            break
        gp = R(conv3_dgrad(g, P[f"e{l}a"][0]))
        GT[("gP", l - 1)] = gp
        g = R((pool2_bwd(gp) + cat_grads[l - 1]) * (C[f"e{l - 1}b:out"] > 0))
        GT[("gS", l - 1)] = g
    out = []
    for name, ci, co, k, _ in arch:
        gW, gb = G[name]
        out.append(np.asarray(gW).reshape(-1))
        out.append(np.asarray(gb).reshape(-1))
    if keep:
        return loss, np.concatenate(out), C, GT
    return loss, np.concatenate(out)


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------- warm-start handoff
def denormalise(y, rho_dev_scale, t_dev_scale, rho0, T0, rho_floor=1e-4):
    """Network output -> (rho_hat, T_hat).  Both outputs are deviations from the
    case's initial fields: rho_hat = max(rho0 + rho_dev_scale y0, rho_floor)
    (the method needs a positive density), T_hat = T0 (1 + t_dev_scale y1)."""
    return (np.maximum(rho0 + rho_dev_scale * y[..., 0], rho_floor),
            T0 * (1.0 + t_dev_scale * y[..., 1]))


def warm_project(rho_hat, T_hat, rho0, T0):
    """Per case, match the mass (Eq. 13) and energy (sum C_i = 0 under Eq. 24)
    of the initial state:
    1. move mass inside the interfaces: rho1 = rho_hat + lam w with the
       interface weight w = (rho_hat - lo)(hi - rho_hat), lo/hi the case's
       extreme predicted densities (w = 0 in both bulk phases), and
       lam = (sum rho0 - sum rho_hat) / sum w, limited to |lam| (hi - lo) <= 1
       so that rho1 stays within [lo, hi] (lam = 0 if sum w = 0);
    2. rho = rho1 sum(rho0) / sum(rho1) (exact mass whatever step 1 left);
    3. T = T_hat sum(rho0 T0) / sum(rho T_hat)."""
    ax = tuple(range(1, rho_hat.ndim))
    lo = rho_hat.min(axis=ax, keepdims=True)
    hi = rho_hat.max(axis=ax, keepdims=True)
    w = (rho_hat - lo) * (hi - rho_hat)
    S0 = rho0.sum(axis=ax, keepdims=True)
    SW = w.sum(axis=ax, keepdims=True)
    lam = np.where(SW > 0, (S0 - rho_hat.sum(axis=ax, keepdims=True)) / np.where(SW > 0, SW, 1.0), 0.0)
    cap = 1.0 / np.where(hi > lo, hi - lo, 1.0)
    lam = np.clip(lam, -cap, cap)
    r1 = rho_hat + lam * w
    r = r1 * (S0 / r1.sum(axis=ax, keepdims=True))
    e0 = (rho0 * T0).sum(axis=ax, keepdims=True)
    T = T_hat * (e0 / (r * T_hat).sum(axis=ax, keepdims=True))
    return r, T
