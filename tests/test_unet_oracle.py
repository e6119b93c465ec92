"""Pins of the FP64 warm-start network reference (oracle/unet.py).

Each pin checks the oracle against something other than itself: a library
routine on an independent path (FFT convolution, torch's bfloat16 rounding),
adjoint identities, central finite differences of the loss, closed forms of
the Adam update, and the parameter count worked out by hand."""
import numpy as np
import pytest

from oracle import unet as U


def rng(seed=0):
    return np.random.default_rng(seed)


def test_param_count_by_hand():
    # e0a 32*9*32+32, e0b 32*9*32+32, e1a 64*9*32+64, e1b 64*9*64+64,
    # e2a 128*9*64+128, e2b 128*9*128+128, e3a 256*9*128+256, e3b 256*9*256+256,
    # d2a 128*9*384+128, d2b 128*9*128+128, d1a 64*9*192+64, d1b 64*9*64+64,
    # d0a 32*9*96+32, d0b 32*9*32+32, head 2*32+2
    assert U.param_count(U.architecture()) == 1_955_266
    names = [a[0] for a in U.architecture()]
    assert names == ["e0a", "e0b", "e1a", "e1b", "e2a", "e2b", "e3a", "e3b",
                     "d2a", "d2b", "d1a", "d1b", "d0a", "d0b", "head"]


def test_bf16_round_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    x = rng(1).standard_normal(20000).astype(np.float32) * np.float32(3.0) ** rng(2).integers(-20, 20, 20000)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16_round(x.astype(np.float64)), ref)
    one = 1.0
    assert U.bf16_round(one + 2.0 ** -8) == 1.0                 # tie -> even (1.0)
    assert U.bf16_round(one + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even
    assert U.bf16_round(-(one + 2.0 ** -7)) == -(1.0 + 2.0 ** -7)


def conv_fft(x, W, b):
    """Circular cross-correlation through the FFT (independent of np.roll)."""
    n, h, w, ci = x.shape
    co = W.shape[0]
    K = np.zeros((co, ci, h, w))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            K[:, :, (-dy) % h, (-dx) % w] += W[:, dy + 1, dx + 1, :]
    X = np.fft.fft2(np.moveaxis(x, 3, 1))          # [n, ci, h, w]
    Y = np.einsum("ncyx,ocyx->noyx", X, np.fft.fft2(K))
    y = np.real(np.fft.ifft2(Y))
    return np.moveaxis(y, 1, 3) + b


@pytest.mark.parametrize("h,w", [(8, 8), (6, 10), (3, 5)])
def test_conv3_equals_fft_circular_correlation(h, w):
    r = rng(3)
    x = r.standard_normal((2, h, w, 5))
    W = r.standard_normal((4, 3, 3, 5))
    b = r.standard_normal(4)
    assert np.allclose(U.conv3(x, W, b), conv_fft(x, W, b), atol=1e-12)


def test_conv3_delta_kernel_is_a_shift():
    x = rng(4).standard_normal((1, 6, 7, 2))
    W = np.zeros((2, 3, 3, 2))
    W[0, 0, 2, 0] = 1.0   # tap dy=-1, dx=+1 of channel 0 -> output 0
    W[1, 1, 1, 1] = 1.0   # centre tap of channel 1 -> output 1
    y = U.conv3(x, W, np.zeros(2))
    for yy in range(6):
        for xx in range(7):
            assert y[0, yy, xx, 0] == x[0, (yy - 1) % 6, (xx + 1) % 7, 0]
    assert np.array_equal(y[..., 1], x[..., 1])


def test_dgrad_wgrad_are_adjoints():
    r = rng(5)
    x = r.standard_normal((2, 8, 6, 3))
    W = r.standard_normal((4, 3, 3, 3))
    b = r.standard_normal(4)
    g = r.standard_normal((2, 8, 6, 4))
    lhs = np.sum(U.conv3(x, W, np.zeros(4)) * g)
    assert np.isclose(lhs, np.sum(x * U.conv3_dgrad(g, W)), rtol=1e-12)
    gW, gb = U.conv3_wgrad(g, x)
    assert np.isclose(np.sum(U.conv3(x, W, b) * g), np.sum(W * gW) + np.sum(b * gb), rtol=1e-12)


def test_pool_and_upsample():
    x = np.arange(16.0).reshape(1, 4, 4, 1)
    p = U.pool2(x)
    assert p[0, :, :, 0].tolist() == [[2.5, 4.5], [10.5, 12.5]]
    assert np.array_equal(U.up2(p)[0, :2, :2, 0], np.full((2, 2), 2.5))
    r = rng(6)
    a, g = r.standard_normal((2, 4, 6, 3)), r.standard_normal((2, 2, 3, 3))
    assert np.isclose(np.sum(U.pool2(a) * g), np.sum(a * U.pool2_bwd(g)), rtol=1e-13)
    assert np.isclose(np.sum(U.up2(g) * a), np.sum(g * U.up2_bwd(a)), rtol=1e-13)


def he_init(arch, r):
    parts = []
    for _, ci, co, k, fan in arch:
        parts.append(r.standard_normal(co * k * k * ci) * np.sqrt((2.0 if k == 3 else 1.0) / (k * k * fan)))
        parts.append(0.1 * r.standard_normal(co))
    return np.concatenate(parts)


def tiny_problem(seed=7, base=2, hw=16, he=False):
    arch = U.architecture(base=base, cin=3, cin_pad=4)
    r = rng(seed)
    flat = he_init(arch, r) if he else r.standard_normal(U.param_count(arch)) * 0.5
    x = r.standard_normal((2, hw, hw, 4))
    x[..., 3] = 0.0
    t = r.standard_normal((2, hw, hw, 2))
    return arch, flat, x, t


def fd_check(loss_and_grad, n_samples=300, seed=8):
    arch, flat, x, t = tiny_problem()
    _, g = loss_and_grad(flat, x, t, arch)
    idx = rng(seed).choice(flat.size, n_samples, replace=False)
    eps = 1e-6
    worst = 0.0
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += eps
        fm[i] -= eps
        fd = (U.loss_and_grad(fp, x, t, arch)[0] - U.loss_and_grad(fm, x, t, arch)[0]) / (2 * eps)
        worst = max(worst, abs(fd - g[i]))
    return worst / np.abs(g).max()


def test_gradient_matches_central_differences():
    assert fd_check(U.loss_and_grad) < 1e-6


def test_finite_difference_check_catches_a_wrong_adjoint(monkeypatch):
    """Planting a mistake in the oracle (dgrad without the tap flip) must fail the pin."""
    def wrong_dgrad(gy, W):
        gx = np.zeros(gy.shape[:3] + (W.shape[3],))
        for dy, dx in U.TAPS:
            gx += U.shifted(gy @ W[:, dy + 1, dx + 1, :], dy, dx)
        return gx
    monkeypatch.setattr(U, "conv3_dgrad", wrong_dgrad)
    assert fd_check(U.loss_and_grad, n_samples=60) > 1e-3


def test_adam_closed_forms():
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = v = np.zeros(3)
    q = p.copy()
    for t in range(1, 6):   # constant gradient: every step moves lr g / (|g| + eps)
        q, m, v = U.adam_step(q, g, m, v, t, lr, b1, b2, eps)
        assert np.allclose(q, p - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # gradient +1 then -1: the second step is +lr (1 - b1)/(1 + b1) / (1 + eps)
    q, m, v = U.adam_step(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), 1, lr, b1, b2, eps)
    q2, _, _ = U.adam_step(q, -np.ones(1), m, v, 2, lr, b1, b2, eps)
    assert np.isclose(q2[0] - q[0], lr * (1 - b1) / (1 + b1) / (1 + eps), rtol=1e-12)


def test_training_reduces_loss():
    arch, flat, x, _ = tiny_problem(seed=9, base=4, he=True)
    t = np.tanh(x[..., :2])  # a target the network can represent
    m = v = np.zeros_like(flat)
    losses = []
    for step in range(1, 61):
        loss, g = U.loss_and_grad(flat, x, t, arch)
        losses.append(loss)
        flat, m, v = U.adam_step(flat, g, m, v, step, 1e-3)
    assert losses[-1] < 0.85 * losses[0] and losses[30] < losses[0]


def test_rounding_emulation_stays_close():
    arch, flat, x, t = tiny_problem(seed=10, base=4, he=True)
    y = U.forward(flat, x, arch)
    yr = U.forward(flat, x, arch, rnd=U.bf16_round)
    assert np.abs(y - yr).max() <= 5e-2 * np.abs(y).max()
    assert not np.array_equal(y, yr)


def test_warm_project_conserves_mass_and_energy():
    r = rng(11)
    rho0 = 0.05 + r.random((3, 12, 10))
    T0 = 0.08 + 0.01 * r.random((3, 12, 10))
    rho_hat = rho0 * (1.1 + 0.05 * r.standard_normal((3, 12, 10)))
    T_hat = T0 * 0.97
    rho, T = U.warm_project(rho_hat, T_hat, rho0, T0)
    assert np.allclose(rho.sum(axis=(1, 2)), rho0.sum(axis=(1, 2)), rtol=1e-14)
    assert np.allclose((rho * T).sum(axis=(1, 2)), (rho0 * T0).sum(axis=(1, 2)), rtol=1e-14)
    same = U.warm_project(rho0, T0, rho0, T0)
    assert np.allclose(same[0], rho0, rtol=1e-14) and np.allclose(same[1], T0, rtol=1e-14)


def test_warm_project_moves_interfaces_not_bulk():
    """A smooth slab predicted about one site too wide: the correction lands in
    the two interfaces and leaves both bulk densities untouched."""
    L = 64
    x = np.arange(L) + 0.5
    def slab(half):
        return (0.165 + 0.135 * np.tanh((half - np.abs(x - 32)) / 2.0))[None, None, :].repeat(L, axis=1)
    rho0, pred = slab(12.0), slab(12.5)
    T0 = np.full_like(rho0, 0.08)
    rho, _ = U.warm_project(pred, T0, rho0, T0)
    assert np.isclose(rho.sum(), rho0.sum(), rtol=1e-14)
    bulk = (np.abs(x - 32) < 2) | (np.abs(x - 32) > 26)
    assert np.abs(rho[0][:, bulk] - pred[0][:, bulk]).max() < 1e-4
    assert np.abs(rho - rho0).max() < 0.2 * np.abs(pred - rho0).max()
    assert rho.min() >= pred.min() - 1e-15 and rho.max() <= pred.max() + 1e-15


def test_denormalise():
    y = np.array([[[[0.5, 2.0], [-3.0, 0.0]]]])
    rho0 = np.array([[[0.1, 0.2]]])
    T0 = np.full((1, 1, 2), 0.08)
    r, T = U.denormalise(y, 0.1, 0.01, rho0, T0, rho_floor=1e-4)
    assert np.allclose(r, [[[0.15, 1e-4]]]) and np.allclose(T, [[[0.08 * 1.02, 0.08]]])
    # a zero output gives back the initial state
    r, T = U.denormalise(np.zeros((1, 1, 2, 2)), 0.1, 0.01, rho0, T0)
    assert np.array_equal(r, rho0) and np.array_equal(T, T0)


def test_initial_parameters_recipe():
    from paper_1405_2232_gb300 import inputs as I
    arch = U.architecture()
    flat = I.unet_init_params(arch)
    assert flat.dtype == np.float32 and flat.size == U.param_count(arch)
    P = U.unpack(flat.astype(np.float64), arch)
    W0, b0 = P["e0a"]
    assert np.all(W0[..., 3:] == 0) and np.all(b0 == 0)
    # He-normal spread: std sqrt(2/(9*3)) for the first layer, sqrt(2/(9*256)) for e3b
    assert abs(W0[..., :3].std() / np.sqrt(2 / 27) - 1) < 0.1
    assert abs(P["e3b"][0].std() / np.sqrt(2 / 2304) - 1) < 0.01
    assert abs(P["head"][0].std() / np.sqrt(1 / 32) - 1) < 0.3
