"""Warm-start network on the GPU against the FP64 reference (oracle/unet.py).

Layer by layer, each BF16 tensor-core convolution is fed the GPU's own input
tensor and compared with the reference convolution of that input (BF16
weights, FP64 sums, one rounding to BF16): the only difference left is the
FP32 accumulation order, so the tolerance is about one BF16 unit.  The whole
network is compared with the reference run in BF16-rounding emulation, and
the gradients layer by layer (each weight gradient from the GPU's own
gradient and input tensors: FP32 accumulation only) and as a whole."""
import numpy as np
import pytest

from oracle import unet as U
from paper_1405_2232_gb300 import inputs as I

H = W = 32
NB = 2
BASE = 32
# (H, W, batch) of the layer-by-layer checks: 32 x 32 runs the mma.sync
# kernels at every level; 128 x 256 also runs the tcgen05 convolution on the
# two finest levels (image widths 256 and 128)
SHAPES = [(32, 32, 2), (128, 256, 1)]


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    return _t


@pytest.fixture(scope="module")
def N():
    from paper_1405_2232_gb300 import unet as _n
    _n.load()
    return _n


def problem(seed=21, shape=(H, W, NB)):
    h, w, nb = shape
    arch = U.architecture(base=BASE)
    flat = I.unet_init_params(arch).astype(np.float64)
    r = np.random.default_rng(seed)
    P = U.unpack(flat, arch)
    for name, (Wt, b) in P.items():
        b[:] = 0.05 * r.standard_normal(b.size)
    flat = flat.astype(np.float32)
    x = r.standard_normal((nb, h, w, 3)).astype(np.float32)
    t = np.tanh(x[..., :2] + 0.5 * x[..., 2:3]).astype(np.float32)
    return arch, flat, x, t


def pad(x):
    out = np.zeros(x.shape[:3] + (32,))
    out[..., :3] = x
    return out


@pytest.fixture(scope="module", params=SHAPES, ids=lambda s: f"{s[0]}x{s[1]}x{s[2]}")
def run(torch, N, request):
    """One forward + backward on the GPU; every tensor fetched to the host."""
    H, W, NB = request.param
    arch, flat, x, t = problem(shape=request.param)
    dev = torch.device("cuda")
    with N.UNet(H, W, NB, BASE) as net:
        net.set_params(flat)
        d_in = torch.from_numpy(x).to(dev)
        d_t = torch.from_numpy(t).to(dev)
        d_out = torch.empty((NB, H, W, 2), dtype=torch.float32, device=dev)
        torch.cuda.synchronize()  # inputs copied on torch's stream, read on the net's
        net.forward(d_in, d_out, NB)
        net.synchronize()  # the net runs on a stream of its own
        y = d_out.cpu().numpy().astype(np.float64)
        loss = net.loss_grad(d_in, d_t, NB)
        grads = net.grads().astype(np.float64)
        T = {}
        for l in range(4):
            s = (NB, H >> l, W >> l)
            c = BASE << l
            T[("A", l)] = net.tensor(N.UN_T_A + l, s + (c,))
            T[("gA", l)] = net.tensor(N.UN_T_GRAD + N.UN_T_A + l, s + (c,))
            if l < 3:
                cc = (BASE << (l + 1)) + c
                T[("CAT", l)] = net.tensor(N.UN_T_CAT + l, s + (cc,))
                T[("gCAT", l)] = net.tensor(N.UN_T_GRAD + N.UN_T_CAT + l, s + (cc,))
                s1 = (NB, H >> (l + 1), W >> (l + 1))
                T[("P", l)] = net.tensor(N.UN_T_P + l, s1 + (c,))
                T[("gP", l)] = net.tensor(N.UN_T_GRAD + N.UN_T_P + l, s1 + (c,))
                T[("C", l)] = net.tensor(N.UN_T_C + l, s + (c,))
                T[("gC", l)] = net.tensor(N.UN_T_GRAD + N.UN_T_C + l, s + (c,))
                T[("gS", l)] = net.tensor(N.UN_T_GRAD + N.UN_T_SKIP + l, s + (c,))
            if l >= 1:
                T[("gUP", l)] = net.tensor(N.UN_T_GRAD + N.UN_T_UP + l, s + (c,))
        T["X0"] = net.tensor(N.UN_T_X0, (NB, H, W, 32))
        T["D0"] = net.tensor(N.UN_T_D0, (NB, H, W, BASE))
        T["gD0"] = net.tensor(N.UN_T_GRAD + N.UN_T_D0, (NB, H, W, BASE))
    return dict(arch=arch, flat=flat.astype(np.float64), x=x, t=t, y=y, loss=loss, grads=grads,
                T={k: v.astype(np.float64) for k, v in T.items()})


def close_bf16(gpu, ref, what):
    """|gpu - ref| within about one BF16 unit of ref (FP32 vs FP64 sums before the rounding)."""
    tol = 2.0 ** -7 * np.abs(ref) + 1e-6 * np.abs(ref).max() + 1e-30
    bad = np.abs(gpu - ref) > tol
    assert bad.mean() < 1e-3, (what, bad.mean(), np.abs(gpu - ref).max(), np.abs(ref).max())


def conv_ref(x, P, name, relu=True):
    Wt, b = P[name]
    y = U.conv3(x, U.bf16_round(Wt), b)
    return U.bf16_round(U.relu(y) if relu else y)


@pytest.mark.gpu
def test_input_and_each_forward_layer(run):
    T, P = run["T"], U.unpack(run["flat"], run["arch"])
    assert np.array_equal(T["X0"], U.bf16_round(pad(run["x"])))
    close_bf16(T[("A", 0)], conv_ref(T["X0"], P, "e0a"), "e0a")
    for l in range(4):
        if l > 0:
            close_bf16(T[("A", l)], conv_ref(T[("P", l - 1)], P, f"e{l}a"), f"e{l}a")
        if l < 3:
            c = BASE << l
            skip = T[("CAT", l)][..., (BASE << (l + 1)):]
            close_bf16(skip, conv_ref(T[("A", l)], P, f"e{l}b"), f"e{l}b")
            close_bf16(T[("P", l)], U.bf16_round(U.pool2(skip)), f"pool{l}")
    close_bf16(T[("CAT", 2)][..., :BASE << 3], U.up2(conv_ref(T[("A", 3)], P, "e3b")), "e3b+up")
    for l in (2, 1, 0):
        close_bf16(T[("C", l)], conv_ref(T[("CAT", l)], P, f"d{l}a"), f"d{l}a")
        out = T["D0"] if l == 0 else T[("CAT", l - 1)][..., :BASE << l]
        ref = conv_ref(T[("C", l)], P, f"d{l}b")
        close_bf16(out, ref if l == 0 else U.up2(ref), f"d{l}b")
    Wh, bh = P["head"]
    yh = T["D0"] @ Wh[:, 0, 0, :].T + bh
    assert np.abs(run["y"] - yh).max() <= 1e-5 * np.abs(yh).max()


@pytest.mark.gpu
def test_whole_forward_against_rounding_emulation(run):
    ref = U.forward(run["flat"], pad(run["x"]), run["arch"], rnd=U.bf16_round)
    e = np.abs(run["y"] - ref).max() / np.abs(ref).max()
    assert e < 2e-2, e
    plain = U.forward(run["flat"], pad(run["x"]), run["arch"])
    assert np.abs(run["y"] - plain).max() / np.abs(plain).max() < 5e-2


@pytest.mark.gpu
def test_each_backward_tensor(run):
    T, P = run["T"], U.unpack(run["flat"], run["arch"])
    R = U.bf16_round
    Wb = {k: R(v[0]) for k, v in P.items() if v[0].shape[1] == 3}
    # head: gD0 = R((gy Wh) * (d0 > 0)), gy = 2 (y - t) / count
    gy = 2.0 * (run["y"] - run["t"]) / run["y"].size
    close_bf16(T["gD0"], R((gy @ P["head"][0][:, 0, 0, :]) * (T["D0"] > 0)), "head")
    for l in range(3):
        gin = T["gD0"] if l == 0 else T[("gUP", l)]
        close_bf16(T[("gC", l)], R(U.conv3_dgrad(gin, Wb[f"d{l}b"]) * (T[("C", l)] > 0)), f"d{l}b dgrad")
        close_bf16(T[("gCAT", l)], R(U.conv3_dgrad(T[("gC", l)], Wb[f"d{l}a"])), f"d{l}a dgrad")
        cu = BASE << (l + 1)
        close_bf16(T[("gUP", l + 1)], R(U.up2_bwd(T[("gCAT", l)][..., :cu]) *
                                         (T[("CAT", l)][..., :cu][:, ::2, ::2] > 0)), f"up{l + 1}")
    for l in (3, 2, 1, 0):
        gin = T[("gUP", 3)] if l == 3 else T[("gS", l)]
        close_bf16(T[("gA", l)], R(U.conv3_dgrad(gin, Wb[f"e{l}b"]) * (T[("A", l)] > 0)), f"e{l}b dgrad")
        if l > 0:
            close_bf16(T[("gP", l - 1)], R(U.conv3_dgrad(T[("gA", l)], Wb[f"e{l}a"])), f"e{l}a dgrad")
            cs = BASE << l
            s = T[("CAT", l - 1)][..., cs:]
            close_bf16(T[("gS", l - 1)], R((U.pool2_bwd(T[("gP", l - 1)]) + T[("gCAT", l - 1)][..., cs:]) * (s > 0)),
                       f"skip{l - 1}")


def layer_grads(flat_grads, arch):
    return U.unpack(flat_grads, arch)


@pytest.mark.gpu
def test_each_weight_gradient(run):
    T, arch = run["T"], run["arch"]
    G = layer_grads(run["grads"], arch)
    inputs = {"e0a": T["X0"], "d0b": T[("C", 0)]}
    outg = {"d0b": T["gD0"]}
    for l in range(4):
        inputs[f"e{l}b"] = T[("A", l)]
        outg[f"e{l}a"] = T[("gA", l)]
        outg[f"e{l}b"] = T[("gUP", 3)] if l == 3 else T[("gS", l)]
        if l > 0:
            inputs[f"e{l}a"] = T[("P", l - 1)]
    for l in range(3):
        inputs[f"d{l}a"] = T[("CAT", l)]
        outg[f"d{l}a"] = T[("gC", l)]
        if l > 0:
            inputs[f"d{l}b"] = T[("C", l)]
            outg[f"d{l}b"] = T[("gUP", l)]
    for name, *_ in arch[:-1]:
        gW, gb = U.conv3_wgrad(outg[name], inputs[name])
        eW = np.abs(G[name][0] - gW).max() / np.abs(gW).max()
        eb = np.abs(G[name][1] - gb).max() / np.abs(gb).max()
        assert eW < 1e-4 and eb < 1e-4, (name, eW, eb)
    h = T["D0"].reshape(-1, BASE)
    gy = (2.0 * (run["y"] - run["t"]) / run["y"].size).reshape(-1, 2)
    assert np.abs(G["head"][0][:, 0, 0, :] - gy.T @ h).max() <= 1e-4 * np.abs(gy.T @ h).max()
    assert np.abs(G["head"][1] - gy.sum(axis=0)).max() <= 1e-4 * np.abs(gy.sum(axis=0)).max()


@pytest.mark.gpu
def test_loss_and_whole_gradient_against_emulation(run):
    loss, g = U.loss_and_grad(run["flat"], pad(run["x"]), run["t"], run["arch"], rnd=U.bf16_round)
    assert run["loss"] == pytest.approx(loss, rel=2e-2)
    G, Gr = layer_grads(run["grads"], run["arch"]), layer_grads(g, run["arch"])
    for name in G:
        e = np.linalg.norm(G[name][0] - Gr[name][0]) / np.linalg.norm(Gr[name][0])
        assert e < 5e-2, (name, e)
    # padding channels of the input get no gradient
    assert np.all(G["e0a"][0][..., 3:] == 0)


@pytest.mark.gpu
def test_adam_step_and_training(torch, N):
    arch, flat, x, t = problem(seed=22)
    dev = torch.device("cuda")
    with N.UNet(H, W, NB, BASE) as net:
        net.set_params(flat)
        d_in, d_t = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
        torch.cuda.synchronize()  # inputs copied on torch's stream, read on the net's
        net.loss_grad(d_in, d_t, NB)
        g = net.grads().astype(np.float64)
        net.adam_step(1e-3)
        p1 = net.params().astype(np.float64)
        ref, _, _ = U.adam_step(flat.astype(np.float64), g, 0 * g, 0 * g, 1, 1e-3)
        assert np.abs(p1 - ref).max() <= 1e-6
        net.set_params(flat)
        losses = [net.train_step(d_in, d_t, NB, 2e-3) for _ in range(40)]
    assert losses[-1] < 0.7 * losses[0], losses[::8]


@pytest.mark.gpu
def test_warm_handoff(torch, N):
    r = np.random.default_rng(23)
    n, h, w = 3, 16, 24
    pred = r.standard_normal((n, h, w, 2)).astype(np.float32)
    pred[0, :3, :3, 0] = -5.0   # below the density floor
    rho0 = 0.05 + 0.3 * r.random((n, h, w))
    T0 = 0.08 + 0.01 * r.random((n, h, w))
    dev = torch.device("cuda")
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_rho, d_T = torch.empty((n, h, w), dtype=torch.float64, device=dev), torch.empty((n, h, w), dtype=torch.float64, device=dev)
    N.warm_fields(n, h, w, d(pred), I.UNET_NORM, d(rho0), d(T0), d_rho, d_T)
    torch.cuda.synchronize()
    nm = I.UNET_NORM
    rh, th = U.denormalise(pred.astype(np.float64), nm["rho_dev_scale"], nm["t_dev_scale"], rho0, T0)
    rr, tr = U.warm_project(rh, th, rho0, T0)
    assert np.allclose(d_rho.cpu().numpy(), rr, rtol=1e-13, atol=0)
    assert np.allclose(d_T.cpu().numpy(), tr, rtol=1e-13, atol=0)


@pytest.mark.gpu
def test_warmstart_training_learns_without_per_step_sync(torch, N):
    """warmstart.train issues its steps without synchronising and builds every
    augmented batch with torch ops; with the network on the same stream as the
    batches it learns a target that is a fixed local, mirror-symmetric function
    of the input planes (a smoothed mask and the T/T_c plane): the fit error
    ends below a third of the zero predictor's."""
    import torch.nn.functional as F
    from paper_1405_2232_gb300 import warmstart as WS
    L = 64
    doms, masks = I.warm_start_cases(64, L=L, seed=9)
    X = torch.from_numpy(WS.case_inputs(doms, masks)).cuda()
    m = X[..., 2:3].permute(0, 3, 1, 2)
    k = torch.ones(1, 1, 5, 5, device=X.device) / 25
    sm = F.conv2d(F.pad(m, (2, 2, 2, 2), mode="circular"), k)
    Y = torch.cat([torch.tanh(2 * sm).permute(0, 2, 3, 1), 0.3 * X[..., 0:1]], dim=3).contiguous()
    torch.cuda.synchronize()
    net, losses, _ = WS.train(X, Y, L, epochs=40, batch=16, lr=1e-3)
    P = WS.predict(net, X, 16)
    fit = float(((P - Y) ** 2).mean().sqrt())
    zero = float((Y ** 2).mean().sqrt())
    net.close()
    assert fit < zero / 3, (fit, zero, losses[::8])
