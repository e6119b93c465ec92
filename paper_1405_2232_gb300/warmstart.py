"""Learned warm start of the batched steady-state solve.

Pipeline (every numerical step runs in the CUDA library):

1. ``generate``: run sweep cases (``inputs.warm_start_cases``: T/T_c, G,
   tau_f from the batched sweep's distributions, droplet or slab, fixed L x L)
   to steady state with the batched solver; the converged states are the
   training targets.
2. ``train``: fit the U-Net (include/unet.h) to map (T/T_c, G, initial liquid
   mask) to the steady (rho, T), with Adam on shuffled mini-batches.
3. ``evaluate``: on unseen cases, solve once from the plain initial state and
   once from the network's prediction (handoff ``un_warm_fields``: density and
   temperature rescaled to the initial mass and energy, then the start at rest
   under the force, lb_params.init_balanced), both with the same batched
   solver and residual test; report wall-clock seconds and steps, and three
   more arms on the same cases: the plain fields at rest (no network), the
   predicted density with the initial temperature, and the prediction at
   u = 0 in f^eq.

Run as ``python -m paper_1405_2232_gb300.warmstart [--train N] [--test N]``;
it prints one JSON object.  The sweep recipe: psi from the domain's T0
(passive temperature), the mixed force of Eq. (4) with beta = 1.3, Eq. (24)
for g, FP32 storage, tau_g = 0.8.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs as I
from . import lb
from . import unet as UN

BETA = 1.3
TOL = 1e-8
K = 100


def sweep_params(doms, thermal=lb.LB_THERMAL_EQ24, precision="fp32", init_balanced=0):
    return [lb.lb_params_default(nx=d.L, ny=d.L, tau_f=d.tau_f, tau_g=d.tau_g, G=d.G, beta=BETA,
                                 thermal=thermal, precision=precision, psi_uses_local_T=0,
                                 T_psi=d.T_over_Tc * I.CS_TC, init_balanced=init_balanced)
            for d in doms]


def _sync():
    import torch
    torch.cuda.synchronize()


def solve(params, rhos, Ts, cap, device_inputs=False, chunk_rows=None):
    """Batched run to r < TOL; returns steps, residual, status, wall seconds, batch."""
    B = lb.Batch(params, rhos, Ts, device_inputs=device_inputs)
    if chunk_rows:
        B.chunk_rows = chunk_rows
    t0 = time.perf_counter()
    steps, resid, st = B.run(TOL, K=K, max_steps=cap)
    return steps, resid, st, time.perf_counter() - t0, B


def generate(n, L=256, seed=5, cap=40000, chunk_rows=None, near_tol=0.0):
    """Steady states of n sweep cases: (domains, masks, index, rho, T, info).

    The targets are the converged cases, plus (near_tol > 0) those stopped by
    the step cap with a residual below near_tol."""
    doms, masks = I.warm_start_cases(n, L=L, seed=seed)
    params = sweep_params(doms)
    steps, resid, st, wall, B = solve(params, [d.rho for d in doms], [d.T for d in doms], cap,
                                      chunk_rows=chunk_rows)
    ok = np.flatnonzero((st == lb.LB_OK) | ((st == lb.LB_ERR_NOT_CONVERGED) & (resid < near_tol)))
    rho = np.empty((ok.size, L, L), dtype=np.float32)
    T = np.empty((ok.size, L, L), dtype=np.float32)
    for j, d in enumerate(ok):
        r, t = B.fields(int(d))
        rho[j], T[j] = r, t
    B.close()
    info = dict(cases=n, converged=int(np.sum(st == lb.LB_OK)), targets=int(ok.size), failed=int(np.sum((st != lb.LB_OK) & (st != lb.LB_ERR_NOT_CONVERGED))),
                capped=int(np.sum(st == lb.LB_ERR_NOT_CONVERGED)), wall_s=wall,
                median_steps=float(np.median(steps[st == lb.LB_OK])) if np.any(st == lb.LB_OK) else None)
    return doms, masks, ok, rho, T, info


def case_inputs(doms, masks):
    return I.unet_input_planes([d.T_over_Tc for d in doms], [d.G for d in doms], masks)


def train(X, Y, L, epochs=30, batch=16, lr=1e-3, seed=7, log=None, augment=True):
    """Train a fresh network on device tensors X [n, L, L, 3], Y [n, L, L, 2].

    The network and the batch preparation share one CUDA stream: the training
    step does not synchronise, so a batch built on another stream could be
    freed and its memory handed to the next batch by torch's caching allocator
    while the network's kernels still read it."""
    import torch
    s_train = torch.cuda.Stream()
    s_train.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s_train):
        return _train_on_stream(X, Y, L, epochs, batch, lr, seed, log, augment, s_train)


def _train_on_stream(X, Y, L, epochs, batch, lr, seed, log, augment, stream):
    import torch
    net = UN.UNet(L, L, batch, stream=stream)
    arch = [("", ci, co, k, (3 if i == 0 else ci)) for i, (ci, co, k, _) in enumerate(UN.layer_table(net.cfg))]
    net.set_params(I.unet_init_params(arch, seed=11))
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    per_epoch = max(1, n // batch)
    total = epochs * per_epoch
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = rng.permutation(n)
        for s in range(0, n - batch + 1, batch):
            idx = torch.from_numpy(order[s:s + batch]).to(X.device)
            xb = X.index_select(0, idx)
            yb = Y.index_select(0, idx)
            if augment:
                # the periodic box is invariant under shifts, reflections and
                # the transposition of x and y: one random symmetry per batch
                sh = (int(rng.integers(L)), int(rng.integers(L)))
                xb, yb = torch.roll(xb, sh, dims=(1, 2)), torch.roll(yb, sh, dims=(1, 2))
                for ax in (1, 2):
                    if rng.random() < 0.5:
                        xb, yb = torch.flip(xb, (ax,)), torch.flip(yb, (ax,))
                if rng.random() < 0.5:
                    xb, yb = xb.transpose(1, 2), yb.transpose(1, 2)
            xb, yb = xb.contiguous(), yb.contiguous()
            last = s + 2 * batch > n
            # cosine decay from lr to lr / 20
            lr_t = lr * (0.05 + 0.95 * 0.5 * (1.0 + np.cos(np.pi * step / total)))
            loss = net.train_step(xb, yb, batch, lr_t, want_loss=last)
            step += 1
        losses.append(loss)
        if log:
            log(f"epoch {ep}: loss {loss:.5f}")
    net.synchronize()
    return net, losses, time.perf_counter() - t0


def predict(net, X, batch):
    import torch
    n, L = X.shape[0], X.shape[1]
    out = torch.empty((n, L, L, 2), dtype=torch.float32, device=X.device)
    for s in range(0, n, batch):
        m = min(batch, n - s)
        net.forward(X[s:s + m], out[s:s + m], m)
    net.synchronize()
    return out


def handoff(net, doms, masks, batch, norm=None):
    """Network prediction -> device fields (rho, T) of every case after the
    handoff (un_warm_fields: mass and energy of the initial fields restored);
    returns (d_rho, d_T, seconds), inference and handoff timed together."""
    import torch
    dev = torch.device("cuda")
    L = doms[0].L
    rho0 = torch.from_numpy(np.stack([d.rho for d in doms])).to(dev)
    T0 = torch.from_numpy(np.stack([d.T for d in doms])).to(dev)
    X = torch.from_numpy(case_inputs(doms, masks)).to(dev)
    _sync()
    t0 = time.perf_counter()
    pred = predict(net, X, batch)
    d_rho = torch.empty_like(rho0)
    d_T = torch.empty_like(T0)
    UN.warm_fields(len(doms), L, L, pred, I.UNET_NORM if norm is None else norm, rho0, T0, d_rho, d_T)
    _sync()
    return d_rho, d_T, time.perf_counter() - t0


def solve_with_fallback(params_warm, warm_fields, params_plain, plain_fields, cap, probe, chunk_rows=None):
    """Warm-started batched solve with the plain solve as fallback.

    Every domain starts from its warm fields; after `probe` steps each domain
    that has not converged (still relaxing, or failed) restarts from its plain
    initial fields (lb_batch_restart) and runs on with the remaining budget,
    so no domain takes more than `cap` steps over both starts.  warm_fields /
    plain_fields: (rho list, T list) of device addresses or host arrays.
    Returns steps, residual, status, wall seconds and the number of restarts."""
    rw, tw = warm_fields
    dev_in = not isinstance(rw[0], np.ndarray)
    B = lb.Batch(params_warm, rw, tw, device_inputs=dev_in)
    if chunk_rows:
        B.chunk_rows = chunk_rows
    t0 = time.perf_counter()
    steps, resid, st = B.run(TOL, K=K, max_steps=probe)
    restarts = 0
    for d in np.flatnonzero(st != lb.LB_OK):
        B.restart(int(d), plain_fields[0][d], plain_fields[1][d], init_balanced=params_plain[d].init_balanced)
        restarts += 1
    if restarts:
        steps, resid, st = B.run(TOL, K=K, max_steps=max(0, cap - probe))
    wall = time.perf_counter() - t0
    B.close()
    return steps, resid, st, wall, restarts


def evaluate(net, doms, masks, cap, batch=16, chunk_rows=None, probe=2000,
             arms_wanted=("plain", "plain_balanced", "warm", "warm_T0", "warm_fallback")):
    """Plain solve from the initial fields (f^eq at u = 0) against warm solves
    from the network's prediction after the handoff (mass and energy restored),
    with the start at rest under the force.  Beside them: the plain fields
    started at rest (no network), the predicted density with the initial
    temperature (t_dev_scale = 0 in the handoff), and the warm start with the
    plain solve as fallback (solve_with_fallback after `probe` steps).  The
    warm arms' wall seconds include inference and handoff."""
    L = doms[0].L
    params = sweep_params(doms)
    params_bal = sweep_params(doms, init_balanced=1)
    rho0 = np.stack([d.rho for d in doms])
    T0 = np.stack([d.T for d in doms])
    arms, per_case = {}, {}

    def record(name, steps, st, wall, extra_s, start, **kw):
        arms[name] = dict(wall_s=wall + extra_s, solve_s=wall, converged=int(np.sum(st == lb.LB_OK)),
                          failed=int(np.sum((st != lb.LB_OK) & (st != lb.LB_ERR_NOT_CONVERGED))),
                          capped=int(np.sum(st == lb.LB_ERR_NOT_CONVERGED)), start=start, **kw)
        per_case[name] = (steps, st)

    def run(name, prm, rhos, Ts, device_inputs, start, extra_s=0.0, keep=False):
        steps, _, st, wall, B = solve(prm, rhos, Ts, cap, device_inputs=device_inputs, chunk_rows=chunk_rows)
        kept = {int(d): B.fields(int(d)) for d in np.flatnonzero(st == lb.LB_OK)} if keep else None
        B.close()
        record(name, steps, st, wall, extra_s, start)
        return kept

    ref = run("plain", params, list(rho0), list(T0), False, "f^eq at u = 0", keep=True)
    if "plain_balanced" in arms_wanted:
        run("plain_balanced", params_bal, list(rho0), list(T0), False, "at rest under the force")
    stride = L * L * 8
    d_rho, d_T, t_inf = handoff(net, doms, masks, batch)
    rp = [d_rho.data_ptr() + i * stride for i in range(len(doms))]
    tp = [d_T.data_ptr() + i * stride for i in range(len(doms))]
    if "warm" in arms_wanted:
        run("warm", params_bal, rp, tp, True, "at rest under the force", t_inf)
        arms["warm"]["inference_s"] = t_inf
    if "warm_fallback" in arms_wanted:
        steps, _, st, wall, nr = solve_with_fallback(params_bal, (rp, tp), params, (list(rho0), list(T0)), cap,
                                                     probe, chunk_rows=chunk_rows)
        record("warm_fallback", steps, st, wall, t_inf, f"at rest under the force; plain restart after {probe} steps",
               restarts=nr, inference_s=t_inf)
    if "warm_T0" in arms_wanted:
        d_rho0_, d_T0_, t_inf0 = handoff(net, doms, masks, batch, dict(I.UNET_NORM, t_dev_scale=0.0))
        rp0 = [d_rho0_.data_ptr() + i * stride for i in range(len(doms))]
        tp0 = [d_T0_.data_ptr() + i * stride for i in range(len(doms))]
        run("warm_T0", params_bal, rp0, tp0, True, "at rest under the force", t_inf0)
        arms["warm_T0"]["inference_s"] = t_inf0
    # prediction error against the plain steady state
    h_rho, h_T = d_rho.cpu().numpy(), d_T.cpu().numpy()
    e_rho = [np.abs(h_rho[d] - ref[d][0]).max() / np.abs(ref[d][0]).max() for d in ref]
    e_T = [np.abs(h_T[d] - ref[d][1]).max() / np.abs(ref[d][1]).max() for d in ref]
    e_T0 = [np.abs(T0[d] - ref[d][1]).max() / np.abs(ref[d][1]).max() for d in ref]
    rms_rho = [float(np.sqrt(np.mean((h_rho[d] - ref[d][0]) ** 2))) for d in ref]
    rms_rho0 = [float(np.sqrt(np.mean((rho0[d] - ref[d][0]) ** 2))) for d in ref]
    rms_T = [float(np.sqrt(np.mean((h_T[d] - ref[d][1]) ** 2)) / ref[d][1].mean()) for d in ref]
    rms_T0 = [float(np.sqrt(np.mean((T0[d] - ref[d][1]) ** 2)) / ref[d][1].mean()) for d in ref]
    st_p, steps_p = per_case["plain"][1], per_case["plain"][0]
    allc = np.flatnonzero(np.all([v[1] == lb.LB_OK for v in per_case.values()], axis=0))
    vs_plain = {}
    for k, (steps_k, st_k) in per_case.items():
        if k == "plain":
            continue
        both = np.flatnonzero((st_p == lb.LB_OK) & (st_k == lb.LB_OK))
        vs_plain[k] = dict(both_converged=int(both.size),
                           median_steps_plain=float(np.median(steps_p[both])) if both.size else None,
                           median_steps=float(np.median(steps_k[both])) if both.size else None,
                           steps_ratio=float(np.sum(steps_k[both]) / np.sum(steps_p[both])) if both.size else None,
                           total_steps_ratio=float(np.sum(steps_k) / np.sum(steps_p)))
    med = lambda v: float(np.median(v)) if v else None
    out = dict(
        cases=len(doms), L=L, cap=cap, probe=probe, **arms,
        all_arms_converged=int(allc.size),
        median_steps_all_arms={k: (float(np.median(v[0][allc])) if allc.size else None)
                               for k, v in per_case.items()},
        vs_plain=vs_plain,
        prediction_error=dict(e_rho_median=med(e_rho), e_T_median=med(e_T), e_T_initial_state_median=med(e_T0),
                              e_rho_max=float(np.max(e_rho)) if e_rho else None, rms_rho_median=med(rms_rho),
                              rms_rho_initial_state_median=med(rms_rho0), rms_T_rel_median=med(rms_T),
                              rms_T_initial_state_rel_median=med(rms_T0)),
    )
    pc = dict(T_over_Tc=[d.T_over_Tc for d in doms], tau_f=[d.tau_f for d in doms],
              kind=[d.kind for d in doms], e_rho={int(d): float(e) for d, e in zip(ref, e_rho)})
    for k, (steps, st) in per_case.items():
        pc["steps_" + k] = steps.tolist()
        pc["status_" + k] = st.tolist()
    out["per_case"] = pc
    return out


def compare(L=128, n_train=1024, n_test=128, train_cap=20000, test_cap=40000, epochs=60, batch=16, probe=2000):
    """Warm vs plain on a reduced case (for the benchmark): train a network on
    n_train solves at L x L, then solve n_test unseen cases plain, warm, and
    warm with the plain fallback.  Returns the evaluation summary (no per-case
    lists) with the training figures."""
    import torch
    dev = torch.device("cuda")
    t0 = time.perf_counter()
    doms, masks, ok, rho, T, gen = generate(n_train, L=L, seed=5, cap=train_cap, near_tol=0.0)
    X = torch.from_numpy(case_inputs([doms[i] for i in ok], masks[ok])).to(dev)
    Y = torch.from_numpy(I.unet_target_planes(rho, T, np.stack([doms[i].rho for i in ok]),
                                              [doms[i].T_over_Tc * I.CS_TC for i in ok])).to(dev)
    net, losses, t_train = train(X, Y, L, epochs=epochs, batch=batch)
    tdoms, tmasks = I.warm_start_cases(n_test, L=L, seed=6)
    ev = evaluate(net, tdoms, tmasks, test_cap, batch=batch, probe=probe,
                  arms_wanted=("plain", "warm", "warm_fallback"))
    net.close()
    ev.pop("per_case")
    ev["train"] = dict(cases=n_train, targets=int(ok.size), epochs=epochs, seconds=round(t_train, 2),
                       train_cap=train_cap, generate_s=round(gen["wall_s"], 2), loss_last=float(losses[-1]))
    ev["seconds_total"] = round(time.perf_counter() - t0, 1)
    return ev


def train_step_bench(L=256, batch=16, steps=10, warmup=3):
    """Time the network's training step (forward, backward, Adam) on random
    inputs with CUDA events on the net's stream; returns (ms per step, GFLOP)."""
    import torch
    dev = torch.device("cuda")
    s = torch.cuda.Stream()
    net = UN.UNet(L, L, batch, stream=s)
    table = UN.layer_table(net.cfg)
    arch = [("", ci, co, k, (3 if i == 0 else ci)) for i, (ci, co, k, _) in enumerate(table)]
    net.set_params(I.unet_init_params(arch))
    g = torch.Generator(device=dev).manual_seed(0)
    x = torch.randn((batch, L, L, 3), device=dev, generator=g)
    t = torch.tanh(x[..., :2]).contiguous()
    torch.cuda.synchronize()
    for _ in range(warmup):
        net.train_step(x, t, batch, 1e-3, want_loss=False)
    net.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        net.train_step(x, t, batch, 1e-3, want_loss=False)
    e1.record(s)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / max(steps, 1)
    levels = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0, 0]
    gflop = 0.0
    for (ci, co, k, _), lev in zip(table, levels):
        px = batch * (L >> lev) ** 2
        gflop += 2.0 * px * co * ci * k * k * (3 if k == 3 else 2) / 1e9  # forward, input and weight gradients
    net.close()
    return ms, gflop


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=256)
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--cap", type=int, default=40000)
    ap.add_argument("--test-cap", type=int, default=80000)
    ap.add_argument("--epochs", type=int, default=120)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--dump", default=None, help="write per-case results (JSON) to this path")
    ap.add_argument("--train-step-bench", action="store_true",
                    help="only time the training step on random data (--L, --batch) and exit")
    ap.add_argument("--steps", type=int, default=10, help="timed steps of --train-step-bench")
    a = ap.parse_args(argv)
    if a.train_step_bench:
        ms, gflop = train_step_bench(a.L, a.batch, a.steps, warmup=min(3, a.steps))
        print(json.dumps(dict(L=a.L, batch=a.batch, ms_per_step=ms, gflop_per_step=gflop,
                              tflops=gflop / ms)))
        return
    import torch
    dev = torch.device("cuda")
    log = (lambda s: print(s, flush=True)) if a.verbose else None
    doms, masks, ok, rho, T, gen = generate(a.train, L=a.L, seed=5, cap=a.cap)
    if log:
        log(f"generated: {gen}")
    X = torch.from_numpy(case_inputs([doms[i] for i in ok], masks[ok])).to(dev)
    Y = torch.from_numpy(I.unet_target_planes(rho, T, np.stack([doms[i].rho for i in ok]),
                                              [doms[i].T_over_Tc * I.CS_TC for i in ok])).to(dev)
    net, losses, t_train = train(X, Y, a.L, epochs=a.epochs, batch=a.batch, lr=a.lr, log=log)
    # fit on (up to) 64 training cases, in the units of the targets
    m = min(64, X.shape[0])
    P = predict(net, X[:m], a.batch)
    fit = ((P - Y[:m]) ** 2).mean(dim=(0, 1, 2)).sqrt().cpu().numpy()
    if log:
        log(f"train fit rms (rho, T channels, normalised): {fit}")
    tdoms, tmasks = I.warm_start_cases(a.test, L=a.L, seed=6)
    ev = evaluate(net, tdoms, tmasks, a.test_cap, batch=a.batch)
    net.close()
    per_case = ev.pop("per_case")
    if a.dump:
        with open(a.dump, "w") as fh:
            json.dump(per_case, fh)
    print(json.dumps(dict(generate=gen, train=dict(samples=int(ok.size), epochs=a.epochs, batch=a.batch,
                                                   lr=a.lr, seconds=t_train, loss_first=losses[0],
                                                   loss_last=losses[-1], fit_rms_normalised=fit.tolist()),
                          test=ev)))


if __name__ == "__main__":
    main()
