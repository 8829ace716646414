"""Learned collision-side closure: data, training and evaluation driver.

The paper leaves the constitutive determination of the turbulent relaxation
(more generally of the turbulent collision operator) as its main open point
(Sec. 8).  The learned closure keeps the KC-MP structure (App. F.3: SGS
carrier f_sgs = w/(2 theta^2) H:m_sgs, rate from k_sgs = |tr m_sgs|/2, clip by
the molecular rate) and learns m_sgs itself from data the method generates:

  1. fine-lattice decaying-turbulence runs (D3Q27, FP32, KC-MP);
  2. box filter by F of the fine populations -> coarse populations and the
     exact SGS stress of Eq. (m_sgs_2) (lbm_box_filter);
  3. per coarse cell the ten inputs (m_neq/rho, invariants of m_CE/rho,
     tau_hat of the coarse lattice, nu_coarse = nu_fine / F under acoustic
     scaling) and the target m_sgs/rho (lbm_closure_features);
  4. training with the library's own forward/backward/AdamW kernels;
  5. fused BF16 tensor-core inference in the step kernel (closure "learned").

A second training target ("dissipation") keeps the deviatoric part of the
exact SGS stress and replaces its trace by the one whose rate reproduces the
filtered field's local SGS energy transfer -m_sgs : S (the paper's open point
on determining the turbulent relaxation from collision statistics, Sec. 8).

Orchestration only: every numerical step runs in liblbm's kernels; torch holds
device buffers, computes the energy spectra used for evaluation and the
elementwise trace replacement of the dissipation target.
"""
from __future__ import annotations

import math
from typing import Dict, Sequence

import numpy as np
import torch

from . import inputs, lbm


def snapshot_features(s: lbm.Solver, factor: int, nu_coarse: float, nu_fine: float = None, pull: bool = True):
    """Box-filtered coarse state of a solver's current populations:
    (x [N,10], targets [N,6], analytic KC-MP estimate [N,6], coarse populations [q,nz,ny,nx]).

    pull: filter the streamed (pre-collision) populations, the state from which
    a step computes the closure inputs (features and targets); without it, the
    stored post-collision populations (an initial state for a coarse run).
    With nu_fine given, the filtered fine non-equilibrium part is rescaled by
    r = F tau_hat_c / tau_hat_f to the size the coarse lattice gives the same
    flow under acoustic scaling (the SGS part is kept)."""
    ptr, _ = s.population_buffer()
    nx, ny, nz = s.shape
    q = s.q
    ncx, ncy, ncz = nx // factor, ny // factor, nz // factor
    nc = ncx * ncy * ncz
    dev = torch.device("cuda")
    fc = torch.empty((q, ncz, ncy, ncx), dtype=torch.float32, device=dev)
    ms = torch.empty((6, ncz, ncy, ncx), dtype=torch.float32, device=dev)
    r = 1.0
    if nu_fine is not None:
        th = 1.0 / 3.0
        r = factor * (nu_coarse / th + 0.5) / (nu_fine / th + 0.5)
    lbm.lbm_box_filter(ptr, q, s.cfg.storage, nx, ny, nz, factor, fc.data_ptr(), ms.data_ptr(), neq_scale=r,
                       pull=pull)
    x = torch.empty((nc, 10), dtype=torch.float32, device=dev)
    t = torch.empty((nc, 6), dtype=torch.float32, device=dev)
    kc = torch.empty((nc, 6), dtype=torch.float32, device=dev)
    lbm.lbm_closure_features(fc.data_ptr(), q, ncx, ncy, ncz, nu_coarse, ms.data_ptr(), x.data_ptr(), t.data_ptr(),
                             kc.data_ptr())
    torch.cuda.synchronize()
    return x, t, kc, fc


def snapshot_strain(fc: torch.Tensor) -> torch.Tensor:
    """Strain rate S [N, 6] (xx yy zz xy xz yz) of coarse FP32 populations fc
    [q, nz, ny, nx] (lbm_closure_strain: the features' central differences)."""
    q, nz, ny, nx = fc.shape
    out = torch.empty((nz * ny * nx, 6), dtype=torch.float32, device=fc.device)
    lbm.lbm_closure_strain(fc.data_ptr(), q, nx, ny, nz, out.data_ptr())
    torch.cuda.synchronize()
    return out


def dissipation_targets(T: torch.Tensor, S: torch.Tensor, c_nu: float, delta: float = 1.0,
                        cap_quantile: float = 1.0) -> torch.Tensor:
    """The exact targets T = m_sgs/rho [N, 6] with their trace replaced by the
    one whose turbulent rate carries the local SGS energy transfer.  With the
    transfer Pi = -T : S (off-diagonal terms twice) and the eddy viscosity that
    dissipates it, nu* = max(Pi, 0) / (2 S : S), the rate nu_t = C_nu Delta
    sqrt(|tr m_sgs| / 2) of Eq. (omega_sgs_operational) equals nu* for
    tr = 2 (nu* / (C_nu Delta))^2.  The deviatoric part of T is kept.
    cap_quantile < 1 clips nu* at that quantile of its values in T (the ratio
    diverges where the filtered strain vanishes)."""
    Td, Sd = T.double(), S.double()
    w = torch.tensor([1.0, 1.0, 1.0, 2.0, 2.0, 2.0], dtype=torch.float64, device=T.device)
    pi = -(Td * Sd * w).sum(1)
    ss = (Sd * Sd * w).sum(1)
    nu_star = torch.where(ss > 0, torch.clamp(pi, min=0.0) / (2.0 * ss + 1e-300), torch.zeros_like(ss))
    if cap_quantile < 1.0:
        k = max(1, int(round(cap_quantile * nu_star.numel())))
        cap = torch.kthvalue(nu_star.cpu(), k).values.item()
        nu_star = torch.clamp(nu_star, max=cap)
    tr_new = 2.0 * (nu_star / (c_nu * delta)) ** 2
    tr_old = Td[:, 0] + Td[:, 1] + Td[:, 2]
    out = Td.clone()
    for k in range(3):
        out[:, k] += (tr_new - tr_old) / 3.0
    return out.float()


def generate(n_fine: int = 512, factor: int = 4, seeds: Sequence[int] = (0, 1, 2, 3, 4),
             k0s: Sequence[float] = (4.0, 8.0), nu_fine: float = 1e-4, urms: float = 0.04,
             snap_steps: Sequence[int] = (300, 600), keep: float = 0.25, sample_seed: int = 0,
             target: str = "exact", c_nu: float = 0.035, cap_quantile: float = 0.99):
    """Training samples from fine runs: returns (X, T, KC) on the GPU; target
    "exact" (the SGS stress of Eq. m_sgs_2) or "dissipation" (its trace
    replaced by dissipation_targets at this C_nu, nu* clipped at the snapshot's
    cap_quantile)."""
    assert target in ("exact", "dissipation"), target
    gen = torch.Generator(device="cuda").manual_seed(sample_seed)
    X, T, KC = [], [], []
    for k0 in k0s:
        for sd in seeds:
            with lbm.Solver(27, (n_fine,) * 3, nu_fine, closure="kcmp", storage="fp32") as s:
                rho, u = inputs.hit_fields(n_fine, k0=k0, urms=urms, seed=sd, device="cuda")
                s.init_velocity_device(rho, u)
                del rho, u
                done = 0
                for st in snap_steps:
                    s.step(st - done)
                    done = st
                    x, t, kc, fc = snapshot_features(s, factor, nu_fine / factor, nu_fine)
                    if target == "dissipation":
                        t = dissipation_targets(t, snapshot_strain(fc), c_nu, cap_quantile=cap_quantile)
                    n = x.shape[0]
                    idx = torch.randperm(n, generator=gen, device="cuda")[: max(1, int(keep * n))]
                    X.append(x[idx])
                    T.append(t[idx])
                    KC.append(kc[idx])
    return torch.cat(X), torch.cat(T), torch.cat(KC)


def standardisation(X: torch.Tensor, T: torch.Tensor) -> np.ndarray:
    """32 values: mean[10], std[10] of the inputs, mean[6], std[6] of the targets."""
    xm, xs = X.double().mean(0), X.double().std(0)
    tm, ts = T.double().mean(0), T.double().std(0)
    # a column that is constant up to rounding (tau_hat within one lattice) has a
    # spread of a few ulps of its mean: standardise it by 1, not by that spread
    xs = torch.where(xs > 1e-6 * xm.abs(), xs, torch.ones_like(xs))
    ts = torch.where(ts > 1e-6 * tm.abs(), ts, torch.ones_like(ts))
    return torch.cat([xm, xs, tm, ts]).cpu().numpy().astype(np.float32)


def init_params(seed: int = 0) -> np.ndarray:
    """U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, flat W1 b1 ... W4 b4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = (10, 64, 64, 64, 6)
    out = []
    for l in range(4):
        fi, fo = sizes[l], sizes[l + 1]
        out.append(rng.uniform(-1.0, 1.0, size=fo * fi) / math.sqrt(fi))
        out.append(np.zeros(fo))
    return np.concatenate(out).astype(np.float32)


def train(X: torch.Tensor, T: torch.Tensor, stats: np.ndarray, iters: int = 3000, batch: int = 8192,
          lr: float = 2e-3, wd: float = 1e-4, seed: int = 0, log_every: int = 0) -> Dict:
    """AdamW training on standardised data with the library's kernels."""
    dev = torch.device("cuda")
    st = torch.as_tensor(stats, device=dev)
    Xs = ((X.double() - st[:10].double()) / st[10:20].double()).float().contiguous()
    Ts = ((T.double() - st[20:26].double()) / st[26:32].double()).float().contiguous()
    n = Xs.shape[0]
    npar = lbm.lbm_mlp_param_count()
    p = torch.as_tensor(init_params(seed), device=dev)
    g = torch.zeros(npar, dtype=torch.float32, device=dev)
    m = torch.zeros_like(g)
    v = torch.zeros_like(g)
    b = min(batch, n)
    ws = torch.empty(lbm.lbm_mlp_workspace_floats(b), dtype=torch.float32, device=dev)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    hist = []
    for it in range(1, iters + 1):
        idx = torch.randint(0, n, (b,), generator=gen, device=dev)
        xb, tb = Xs[idx].contiguous(), Ts[idx].contiguous()
        want = log_every and (it % log_every == 0 or it == 1)
        loss = lbm.lbm_mlp_grad(p.data_ptr(), xb.data_ptr(), tb.data_ptr(), b, g.data_ptr(), ws.data_ptr(),
                                want_loss=bool(want))
        if want:
            hist.append((it, loss))
        lr_t = lr * 0.5 * (1 + math.cos(math.pi * it / iters))  # cosine decay
        lbm.lbm_mlp_adamw(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), it, lr_t, weight_decay=wd)
    torch.cuda.synchronize()
    return {"params": p.cpu().numpy(), "stats": stats, "history": hist}


def predict(params: np.ndarray, stats: np.ndarray, X: torch.Tensor) -> torch.Tensor:
    """Network prediction of m_sgs/rho (FP32 forward kernel) for raw inputs X."""
    dev = X.device
    st = torch.as_tensor(stats, device=dev)
    Xs = ((X.double() - st[:10].double()) / st[10:20].double()).float().contiguous()
    n = Xs.shape[0]
    p = torch.as_tensor(params, device=dev)
    ys = torch.empty((n, 6), dtype=torch.float32, device=dev)
    ws = torch.empty(lbm.lbm_mlp_workspace_floats(n), dtype=torch.float32, device=dev)
    lbm.lbm_mlp_forward(p.data_ptr(), Xs.data_ptr(), n, ys.data_ptr(), ws.data_ptr())
    torch.cuda.synchronize()
    return ys.double() * st[26:32].double() + st[20:26].double()


def a_priori(params, stats, X, T, KC) -> Dict:
    """Held-out errors of the m_sgs/rho estimates, normalised by the target variance:
    the network, the analytic KC-MP estimate (m_neq - m_CE)/rho, and zero."""
    var = float(((T.double() - T.double().mean(0)) ** 2).sum())
    net = float(((predict(params, stats, X) - T.double()) ** 2).sum()) / var
    kc = float(((KC.double() - T.double()) ** 2).sum()) / var
    zero = float((T.double() ** 2).sum()) / var
    trace_t = T[:, 0] + T[:, 1] + T[:, 2]
    trace_n = predict(params, stats, X)[:, :3].sum(1)
    trace_k = KC[:, 0] + KC[:, 1] + KC[:, 2]
    tv = float(((trace_t - trace_t.mean()) ** 2).sum())
    return {"rel_mse_network": net, "rel_mse_kcmp": kc, "rel_mse_zero": zero,
            "trace_rel_mse_network": float(((trace_n - trace_t.double()) ** 2).sum()) / tv,
            "trace_rel_mse_kcmp": float(((trace_k - trace_t) ** 2).double().sum()) / tv}


def spectrum(u: torch.Tensor) -> torch.Tensor:
    """Shell-averaged kinetic energy spectrum E(k) = 1/2 sum_{|k'| in [k-1/2, k+1/2)} |u_hat(k')|^2,
    u_hat normalised by 1/N (periodic cube, u [3, n, n, n])."""
    n = u.shape[-1]
    uh = torch.fft.fftn(u.double(), dim=(1, 2, 3)) / (n ** 3)
    e = 0.5 * (uh.real ** 2 + uh.imag ** 2).sum(0)
    k = torch.fft.fftfreq(n, d=1.0 / n, device=u.device)
    kk = torch.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    shell = torch.round(kk).long().ravel()
    return torch.zeros(n, dtype=torch.float64, device=u.device).index_add_(
        0, shell.clamp(max=n - 1), e.ravel())[: n // 2]


def _velocity(s: lbm.Solver) -> torch.Tensor:
    nx, ny, nz = s.shape
    r = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    u = torch.empty((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    s.moments_device(r, u)
    torch.cuda.synchronize()
    return u


def filtered_reference(n_fine: int, factor: int, k0: float, seed: int, nu_fine: float, urms: float, t0: int,
                       coarse_steps: int) -> Dict:
    """Fine run box-filtered at fine steps t0 and t0 + factor * coarse_steps: the
    coarse initial state (post-collision, rescaled non-equilibrium part), the
    filtered velocity, spectrum and kinetic energy at the end, and the filtered
    run's dissipation rate -dE_k/dt per coarse step over the window."""
    nu_c = nu_fine / factor
    with lbm.Solver(27, (n_fine,) * 3, nu_fine, closure="kcmp", storage="fp32") as fine:
        rho, u = inputs.hit_fields(n_fine, k0=k0, urms=urms, seed=seed, device="cuda")
        fine.init_velocity_device(rho, u)
        del rho, u
        fine.step(t0)
        _, _, _, fc0 = snapshot_features(fine, factor, nu_c, nu_fine, pull=False)
        f0 = fc0.double().cpu().numpy()
        fine.step(factor * coarse_steps)
        _, _, _, fc1 = snapshot_features(fine, factor, nu_c, nu_fine, pull=False)
    ref = _coarse_velocity(fc1, nu_c)
    ek0 = float(0.5 * (_coarse_velocity(fc0, nu_c) ** 2).sum(0).mean())
    ek1 = float(0.5 * (ref ** 2).sum(0).mean())
    return {"f0": f0, "spectrum": spectrum(ref), "E_k0": ek0, "E_k": ek1, "dissipation": (ek0 - ek1) / coarse_steps,
            "nu_c": nu_c, "coarse_steps": coarse_steps}


def coarse_run(closure: str, ref: Dict, params=None, stats=None, c_nu: float = None) -> Dict:
    """Coarse LES of `closure` from ref's initial state: E(k) relative L2 error
    over the resolved shells against the filtered fine run, E_k, dissipation."""
    nc = ref["f0"].shape[-1]
    kw = {} if c_nu is None else {"c_nu": c_nu}
    with lbm.Solver(27, (nc,) * 3, ref["nu_c"], closure=closure, storage="fp32", **kw) as s:
        if closure == "learned":
            s.set_learned_closure(params, stats)
        s.set_populations(ref["f0"])
        s.step(ref["coarse_steps"])
        u = _velocity(s)
    e = spectrum(u)
    ek = float(0.5 * (u ** 2).sum(0).mean())
    kmax = nc // 2
    e_ref = ref["spectrum"]
    err = torch.sqrt(((e[1:kmax] - e_ref[1:kmax]) ** 2).sum() / (e_ref[1:kmax] ** 2).sum())
    return {"spectrum_rel_l2": float(err), "E_k": ek, "dissipation": (ref["E_k0"] - ek) / ref["coarse_steps"]}


def calibrate_c_nu(closure: str, ref: Dict, params=None, stats=None, lo: float = 1e-3, hi: float = 0.5,
                   iters: int = 14) -> float:
    """C_nu whose coarse run dissipates as the filtered fine run over the window
    (bisection in log C_nu; the dissipation grows with C_nu); clamped to [lo, hi]."""
    target = ref["dissipation"]
    if coarse_run(closure, ref, params, stats, lo)["dissipation"] >= target:
        return lo
    if coarse_run(closure, ref, params, stats, hi)["dissipation"] <= target:
        return hi
    a, b = math.log(lo), math.log(hi)
    for _ in range(iters):
        m = 0.5 * (a + b)
        if coarse_run(closure, ref, params, stats, math.exp(m))["dissipation"] < target:
            a = m
        else:
            b = m
    return math.exp(0.5 * (a + b))


def a_posteriori(params, stats, n_fine: int = 512, factor: int = 4, k0: float = 4.0, seed: int = 99,
                 nu_fine: float = 1e-4, urms: float = 0.04, t0: int = 400, coarse_steps: int = 100,
                 closures=("kcmp", "learned", "bgk")) -> Dict:
    """Coarse LES from the filtered fine state at fine step t0, run `coarse_steps`
    coarse steps (= factor x as many fine steps under acoustic scaling) with each
    closure, against the box-filtered fine run: relative L2 error of E(k) over the
    resolved shells 1 <= k < n_coarse/2 and of the kinetic energy, and the
    dissipation rate -dE/dt over the window."""
    nc = n_fine // factor
    nu_c = nu_fine / factor
    out = {}
    with lbm.Solver(27, (n_fine,) * 3, nu_fine, closure="kcmp", storage="fp32") as fine:
        rho, u = inputs.hit_fields(n_fine, k0=k0, urms=urms, seed=seed, device="cuda")
        fine.init_velocity_device(rho, u)
        del rho, u
        fine.step(t0)
        _, _, _, fc0 = snapshot_features(fine, factor, nu_c, nu_fine, pull=False)
        f0 = fc0.double().cpu().numpy()
        fine.step(factor * coarse_steps)
        _, _, _, fc1 = snapshot_features(fine, factor, nu_c, nu_fine, pull=False)
    ref = _coarse_velocity(fc1, nu_c)
    e_ref = spectrum(ref)
    ek_ref = float(0.5 * (ref ** 2).sum(0).mean())
    ek_ref0 = float(0.5 * (_coarse_velocity(fc0, nu_c) ** 2).sum(0).mean())
    kmax = nc // 2
    for cl in closures:
        with lbm.Solver(27, (nc,) * 3, nu_c, closure=cl, storage="fp32") as s:
            if cl == "learned":
                s.set_learned_closure(params, stats)
            s.set_populations(f0)
            s.step(coarse_steps)
            u = _velocity(s)
        e = spectrum(u)
        ek = float(0.5 * (u ** 2).sum(0).mean())
        err = torch.sqrt(((e[1:kmax] - e_ref[1:kmax]) ** 2).sum() / (e_ref[1:kmax] ** 2).sum())
        out[cl] = {"spectrum_rel_l2": float(err), "E_k": ek, "dissipation": (ek_ref0 - ek) / coarse_steps}
    out["filtered_fine"] = {"E_k": ek_ref, "dissipation": (ek_ref0 - ek_ref) / coarse_steps}
    return out


def _coarse_velocity(fc: torch.Tensor, nu: float) -> torch.Tensor:
    """Velocity of a (filtered) FP32 population array, through the library's
    moments kernel on an FP64-storage solver holding those populations."""
    q, nz, ny, nx = fc.shape
    with lbm.Solver(q, (nx, ny, nz), nu, closure="bgk", storage="fp64") as s:
        s.set_populations(fc.double().cpu().numpy())
        return _velocity(s)


def _mlups(closure: str, n: int, nu: float, params=None, stats=None, steps: int = 50) -> float:
    """Steps per second of one closure on an n^3 FP32 D3Q27 box (CUDA events, graph replay)."""
    rho, u = inputs.hit_fields(n, k0=4.0, urms=0.04, seed=5, device="cuda")
    with lbm.Solver(27, (n,) * 3, nu, closure=closure, storage="fp32") as s:
        if closure == "learned":
            s.set_learned_closure(params, stats)
        s.init_velocity_device(rho, u)
        s.step(steps)  # warm-up and graph capture
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(steps)
        s.synchronize()
        e1.record(stream)
        torch.cuda.synchronize()
        return n ** 3 * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6


def main(argv=None) -> Dict:
    """Full pipeline: fine runs -> filtered data -> training -> held-out a priori
    errors -> a posteriori coarse LES -> throughput; writes the trained network
    (params, stats) to --out and prints one JSON line of results."""
    import argparse
    import json
    import os
    import time

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--n-fine", type=int, default=512)
    ap.add_argument("--factor", type=int, default=4)
    ap.add_argument("--train-seeds", default="0,1,2,3")
    ap.add_argument("--test-seeds", default="4")
    ap.add_argument("--k0s", default="4,8")
    ap.add_argument("--snap-steps", default="300,600")
    ap.add_argument("--keep", type=float, default=0.25)
    ap.add_argument("--iters", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--t0", type=int, default=400)
    ap.add_argument("--coarse-steps", type=int, default=150)
    ap.add_argument("--mlups-sizes", default="128,256")
    ap.add_argument("--target", default="exact", choices=["exact", "dissipation"],
                    help="training target: the exact SGS stress, or its trace set by the SGS energy transfer")
    ap.add_argument("--c-nu", type=float, default=0.035, help="C_nu of the dissipation target and its coarse runs")
    ap.add_argument("--out", default=None,
                    help="checkpoint (default data/learned_closure.npz, data/learned_closure_dissipation.npz)")
    a = ap.parse_args(argv)
    if a.out is None:
        name = "learned_closure.npz" if a.target == "exact" else "learned_closure_dissipation.npz"
        a.out = os.path.join(os.path.dirname(__file__), "data", name)
    ints = lambda s: tuple(int(v) for v in s.split(",") if v)
    floats = lambda s: tuple(float(v) for v in s.split(",") if v)
    nu_fine = 1e-4
    t = time.perf_counter()
    X, T, KC = generate(a.n_fine, a.factor, ints(a.train_seeds), floats(a.k0s), nu_fine, snap_steps=ints(a.snap_steps),
                        keep=a.keep, target=a.target, c_nu=a.c_nu)
    Xh, Th, KCh = generate(a.n_fine, a.factor, ints(a.test_seeds), floats(a.k0s), nu_fine,
                           snap_steps=ints(a.snap_steps), keep=a.keep, sample_seed=1, target=a.target, c_nu=a.c_nu)
    t_data = time.perf_counter() - t
    stats = standardisation(X, T)
    t = time.perf_counter()
    res = train(X, T, stats, iters=a.iters, batch=a.batch, lr=a.lr, log_every=max(1, a.iters // 8))
    t_train = time.perf_counter() - t
    apr = a_priori(res["params"], stats, Xh, Th, KCh)
    post = a_posteriori(res["params"], stats, n_fine=a.n_fine, factor=a.factor, t0=a.t0, coarse_steps=a.coarse_steps,
                        nu_fine=nu_fine)
    # C_nu calibrated per closure on a training seed (dissipation of its filtered
    # fine run), then both closures evaluated on the evaluation seed
    cal_ref = filtered_reference(a.n_fine, a.factor, 4.0, ints(a.train_seeds)[0], nu_fine, 0.04, a.t0, a.coarse_steps)
    cal = {cl: calibrate_c_nu(cl, cal_ref, res["params"], stats) for cl in ("kcmp", "learned")}
    ev_ref = filtered_reference(a.n_fine, a.factor, 4.0, 99, nu_fine, 0.04, a.t0, a.coarse_steps)
    calibrated = {"c_nu": cal, "evaluation_filtered_fine": {"E_k": ev_ref["E_k"], "dissipation": ev_ref["dissipation"]}}
    for cl in ("kcmp", "learned"):
        calibrated[cl] = coarse_run(cl, ev_ref, res["params"], stats, cal[cl])
    calibrated["bgk"] = coarse_run("bgk", ev_ref)
    # the learned closure at the C_nu its targets were built for
    calibrated["learned_at_target_c_nu"] = coarse_run("learned", ev_ref, res["params"], stats, a.c_nu)
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    np.savez(a.out, params=res["params"], stats=stats, n_fine=a.n_fine, factor=a.factor, nu_fine=nu_fine,
             nu_coarse=nu_fine / a.factor)
    # the same network in the library's file form (lbm_set_learned_closure_file)
    lbm.write_learned_closure(os.path.splitext(a.out)[0] + ".bin", res["params"], stats)
    nu_c = nu_fine / a.factor
    mlups = {}
    for n in ints(a.mlups_sizes):
        mlups[f"{n}^3"] = {cl: _mlups(cl, n, nu_c, res["params"], stats) for cl in ("kcmp", "learned")}
    out = {"samples_train": int(X.shape[0]), "samples_test": int(Xh.shape[0]), "t_data_s": t_data,
           "t_train_s": t_train, "loss_history": res["history"], "a_priori_heldout": apr, "a_posteriori": post,
           "a_posteriori_calibrated": calibrated,
           "mlups": mlups, "checkpoint": os.path.relpath(a.out, os.path.dirname(os.path.dirname(__file__))),
           "config": vars(a)}
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
