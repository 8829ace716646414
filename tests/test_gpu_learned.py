"""GPU checks of the learned closure's training-side kernels against the FP64
oracle (oracle/mlp.py, oracle/closure_data.py), through the C ABI.

Tolerances: FP32 kernels against FP64 references: forward outputs and loss
1e-5 relative, parameter gradients 1e-4 relative to the largest entry of each
layer's gradient (sums of up to ~300 FP32 products), one AdamW step 1e-6
absolute on the parameters; box filter and features 1e-5 relative to each
quantity's scale (FP32 outputs of FP64 arithmetic)."""
import numpy as np
import pytest

from paper_2605_19796_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_19796_gb300 import build

    build.build()
    from paper_2605_19796_gb300 import lbm

    return lbm, torch


def _params(seed):
    from oracle import mlp

    p = mlp.init_params(seed)
    rng = np.random.default_rng(seed + 11)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    return p


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


@pytest.mark.parametrize("n", [1, 37, 300])
def test_mlp_forward_and_gradients(env, n):
    lbm, torch = env
    from oracle import mlp

    assert lbm.lbm_mlp_param_count() == mlp.NPARAM
    p = _params(n)
    rng = np.random.default_rng(n)
    xs, ts = rng.standard_normal((n, 10)), rng.standard_normal((n, 6))
    pd = _dev(torch, mlp.flat(p))
    xd, td = _dev(torch, xs), _dev(torch, ts)
    ws = torch.zeros(lbm.lbm_mlp_workspace_floats(n), dtype=torch.float32, device="cuda")
    ys = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    lbm.lbm_mlp_forward(pd.data_ptr(), xd.data_ptr(), n, ys.data_ptr(), ws.data_ptr())
    yref, _ = mlp.forward(p, xs)
    assert np.abs(ys.cpu().numpy() - yref).max() <= 1e-5 * max(1.0, np.abs(yref).max())
    g = torch.zeros(mlp.NPARAM, dtype=torch.float32, device="cuda")
    loss = lbm.lbm_mlp_grad(pd.data_ptr(), xd.data_ptr(), td.data_ptr(), n, g.data_ptr(), ws.data_ptr())
    assert loss == pytest.approx(mlp.loss(p, xs, ts), rel=1e-5)
    gref = mlp.backward(p, xs, ts)
    gg = mlp.unflat(g.cpu().numpy().astype(np.float64))
    for k in gref:
        scale = np.abs(gref[k]).max()
        assert np.abs(gg[k] - gref[k]).max() <= 1e-4 * scale + 1e-9, k


def test_adamw_step(env):
    lbm, torch = env
    from oracle import mlp

    p = _params(3)
    rng = np.random.default_rng(3)
    g = {k: rng.standard_normal(v.shape) * 1e-2 for k, v in p.items()}
    m = {k: rng.standard_normal(v.shape) * 1e-3 for k, v in p.items()}
    v = {k: np.abs(rng.standard_normal(v.shape)) * 1e-4 for k, v in p.items()}
    pd, gd, md, vd = (_dev(torch, mlp.flat(x)) for x in (p, g, m, v))
    lbm.lbm_mlp_adamw(pd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), 5, 1e-3, weight_decay=0.01)
    torch.cuda.synchronize()
    mlp.adamw_step(p, g, m, v, 5, 1e-3, wd=0.01)
    assert np.abs(pd.cpu().numpy() - mlp.flat(p)).max() < 1e-6
    assert np.abs(md.cpu().numpy() - mlp.flat(m)).max() < 1e-7


@pytest.mark.parametrize("q", [19, 27])
def test_closure_strain_matches_oracle(env, orc, q):
    """lbm_closure_strain (the strain the dissipation target is built from)
    against the oracle's strain (App. F.1 step 3) of the same FP32 populations'
    velocity, on a ragged periodic box.  Tolerance: the kernel sums in FP32
    (velocity rounding about 1e-7 of |u| <= 0.1, halved by the central
    difference), 5e-7 absolute."""
    lbm, torch = env
    shape = (16, 9, 12)
    nx, ny, nz = shape
    rho, u = inputs.hit_fields(0, k0=2.0, urms=0.06, seed=17, shape=shape)
    rng = np.random.default_rng(7)
    f = orc.init_equilibrium(q, rho, u) * (1 + 1e-3 * rng.standard_normal((q, nz, ny, nx)))
    f32 = f.astype(np.float32)
    fd = torch.from_numpy(np.ascontiguousarray(f32)).cuda()
    out = torch.full((nx * ny * nz, 6), float("nan"), dtype=torch.float32, device="cuda")
    lbm.lbm_closure_strain(fd.data_ptr(), q, nx, ny, nz, out.data_ptr())
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    _, uo = orc.fields(f32.astype(np.float64))
    S = orc.strain_field(uo)
    want = np.stack([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]], axis=-1).reshape(-1, 6)
    assert np.abs(want).max() > 1e-3
    assert np.abs(got - want).max() <= 5e-7, np.abs(got - want).max()


@pytest.mark.parametrize("q", [19, 27])
def test_box_filter_and_features(env, orc, q):
    lbm, torch = env
    from oracle import closure_data as cd

    shape = (16, 8, 12)
    rho, u = inputs.hit_fields(0, k0=2.0, urms=0.06, seed=4, shape=shape)
    f = orc.run(orc.init_equilibrium(q, rho, u), 3, closure=1, nu=1e-4, c_nu=0.035)
    fb_ref, msgs_ref = cd.filtered_state(f, 4)
    nxc, nyc, nzc = 4, 2, 3
    fd = torch.as_tensor(f, device="cuda")  # FP64 storage layout [q][z][y][x]
    fc = torch.zeros((q, nzc, nyc, nxc), dtype=torch.float32, device="cuda")
    ms = torch.zeros((6, nzc, nyc, nxc), dtype=torch.float32, device="cuda")
    lbm.lbm_box_filter(fd.data_ptr(), q, lbm.LBM_FP64, 16, 8, 12, 4, fc.data_ptr(), ms.data_ptr())
    torch.cuda.synchronize()
    assert np.abs(fc.cpu().numpy() - fb_ref).max() <= 1e-7
    assert np.abs(ms.cpu().numpy() - msgs_ref).max() <= 1e-5 * np.abs(msgs_ref).max()
    # consistent coarse state: the fine non-equilibrium part rescaled by r
    fb_r, _ = cd.filtered_state(f, 4, neq_scale=3.7)
    lbm.lbm_box_filter(fd.data_ptr(), q, lbm.LBM_FP64, 16, 8, 12, 4, fc.data_ptr(), ms.data_ptr(), neq_scale=3.7)
    torch.cuda.synchronize()
    assert np.abs(fc.cpu().numpy() - fb_r).max() <= 1e-7
    assert np.abs(fb_r - fb_ref).max() > 1e-5, "the rescaling must act on this state"
    with pytest.raises(lbm.LbmError):
        lbm.lbm_box_filter(fd.data_ptr(), q, lbm.LBM_FP64, 16, 8, 12, 4, fc.data_ptr(), ms.data_ptr(), neq_scale=0.0)
    # the streamed (pre-collision) state, rescaled
    fb_p, ms_p = cd.filtered_state(f, 4, neq_scale=3.7, pull=True)
    lbm.lbm_box_filter(fd.data_ptr(), q, lbm.LBM_FP64, 16, 8, 12, 4, fc.data_ptr(), ms.data_ptr(), neq_scale=3.7,
                       pull=True)
    torch.cuda.synchronize()
    assert np.abs(fc.cpu().numpy() - fb_p).max() <= 1e-7
    assert np.abs(ms.cpu().numpy() - ms_p).max() <= 1e-5 * np.abs(ms_p).max()
    # features of a coarse-sized state (use the fine field itself as a periodic lattice)
    f32 = torch.as_tensor(f.astype(np.float32), device="cuda")
    N = 16 * 8 * 12
    x = torch.zeros((N, 10), dtype=torch.float32, device="cuda")
    t = torch.zeros((N, 6), dtype=torch.float32, device="cuda")
    mfine = torch.as_tensor(np.random.default_rng(1).standard_normal((6, 12, 8, 16)).astype(np.float32) * 1e-4,
                            device="cuda")
    lbm.lbm_closure_features(f32.data_ptr(), q, 16, 8, 12, 2.5e-5, mfine.data_ptr(), x.data_ptr(), t.data_ptr())
    torch.cuda.synchronize()
    xr, rr = cd.features(f.astype(np.float32).astype(np.float64), 2.5e-5)
    xg = x.cpu().numpy()
    for k in range(10):
        sc = np.abs(xr[:, k]).max()
        assert np.abs(xg[:, k] - xr[:, k]).max() <= 1e-4 * sc + 1e-12, k
    tr = cd.targets(mfine.cpu().numpy().astype(np.float64), rr)
    assert np.abs(t.cpu().numpy() - tr).max() <= 1e-6 * np.abs(tr).max()


# BF16 rounding (8 significand bits, round to nearest): the relative error of
# one rounding is at most 2^-8, and uniformly spread over that interval its
# standard deviation is 2^-8 / sqrt(3)
SIG_BF16 = 2.0 ** -8 / np.sqrt(3.0)
# the fused SiLU h + h tanh(h), h = a/2, on the hardware tanh (relative error
# about 2^-11): standard deviation allowance 2^-11 / sqrt(3) of |h|
SIG_TANH = 2.0 ** -11 / np.sqrt(3.0)
N_SIGMA = 6.0


def bf16_output_bound(p, xs):
    """Bound on |network(xs) on BF16 tensor cores - the FP64 network| per sample
    and output (standardised units), N_SIGMA standard deviations of the
    accumulated rounding error: the inputs, the weights and each hidden
    activation rounded to BF16 (independent, zero-mean errors of standard
    deviation 2^-8/sqrt(3) relative), propagated to first order through the
    four layers (variances weighted by W^2, SiLU by its derivative at the FP64
    pre-activation), plus the hardware-tanh allowance; FP32 accumulation is
    negligible.  The componentwise worst case (absolute row sums) grows about
    fourfold per layer and exceeds the outputs themselves, so it bounds nothing
    useful; the errors are independent sums, whose spread is what this tracks."""
    from oracle import mlp

    W2 = {k: v * v for k, v in p.items() if k.startswith("W")}
    h = xs
    var = (SIG_BF16 * xs) ** 2
    for l in range(1, 4):
        a = h @ p[f"W{l}"].T + p[f"b{l}"]
        var_a = var @ W2[f"W{l}"].T + SIG_BF16 ** 2 * ((h * h) @ W2[f"W{l}"].T)
        h = mlp.silu(a)
        var = mlp.silu_grad(a) ** 2 * var_a + (SIG_BF16 * h) ** 2 + (SIG_TANH * a / 2) ** 2
    var_y = var @ W2["W4"].T + SIG_BF16 ** 2 * ((h * h) @ W2["W4"].T)
    return N_SIGMA * np.sqrt(var_y)


def test_tensor_core_forward_matches(env):
    """The fused inference's tensor-core network (BF16 mma.sync, FP32 accumulate)
    against the unrounded FP64 network within the BF16 rounding error
    propagated through the four layers (bf16_output_bound: six standard
    deviations), and against the FP64 oracle
    network with the same BF16 rounding points (a hidden activation may round to
    the neighbouring BF16 value where FP32 and FP64 sums straddle a rounding
    boundary: 99 % of the outputs within 2e-3 of the output scale)."""
    lbm, torch = env
    from oracle import learned as olearned
    from oracle import mlp

    n = 1000
    rng = np.random.default_rng(8)
    x = rng.standard_normal((n, 10)) * 1e-3 + 2e-4
    x[:, 9] = 0.5
    stats = np.concatenate([x.mean(0), np.where(x.std(0) > 1e-6 * np.abs(x.mean(0)), x.std(0), 1.0), np.full(6, 1e-5),
                            np.full(6, 3e-4)]).astype(np.float32)
    params = np.asarray(mlp.flat(_params(9)), dtype=np.float32)
    packed = torch.as_tensor(lbm.lbm_mlp_pack(params, stats), device="cuda")
    xd = torch.as_tensor(x.astype(np.float32), device="cuda")
    yd = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    lbm.lbm_mlp_forward_tc(packed.data_ptr(), xd.data_ptr(), n, yd.data_ptr())
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    st = stats.astype(np.float64)
    xs = (x.astype(np.float32).astype(np.float64) - st[:10]) / st[10:20]
    p64 = mlp.unflat(params.astype(np.float64))
    yu = olearned.forward(params.astype(np.float64), xs, rounding=False) * st[26:32] + st[20:26]
    bound = bf16_output_bound(p64, xs) * st[26:32]
    assert np.all(np.abs(y - yu) <= bound), np.max(np.abs(y - yu) / bound)
    yo = olearned.forward(params.astype(np.float64), xs, rounding=True) * st[26:32] + st[20:26]
    scale = np.abs(yo - st[20:26]).max()
    assert np.percentile(np.abs(y - yo), 99) <= 2e-3 * scale


def _stats_for(x, scale_out):
    xm, xs = x.mean(0), x.std(0)
    xs = np.where(xs > 1e-6 * np.abs(xm), xs, 1.0)  # tau_hat: constant up to rounding
    return np.concatenate([xm, xs, np.zeros(6), np.full(6, scale_out)]).astype(np.float32)


@pytest.mark.parametrize("q,variant,tile_y", [(27, 1, 8), (27, 8, 8), (27, 12, 8), (27, 1, 4), (27, 12, 4),
                                              (27, 14, 16), (27, 15, 4), (19, 1, 4), (19, 8, 8), (19, 15, 4)])
def test_learned_step_matches_oracle(env, orc, q, variant, tile_y):
    """One step of the fused learned closure (BF16 tensor-core network inside the
    step kernel: the register pull, variant 1, the split-barrier kernel,
    variant 8, and the same with L2 prefetches, variant 12; tiles of 8 rows and
    4, where the register pull evaluates the network for both 16-cell halves of
    a warp together; the four-cell kernel, variant 14, on 64 x 16 tiles, whose
    warps run the network once per cell slot; the register pull with the
    network on the tcgen05 tensor cores, variant 15, one 128-row GEMM per
    layer with its accumulators in tensor memory; D3Q27 and D3Q19)
    against the oracle's learned step with the same BF16 rounding
    points (inputs, weights, hidden activations) and FP64 elsewhere.  The network
    is random, its output scaled so that the turbulent rate is active in most
    cells.  The z-chunk of 5 planes leaves a ragged last chunk.

    Tolerance: the state is stored in FP32, so the resolved part of the update
    carries FP32 rounding noise; it is measured on the same state by the BGK
    and KC-MP steps against the oracle's (the learned closure has KC-MP's
    relaxation form), the larger of the two.  Each cell may differ from the oracle by
    twice that noise plus 2^-7 of its SGS increment (omega - omega_s) f_sgs, the
    BF16 network's share."""
    lbm, torch = env
    from oracle import learned as olearned
    from oracle import mlp

    shape = (32, 16, 12)
    nu = 2e-5
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.08, seed=12, shape=shape)
    f = orc.run(orc.init_equilibrium(q, rho, u), 4, closure=1, nu=nu, c_nu=0.035)
    f = f.astype(np.float32).astype(np.float64)  # the GPU state is FP32
    _, _, _, _, x = olearned.inputs_and_state(f, nu)
    scale = 5.0 * float(np.abs(x[:, :6]).std())
    stats = _stats_for(x, scale)
    params = np.asarray(mlp.flat(mlp.init_params(5)), dtype=np.float32)
    with lbm.Solver(q, shape, nu, closure="learned", storage="fp32", variant=variant, tile_y=tile_y, zchunk=5) as s:
        assert s.launch_config["variant"] == variant and s.launch_config["tile_y"] == tile_y
        s.set_learned_closure(params, stats)
        s.set_populations(f)
        s.step(1)
        fg = s.get_populations()
    with lbm.Solver(q, shape, nu, closure="bgk", storage="fp32") as s:
        s.set_populations(f)
        s.step(1)
        fb = s.get_populations()
    with lbm.Solver(q, shape, nu, closure="kcmp", storage="fp32") as s:
        s.set_populations(f)
        s.step(1)
        fk = s.get_populations()
    fo, msgs = olearned.step(f, nu, params.astype(np.float64), stats.astype(np.float64), 0.035)
    fbo = orc.run(f, 1, closure=0, nu=nu)
    fko = orc.run(f, 1, closure=1, nu=nu, c_nu=0.035)
    # the closure must be active: nu_t > nu in a good share of the cells
    tr = msgs[:, 0] + msgs[:, 1] + msgs[:, 2]
    assert np.mean(0.035 * np.sqrt(np.abs(tr) / 2) > nu) > 0.5
    # FP32 noise of the same relaxation form (BGK, and KC-MP whose D H term the
    # learned closure shares), measured on this state
    noise = max(np.abs(fb - fbo).max(), np.abs(fk - fko).max())
    assert noise < 1e-7
    sgs = np.abs(fo - fbo).reshape(q, -1).max(axis=0)  # per cell SGS increment
    assert sgs.max() > 100 * noise, "the SGS signal must stand well above the FP32 noise"
    err = np.abs(fg - fo).reshape(q, -1).max(axis=0)
    bound = 2 * noise + 2.0 ** -7 * sgs
    assert np.all(err <= bound), (np.max(err / bound), noise, sgs.max())
    # the SGS increments themselves, globally
    inc = np.abs((fg - fb) - (fo - fbo)).max()
    assert inc <= 4 * noise + 1e-2 * sgs.max(), (inc, noise, sgs.max())


@pytest.mark.parametrize("q,variant,tile_y", [(27, 1, 4), (19, 1, 4), (27, 12, 8), (27, 14, 16), (27, 15, 4),
                                              (19, 15, 4)])
def test_learned_step_matches_unrounded_network(env, orc, q, variant, tile_y):
    """One step of the fused learned closure against the oracle's learned step
    with the UNROUNDED FP64 network (oracle/learned.py, rounding=False).  Bound
    per cell: twice the FP32 noise of the same relaxation form (as in
    test_learned_step_matches_oracle) plus the effect of the network error
    allowed by bf16_output_bound: dm = rho sd_y dy enters f_sgs = w/(2 theta^2)
    (H : m) linearly, |d f_sgs_i| <= w_i/(2 theta^2) sum_ab |c_a c_b - theta
    delta_ab| |dm_ab|, and the clipped rate through tr m; omega_s is monotone in
    |tr m|, so its change is bounded by its values at |tr| -+ |d tr|; then
    |d f_post| <= (omega - omega_s) |d f_sgs| + d omega_s (|f_sgs| + |d f_sgs|)."""
    lbm, torch = env
    from oracle import learned as olearned
    from oracle import mlp

    shape = (32, 16, 12)
    nu, c_nu = 2e-5, 0.035
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.08, seed=12, shape=shape)
    f = orc.run(orc.init_equilibrium(q, rho, u), 4, closure=1, nu=nu, c_nu=c_nu)
    f = f.astype(np.float32).astype(np.float64)
    _, rho_p, _, _, x = olearned.inputs_and_state(f, nu)
    scale = 5.0 * float(np.abs(x[:, :6]).std())
    stats = _stats_for(x, scale)
    params = np.asarray(mlp.flat(mlp.init_params(5)), dtype=np.float32)
    with lbm.Solver(q, shape, nu, closure="learned", storage="fp32", variant=variant, tile_y=tile_y, zchunk=5) as s:
        s.set_learned_closure(params, stats)
        s.set_populations(f)
        s.step(1)
        fg = s.get_populations()
    with lbm.Solver(q, shape, nu, closure="bgk", storage="fp32") as s:
        s.set_populations(f)
        s.step(1)
        fb = s.get_populations()
    with lbm.Solver(q, shape, nu, closure="kcmp", storage="fp32") as s:
        s.set_populations(f)
        s.step(1)
        fk = s.get_populations()
    fbo = orc.run(f, 1, closure=0, nu=nu)
    fko = orc.run(f, 1, closure=1, nu=nu, c_nu=c_nu)
    noise = max(np.abs(fb - fbo).max(), np.abs(fk - fko).max())
    fo, msgs = olearned.step(f, nu, params.astype(np.float64), stats.astype(np.float64), c_nu, rounding=False)
    st = stats.astype(np.float64)
    xs = (x.astype(np.float32).astype(np.float64) - st[:10]) / st[10:20]
    dy = bf16_output_bound(mlp.unflat(params.astype(np.float64)), xs)
    dm = rho_p.ravel()[:, None] * st[26:32] * dy  # [N, 6], xx yy zz xy xz yz
    c, w, _ = orc.lattice(q)
    cf = c.astype(float)
    TH = 1.0 / 3.0
    comp = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    Habs = np.zeros((q, 6))
    for k, (a, b) in enumerate(comp):
        Habs[:, k] = np.abs(cf[:, a] * cf[:, b] - (TH if a == b else 0.0)) * (1 if a == b else 2)
    dfs = (w[:, None] / (2 * TH ** 2)) * (Habs @ dm.T)  # [q, N]
    tr = msgs[:, 0] + msgs[:, 1] + msgs[:, 2]
    dtr = dm[:, 0] + dm[:, 1] + dm[:, 2]
    omega = 1.0 / (nu / TH + 0.5)

    def rate(t):
        nut = c_nu * np.sqrt(np.abs(t) / 2.0)
        return np.where(nut > nu, 1.0 / (nut / TH + 0.5), omega)

    om_s = rate(tr)
    dom = np.maximum(np.abs(rate(np.abs(tr) + dtr) - om_s), np.abs(rate(np.maximum(np.abs(tr) - dtr, 0.0)) - om_s))
    M = np.zeros((3, 3, tr.size))
    for k, (a, b) in enumerate(comp):
        M[a, b] = msgs[:, k]
        M[b, a] = msgs[:, k]
    fsgs = (w[:, None] / (2 * TH ** 2)) * (np.einsum("ia,ib,abn->in", cf, cf, M) - TH * tr[None, :])
    bound = 2 * noise + (omega - om_s)[None, :] * dfs + dom[None, :] * (np.abs(fsgs) + dfs)
    err = np.abs(fg - fo).reshape(q, -1)
    assert np.mean(om_s < omega) > 0.5, "the closure must be active"
    assert np.all(err <= bound), (np.max(err / bound), noise)


@pytest.mark.parametrize("variant,tile_y", [(14, 16), (1, 4), (15, 4)])
def test_learned_full_size_sampled_cells(env, orc, variant, tile_y):
    """The learned closure at 256^3 (D3Q27, FP32, decaying HIT, nu = 2.5e-5) in
    its default launch (the register pull on 4-row tiles with the network on
    the tcgen05 tensor cores, variant 15), with mma.sync fragments (variant 1)
    and in the four-cell kernel on 64 x 16 tiles, each with its default
    z-chunk: one GPU step, then sampled cells against the
    oracle's learned step of the periodic 5x5x5 block around each cell, cut from
    the GPU's own pre-step populations (the centre's pulls and the strain at its
    six neighbours stay inside the block, so the centre is exact).  Random
    network as in the small-box test, standardised on the sampled cells' own
    inputs.  Tolerance per cell: 2e-6 x max|f| (the FP32 bound of the KC-MP
    full-size test) plus 2^-7 of the cell's SGS increment against the BGK step
    (the BF16 network's share)."""
    lbm, torch = env
    from oracle import learned as olearned
    from oracle import mlp

    n, nu, c_nu = 256, 2.5e-5, 0.035
    rho, u = inputs.hit_fields(n, k0=4.0, urms=0.04, seed=3)
    rng = np.random.default_rng(2562)
    pts = np.concatenate([rng.integers(0, n, size=(40, 3)),
                          [[0, 0, 0], [n - 1, n - 1, n - 1], [31, 3, 15], [32, 4, 16], [n - 1, 0, n // 2]]])
    offs = np.array([(dx, dy, dz) for dz in range(-2, 3) for dy in range(-2, 3) for dx in range(-2, 3)])
    centre = 62  # (2, 2, 2) of the block
    params = np.asarray(mlp.flat(mlp.init_params(5)), dtype=np.float32)
    with lbm.Solver(27, (n, n, n), nu, closure="learned", storage="fp32", c_nu=c_nu, variant=variant,
                    tile_y=tile_y) as s:
        cfg = s.launch_config
        assert cfg["variant"] == variant and cfg["tile_y"] == tile_y, cfg
        s.init_velocity(rho, u)
        del rho, u
        s.set_learned_closure(params, _stats_for(np.ones((2, 10)), 1.0))
        s.step(3)
        blocks = s.probe((pts[:, None, :] + offs[None, :, :]).reshape(-1, 3)).reshape(len(pts), 125, 27)
        blks = [blocks[k].T.reshape(27, 5, 5, 5).astype(np.float64) for k in range(len(pts))]
        x = np.stack([olearned.inputs_and_state(b, nu)[4][centre] for b in blks])
        stats = _stats_for(x, 5.0 * float(np.abs(x[:, :6]).std()))
        s.set_learned_closure(params, stats)
        s.step(1)
        after = s.probe(pts)
    scale = np.abs(after).max()
    p64, st64 = params.astype(np.float64), stats.astype(np.float64)
    active = 0
    for k, b in enumerate(blks):
        fo, msgs = olearned.step(b, nu, p64, st64, c_nu)
        fbo = orc.step_cell(b, closure=0, nu=nu, c_nu=c_nu)
        ref = fo[:, 2, 2, 2]
        sgs = np.abs(ref - fbo).max()
        tr = msgs[centre, 0] + msgs[centre, 1] + msgs[centre, 2]
        active += c_nu * np.sqrt(abs(tr) / 2) > nu
        err = np.abs(after[k] - ref).max()
        assert err <= 2e-6 * scale + 2.0 ** -7 * sgs, (pts[k], err, sgs)
    assert active > len(pts) // 2, active


def test_learned_closure_from_file_equals_arrays(env, tmp_path):
    """lbm_set_learned_closure_file installs the same network as
    lbm_set_learned_closure with the arrays the file holds: one step from the
    same state gives bitwise equal populations."""
    lbm, torch = env
    from oracle import mlp

    shape = (32, 16, 12)
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.05, seed=21, shape=shape)
    params = np.asarray(mlp.flat(mlp.init_params(8)), dtype=np.float32)
    stats = _stats_for(np.random.default_rng(2).standard_normal((64, 10)), 1e-3)
    path = str(tmp_path / "net.bin")
    lbm.write_learned_closure(path, params, stats)
    out = []
    for from_file in (False, True):
        with lbm.Solver(27, shape, 2e-5, closure="learned", storage="fp32") as s:
            s.init_velocity(rho, u)
            if from_file:
                s.set_learned_closure_file(path)
            else:
                s.set_learned_closure(params, stats)
            s.step(2)
            out.append(s.get_populations())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("storage,launch", [("fp16", {}), ("bf16", {}), ("fp16", {"variant": 14, "tile_y": 8}),
                                            ("bf16", {"variant": 14, "tile_y": 16}),
                                            ("fp16", {"variant": 1, "tile_y": 4})])
def test_learned_step_16bit_storage(env, orc, storage, launch):
    """The learned closure on weight-shifted 16-bit storage (its default launch,
    the register pull on 4-row tiles with the tcgen05 network; the same with
    mma.sync fragments; the four-cell kernel on 128 x 8 tiles, which 16-bit
    staging leaves room for, and on 64 x 16 tiles): one step
    from a state that FP16/BF16 hold exactly gives the density and velocity of
    the same step on FP32 storage within the rounding of the stored results: 8
    units of the format's relative spacing (2^-10 FP16, 2^-7 BF16) times
    max |f - w|, the bound the load-schedule tests use."""
    lbm, torch = env
    from oracle import learned as olearned
    from oracle import mlp

    shape = (32, 16, 12)
    nu = 2e-5
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.08, seed=12, shape=shape)
    f = orc.run(orc.init_equilibrium(27, rho, u), 4, closure=1, nu=nu, c_nu=0.035)
    w = orc.lattice(27)[1][:, None, None, None]
    # a state the 16-bit storage holds exactly: round g = f - w to the format
    gt = torch.from_numpy(np.ascontiguousarray(f - w, dtype=np.float32))
    gt = gt.to(torch.float16 if storage == "fp16" else torch.bfloat16).to(torch.float64).numpy()
    f16 = w + gt
    _, _, _, _, x = olearned.inputs_and_state(f16, nu)
    stats = _stats_for(x, 5.0 * float(np.abs(x[:, :6]).std()))
    params = np.asarray(mlp.flat(mlp.init_params(5)), dtype=np.float32)
    out = {}
    for st in ("fp32", storage):
        kw = launch if st == storage else {}
        with lbm.Solver(27, shape, nu, closure="learned", storage=st, **kw) as s:
            for k, v in kw.items():
                assert s.launch_config[k] == v
            s.set_learned_closure(params, stats)
            s.set_populations(f16)
            s.step(1)
            out[st] = s.get_populations()
    gmax = np.abs(out["fp32"] - w).max()
    tol = 8 * (2.0 ** -10 if storage == "fp16" else 2.0 ** -7) * gmax
    r1, u1 = orc.fields(out["fp32"])
    r2, u2 = orc.fields(out[storage])
    assert np.abs(r2 - r1).max() < tol and np.abs(u2 - u1).max() < tol, (np.abs(u2 - u1).max(), tol)


def test_learned_closure_pipeline(env):
    """Reduced end-to-end run of the learned closure: fine 128^3 runs box-filtered
    by 4 to 32^3, training with the library's kernels, held-out a-priori errors
    (the network must beat the analytic KC-MP estimate of m_sgs and the mean),
    and a stable coarse run with the fused network."""
    lbm, torch = env
    from paper_2605_19796_gb300 import learned

    X, T, KC = learned.generate(n_fine=128, factor=4, seeds=(0, 1, 2), k0s=(4.0,), snap_steps=(150, 300), keep=1.0)
    n = X.shape[0]
    ntr = (2 * n) // 3  # seeds 0, 1 train; seed 2 held out
    stats = learned.standardisation(X[:ntr], T[:ntr])
    res = learned.train(X[:ntr], T[:ntr], stats, iters=1500, batch=4096, lr=2e-3, log_every=500)
    m = learned.a_priori(res["params"], stats, X[ntr:], T[ntr:], KC[ntr:])
    print("a priori (held-out seed):", m)
    assert m["rel_mse_network"] < m["rel_mse_kcmp"]
    assert m["rel_mse_network"] < 1.0
    post = learned.a_posteriori(res["params"], stats, n_fine=128, factor=4, t0=150, coarse_steps=40, seed=7)
    print("a posteriori:", post)
    for cl in ("kcmp", "learned", "bgk"):
        assert np.isfinite(post[cl]["E_k"]) and post[cl]["E_k"] > 0


def test_learned_closure_gain_a_posteriori(env):
    """What the trained network gains over the method without it, a posteriori
    (reduced case: fine 128^3 KC-MP runs, seeds 0 and 1, box-filtered by 4 to
    32^3; 40 coarse steps from the filtered state at fine step 150, evaluation
    seed 7; C_nu calibrated per closure on seed 0 so that the coarse run
    dissipates as the filtered fine run, bisection in [1e-3, 0.5]).  Measured
    on a GB300 (spectrum = E(k) relative L2 error over shells 1..15,
    dissipation against the filtered fine run's 5.82e-6):

      BGK                              6.77 %   -27 %
      KC-MP, C_nu = 0.035              4.91 %   +21 %
      KC-MP, calibrated 0.023          4.94 %    +6 %
      learned (exact m_sgs), 0.035     6.71 %   -27 %
      learned (exact m_sgs), cal. 0.5  6.03 %   -18 %
      learned (dissipation target),
        cal. 0.5                       5.22 %   -12 %

    The outcome asserted: the network trained on the exact SGS stress gains
    nothing at the paper's C_nu (it dissipates as BGK, within 3 %: its trace is
    small at this resolution, so the rate stays clipped) and stays behind
    calibrated KC-MP in spectrum and dissipation even at the largest C_nu; the
    dissipation-carrying target (trace from the local SGS transfer, nu* clipped
    at its 90th percentile) recovers part of the missing dissipation and of the
    spectrum error but still loses to calibrated KC-MP.  The analytic closure
    is the fallback and the judge, as intended."""
    lbm, torch = env
    from paper_2605_19796_gb300 import learned

    n_fine, factor, nu_f, c_nu = 128, 4, 1e-4, 0.035
    cal_ref = learned.filtered_reference(n_fine, factor, 4.0, 0, nu_f, 0.04, 150, 40)
    ev_ref = learned.filtered_reference(n_fine, factor, 4.0, 7, nu_f, 0.04, 150, 40)
    target_diss = ev_ref["dissipation"]
    res = {}
    nets = {}
    for target in ("exact", "dissipation"):
        X, T, KC = learned.generate(n_fine, factor, seeds=(0, 1), k0s=(4.0,), snap_steps=(150, 300), keep=1.0,
                                    target=target, c_nu=c_nu, cap_quantile=0.9)
        stats = learned.standardisation(X, T)
        tr = learned.train(X, T, stats, iters=1500, batch=4096, lr=2e-3)
        nets[target] = (tr["params"], stats)
        cn = learned.calibrate_c_nu("learned", cal_ref, tr["params"], stats)
        res[target + "_cal"] = learned.coarse_run("learned", ev_ref, tr["params"], stats, cn)
        res[target + "_cal"]["c_nu"] = cn
    res["exact_default"] = learned.coarse_run("learned", ev_ref, *nets["exact"], c_nu)
    ck = learned.calibrate_c_nu("kcmp", cal_ref)
    res["kcmp_cal"] = learned.coarse_run("kcmp", ev_ref, c_nu=ck)
    res["kcmp_cal"]["c_nu"] = ck
    res["bgk"] = learned.coarse_run("bgk", ev_ref)
    print({k: v for k, v in res.items()}, "filtered fine dissipation", target_diss)
    derr = {k: abs(v["dissipation"] - target_diss) / target_diss for k, v in res.items()}
    spec = {k: v["spectrum_rel_l2"] for k, v in res.items()}
    assert all(np.isfinite(list(spec.values())))
    # the exact-target network at the paper's C_nu dissipates as BGK
    assert abs(res["exact_default"]["dissipation"] - res["bgk"]["dissipation"]) <= 0.03 * res["bgk"]["dissipation"]
    # calibrated KC-MP wins on both measures against either network
    for t in ("exact_cal", "dissipation_cal"):
        assert spec["kcmp_cal"] < spec[t], (t, spec)
        assert derr["kcmp_cal"] < derr[t], (t, derr)
    # the dissipation target moves the network towards the filtered run
    assert res["dissipation_cal"]["dissipation"] > res["exact_cal"]["dissipation"]
    assert spec["dissipation_cal"] < spec["exact_cal"]
