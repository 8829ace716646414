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
