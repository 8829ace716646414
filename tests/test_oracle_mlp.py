"""Pins of the FP64 oracle network of the learned closure (no GPU): the
backward pass against central finite differences of the loss, the silu
derivative against its closed form, and the first AdamW step against its
textbook value lr * sign(g) (bias-corrected moments equal g and g^2).  Pins of
the learned step around the network: a zero network gives the BGK step, and a
network that returns the KC-MP carrier gives the KC-MP step (App. F.3)."""
import numpy as np
import pytest

from oracle import mlp


def _data(n=7, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 10)), rng.standard_normal((n, 6))


def test_param_count():
    assert mlp.NPARAM == 10 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 * 6 + 6 == 9414
    p = mlp.init_params(1)
    assert np.array_equal(mlp.flat(mlp.unflat(mlp.flat(p))), mlp.flat(p))


def test_silu_derivative_closed_form():
    a = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (mlp.silu(a + h) - mlp.silu(a - h)) / (2 * h)
    assert np.abs(mlp.silu_grad(a) - fd).max() < 1e-9
    assert mlp.silu(0.0) == 0.0 and mlp.silu_grad(0.0) == 0.5


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    p = mlp.init_params(seed)
    for k in p:  # non-zero biases so that their gradients are exercised
        if k.startswith("b"):
            p[k] = 0.1 * np.random.default_rng(seed + 5).standard_normal(p[k].shape)
    xs, ts = _data(seed=seed)
    g = mlp.backward(p, xs, ts)
    rng = np.random.default_rng(seed + 9)
    h = 1e-6
    for k in p:
        idx = [tuple(rng.integers(0, s) for s in p[k].shape) for _ in range(6)]
        for j in idx:
            old = p[k][j]
            p[k][j] = old + h
            lp = mlp.loss(p, xs, ts)
            p[k][j] = old - h
            lm = mlp.loss(p, xs, ts)
            p[k][j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k][j] - fd) <= 1e-7 * max(1.0, abs(fd)), (k, j, g[k][j], fd)


def test_first_adamw_step_is_lr_sign_g():
    p = mlp.init_params(3)
    xs, ts = _data(seed=3)
    g = mlp.backward(p, xs, ts)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    p0 = {k: val.copy() for k, val in p.items()}
    lr = 1e-3
    mlp.adamw_step(p, g, m, v, 1, lr, eps=1e-12, wd=0.0)
    for k in p:
        big = np.abs(g[k]) > 1e-6
        assert np.allclose((p0[k] - p[k])[big], lr * np.sign(g[k][big]), rtol=1e-5)


def test_weight_decay_is_decoupled():
    p = mlp.init_params(4)
    g = {k: np.zeros_like(v) for k, v in p.items()}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    p0 = {k: val.copy() for k, val in p.items()}
    mlp.adamw_step(p, g, m, v, 1, 0.01, wd=0.1)
    assert np.allclose(p["W2"], p0["W2"] * (1 - 0.01 * 0.1))
    assert np.array_equal(p["b2"], p0["b2"])


def test_training_reduces_loss():
    """A few hundred full-batch AdamW steps fit a smooth target (sanity of the
    whole loop)."""
    rng = np.random.default_rng(7)
    xs = rng.standard_normal((256, 10))
    ts = np.tanh(xs[:, :6] * 0.5 + 0.3 * xs[:, 6:7])
    p = mlp.init_params(7)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    l0 = mlp.loss(p, xs, ts)
    for t in range(1, 301):
        mlp.adamw_step(p, mlp.backward(p, xs, ts), m, v, t, 3e-3)
    assert mlp.loss(p, xs, ts) < 0.05 * l0


def test_bf16_rounding_emulation():
    """Round-to-nearest-even to bfloat16: exact values stay, ties go to even,
    the relative error is at most half an ulp (2^-8), and the values agree with
    torch's own float32 -> bfloat16 conversion."""
    from oracle.learned import bf16

    assert bf16(np.array([1.0, -2.5, 0.0]))[0] == 1.0
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: rounds to the even mantissa (1.0)
    assert bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    x = np.random.default_rng(0).standard_normal(10000)
    assert np.abs(bf16(x) / x - 1).max() <= 2.0 ** -8
    torch = pytest.importorskip("torch")
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    assert np.array_equal(bf16(x), ref)


def test_learned_step_with_zero_output_is_bgk():
    """With a network whose output is zero (zero weights and biases, zero output
    mean) m_sgs = 0, the turbulent rate is clipped to omega and the learned step
    is the resolved-BGK step (Sec. 5.1)."""
    import oracle
    from oracle import learned

    f = oracle.init_equilibrium(27, None, np.full((3, 4, 4, 4), 0.02))
    params = np.zeros(mlp.NPARAM)
    stats = np.concatenate([np.zeros(10), np.ones(10), np.zeros(6), np.ones(6)])
    fpost, msgs = learned.step(f, 1e-4, params, stats, 0.035)
    assert np.abs(msgs).max() == 0.0
    ref = oracle.run(f, 1, closure=0, nu=1e-4)
    assert np.abs(fpost - ref).max() < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_learned_step_with_carrier_output_is_kcmp(q, monkeypatch):
    """A network that returns the KC-MP carrier itself (its first six inputs,
    de-standardised with the input statistics) makes m_sgs = m_neq - m_CE, so
    the learned step must be the KC-MP step of the C oracle (App. F.3).  This
    ties the learned step's carrier inputs, its m_sgs -> f_sgs projection, the
    rate clip and the two-rate relaxation to the pinned analytic closure.  The
    remaining inputs (invariants of m_CE / rho, tau_hat) equal those of the
    training-data features of the same streamed state, which are pinned on
    their own."""
    import oracle
    from oracle import closure_data as cd
    from oracle import learned
    from paper_2605_19796_gb300 import inputs

    nu, c_nu = 1e-5, 0.035
    rho, u = inputs.hit_fields(0, k0=2.0, urms=0.08, seed=4, shape=(8, 6, 5))
    f = oracle.run(oracle.init_equilibrium(q, rho, u), 3, closure=1, nu=nu, c_nu=c_nu)
    rng = np.random.default_rng(9)
    xmu, xsd = 1e-3 * rng.standard_normal(10), rng.uniform(0.5, 2.0, 10)
    stats = np.concatenate([xmu, xsd, xmu[:6], xsd[:6]])
    monkeypatch.setattr(learned, "forward", lambda params, xs, rounding: xs[:, :6].copy())
    fpost, msgs = learned.step(f, nu, np.zeros(mlp.NPARAM), stats, c_nu)
    ref = oracle.run(f, 1, closure=1, nu=nu, c_nu=c_nu)
    assert np.abs(fpost - ref).max() <= 1e-14 * np.abs(ref).max()
    # the SGS rate is active in a good share of the cells, so the check has teeth
    tr = msgs[:, 0] + msgs[:, 1] + msgs[:, 2]
    assert np.mean(c_nu * np.sqrt(np.abs(tr) / 2) > nu) > 0.3
    bgk = oracle.run(f, 1, closure=0, nu=nu)
    assert np.abs(ref - bgk).max() > 1e3 * 1e-14 * np.abs(ref).max()
    x = learned.inputs_and_state(f, nu)[4]
    xf, _ = cd.features(cd.stream(f), nu)
    assert np.abs(x - xf).max() <= 1e-15 * max(1.0, np.abs(xf).max())
