"""The dissipation-carrying training target (paper_2605_19796_gb300.learned.
dissipation_targets), checked on the CPU against what its definition fixes:
for an eddy-viscosity stress T = 2 k/3 I - 2 nu_e S (trace-free S) the SGS
energy transfer is -T : S = 2 nu_e S:S, so the target's rate must give back
nu_e, i.e. its trace is 2 (nu_e / (C_nu Delta))^2, with the deviatoric part
-2 nu_e S unchanged; backscatter (negative transfer) gives a zero trace; a
zero strain gives a zero trace."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _sym(rng, n):
    S = rng.standard_normal((n, 6)) * 1e-3
    tr = S[:, :3].sum(1) / 3.0
    S[:, :3] -= tr[:, None]  # trace-free
    return S


def test_eddy_viscosity_stress_gives_back_its_viscosity():
    from paper_2605_19796_gb300.learned import dissipation_targets

    rng = np.random.default_rng(4)
    n, c_nu, delta = 64, 0.035, 1.0
    S = _sym(rng, n)
    nu_e = rng.uniform(1e-5, 1e-3, size=n)
    k = rng.uniform(0.0, 1e-4, size=n)
    T = -2.0 * nu_e[:, None] * S
    T[:, :3] += (2.0 * k / 3.0)[:, None]
    out = dissipation_targets(torch.from_numpy(T).float(), torch.from_numpy(S).float(), c_nu, delta).double().numpy()
    tr = out[:, :3].sum(1)
    want = 2.0 * (nu_e / (c_nu * delta)) ** 2
    assert np.allclose(tr, want, rtol=2e-5, atol=0), np.max(np.abs(tr / want - 1))
    # the deviatoric part is the input's
    # the deviatoric part is the input's (to the FP32 rounding of the output,
    # whose diagonal holds the new trace)
    T32 = T.astype(np.float32).astype(np.float64)
    dev_in = T32.copy()
    dev_in[:, :3] -= T32[:, :3].sum(1)[:, None] / 3.0
    dev_out = out.copy()
    dev_out[:, :3] -= tr[:, None] / 3.0
    assert np.allclose(dev_out, dev_in, rtol=0, atol=4 * 2.0 ** -23 * np.abs(out).max())
    # the rate of Eq. (omega_sgs_operational) recovers nu_e
    assert np.allclose(c_nu * delta * np.sqrt(np.abs(tr) / 2.0), nu_e, rtol=1e-5)


def test_backscatter_and_zero_strain_give_zero_trace():
    from paper_2605_19796_gb300.learned import dissipation_targets

    rng = np.random.default_rng(5)
    S = _sym(rng, 8)
    T = 2.0 * 3e-4 * S  # transfer -T:S < 0 (backscatter)
    out = dissipation_targets(torch.from_numpy(T).float(), torch.from_numpy(S).float(), 0.035).double().numpy()
    assert np.abs(out[:, :3].sum(1)).max() <= 1e-12
    out0 = dissipation_targets(torch.from_numpy(T).float(), torch.zeros((8, 6)), 0.035).double().numpy()
    assert np.abs(out0[:, :3].sum(1)).max() <= 1e-12


def test_planted_mistake_fails():
    """Dropping the off-diagonal weight 2 from the transfer -T : S (but not from
    S : S) changes nu* and fails the eddy-viscosity pin.  (Dropping it from both
    leaves nu* of a pure eddy-viscosity stress unchanged, which is why the pin
    stresses the off-diagonal terms.)"""
    from paper_2605_19796_gb300 import learned

    rng = np.random.default_rng(6)
    n = 16
    S = _sym(rng, n)
    S[:, 3:] *= 5.0  # strong shear components
    nu_e = np.full(n, 2e-4)
    T = -2.0 * nu_e[:, None] * S

    def wrong(T, S, c_nu, delta=1.0):
        Td, Sd = T.double(), S.double()
        w = torch.tensor([1.0, 1.0, 1.0, 2.0, 2.0, 2.0], dtype=torch.float64)
        pi = -(Td * Sd).sum(1)
        ss = (Sd * Sd * w).sum(1)
        nu_star = torch.clamp(pi, min=0.0) / (2.0 * ss)
        out = Td.clone()
        tr_new = 2.0 * (nu_star / (c_nu * delta)) ** 2
        for k in range(3):
            out[:, k] += (tr_new - (Td[:, 0] + Td[:, 1] + Td[:, 2])) / 3.0
        return out.float()

    good = learned.dissipation_targets(torch.from_numpy(T).float(), torch.from_numpy(S).float(), 0.035)
    bad = wrong(torch.from_numpy(T).float(), torch.from_numpy(S).float(), 0.035)
    want = 2.0 * (nu_e / 0.035) ** 2
    assert np.allclose(good[:, :3].sum(1).double().numpy(), want, rtol=2e-5)
    assert not np.allclose(bad[:, :3].sum(1).double().numpy(), want, rtol=2e-5)
