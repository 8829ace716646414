"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (stated in the test, derived from the arithmetic):
  - FP64 storage: max |gpu - oracle| / max |oracle| <= 1e-12 for populations,
    density and velocity (the two sides differ only in rounding order and FMA
    contraction, ~1e-16 per operation, accumulated over at most 200 steps);
  - FP32 storage: max |u_gpu - u_oracle| <= 1e-5 lattice units after 50 steps
    of 64^3 decaying turbulence (u_rms = 0.04): FP32 storage rounding
    (~6e-8 relative per population per step) accumulated over the run.
"""
import math

import numpy as np
import pytest

from paper_2605_19796_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_19796_gb300 import build

    build.build()
    from paper_2605_19796_gb300 import lbm as _lbm

    return _lbm


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


CL = {"bgk": 0, "kcmp": 1, "kcrb_hermite": 2, "kcrb_raw": 3, "kcrr": 4}
CNU = {"bgk": 0.0, "kcmp": 0.035, "kcrb_hermite": 0.02, "kcrb_raw": 0.02, "kcrr": 0.02}


def _run_pair(lbm, orc, q, shape, rho, u, nu, closure, steps, storage="fp64", bc=(0, 0, 0), F=(0.0, 0.0, 0.0),
              checkpoints=None, **kw):
    """Runs GPU and oracle from the same equilibrium state; returns lists of
    (gpu populations, oracle populations) at the checkpoints."""
    nx, ny, nz = shape
    checkpoints = checkpoints or [steps]
    out = []
    with lbm.Solver(q, shape, nu, closure=closure, c_nu=CNU[closure], storage=storage, bc=bc, force=F, **kw) as s:
        s.init_velocity(rho, u)
        f = orc.init_equilibrium(q, rho, u)
        done = 0
        for cp in checkpoints:
            s.step(cp - done)
            f = orc.run(f, cp - done, closure=CL[closure], nu=nu, c_nu=CNU[closure], bc=bc, F=F)
            done = cp
            out.append((s.get_populations(), f.copy(), s))
            s.synchronize()
    return out


def test_tgv_32_d3q19_fp64_kcmp_200_steps(lbm, orc):
    """3D Taylor-Green vortex, periodic 32^3 D3Q19, FP64, U0 = 0.05, Re = 1600
    (nu = U0 L_TGV / 1600, L_TGV = 32/(2 pi)), KC-MP, 200 steps: fields and
    kinetic energy / enstrophy at steps 0, 50, 100, 200."""
    n, u0 = 32, 0.05
    nu = u0 * (n / (2 * math.pi)) / 1600.0
    rho, u = inputs.tgv_fields(n, u0=u0)
    with lbm.Solver(19, (n, n, n), nu, closure="kcmp", storage="fp64") as s:
        s.init_velocity(rho, u)
        f = orc.init_equilibrium(19, rho, u)
        done = 0
        ek = []
        for cp in (0, 50, 100, 200):
            s.step(cp - done)
            f = orc.run(f, cp - done, closure=1, nu=nu, c_nu=0.035)
            done = cp
            r_g, u_g = s.moments()
            r_o, u_o = orc.fields(f)
            assert rel(r_g, r_o) < TOL64 and rel(u_g, u_o) < TOL64, (cp, rel(r_g, r_o), rel(u_g, u_o))
            assert rel(s.get_populations(), f) < TOL64
            d_g, d_o = s.diagnostics(), orc.diagnostics(f)
            # mass, E_k, enstrophy relative; momentum sums (~0 for the TGV) against mass * u0
            for k in (0, 4, 5):
                assert abs(d_g[k] - d_o[k]) <= TOL64 * abs(d_o[k]), (cp, k, d_g[k], d_o[k])
            for k in (1, 2, 3):
                assert abs(d_g[k] - d_o[k]) <= TOL64 * d_o[0] * u0, (cp, k, d_g[k], d_o[k])
            # dissipation rates of the next pre-collision state (FP64 on the GPU)
            e_o = orc.dissipation(f, closure=1, nu=nu, c_nu=0.035)
            assert np.abs(d_g[8:10] - e_o).max() <= TOL64 * np.abs(e_o).max(), (cp, d_g[8:10], e_o)
            ek.append(d_g[4])
        assert ek[-1] < ek[0]  # energy decays


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("closure", ["bgk", "kcmp", "kcrb_hermite", "kcrb_raw"])
def test_closures_ragged_fp64(lbm, orc, q, closure):
    """Ragged box (not a multiple of the 32 x 8 tile or of the z-chunk),
    under-resolved turbulence so that the turbulent rate is active."""
    shape = (37, 21, 13)
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.08, seed=1, shape=shape)
    nu = 2e-5
    (fg, fo, _), = _run_pair(lbm, orc, q, shape, rho, u, nu, closure, 12)
    assert rel(fg, fo) < TOL64
    if closure != "bgk":
        f0 = orc.init_equilibrium(q, rho, u)
        fb = orc.run(f0, 12, closure=0, nu=nu)
        assert np.abs(fo - fb).max() > 1e-7, "the closure must be active in this test"


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("closure", ["bgk", "kcmp", "kcrb_hermite", "kcrb_raw", "kcrr"])
def test_dissipation_matches_oracle_fp64(lbm, orc, q, closure):
    """lbm_diagnostics out[8], out[9] (<2 rho nu_eff S:S>, <2 rho nu S:S> of the
    next pre-collision state, FP64 on the GPU) against the oracle's
    dissipation() of the same stored state to 1e-12, on a ragged
    under-resolved box where the clipped rate is active."""
    if closure == "kcrr" and q == 19:
        pytest.skip("KC-RR is D3Q27 only")
    shape = (37, 21, 13)
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.08, seed=21, shape=shape)
    nu = 2e-5
    with lbm.Solver(q, shape, nu, closure=closure, c_nu=CNU[closure], storage="fp64") as s:
        s.init_velocity(rho, u)
        s.step(6)
        d = s.diagnostics()
        f = s.get_populations()
    e_o = orc.dissipation(f, closure=CL[closure], nu=nu, c_nu=CNU[closure])
    assert np.abs(d[8:10] - e_o).max() <= TOL64 * np.abs(e_o).max(), (d[8:10], e_o)
    if closure != "bgk":
        assert d[8] > 1.5 * d[9], "the clipped rate must be active somewhere"
    else:
        assert abs(d[8] - d[9]) <= TOL64 * d[9]


@pytest.mark.parametrize("q", [19, 27])
def test_dissipation_channel_fp64(lbm, orc, q):
    """The same with bounce-back walls in y and a body force (one-sided strain
    at the wall rows, half-force shift of u), KC-MP."""
    shape = (16, 11, 6)
    rho, u = inputs.channel_fields(*shape, 0.05, seed=5)
    F = (1e-5, 0.0, 0.0)
    with lbm.Solver(q, shape, 2e-3, closure="kcmp", storage="fp64", bc=(0, 1, 0), force=F) as s:
        s.init_velocity(rho, u)
        s.step(4)
        d = s.diagnostics()
        f = s.get_populations()
    e_o = orc.dissipation(f, closure=1, nu=2e-3, c_nu=0.035, bc=(0, 1, 0), F=F)
    assert np.abs(d[8:10] - e_o).max() <= TOL64 * np.abs(e_o).max(), (d[8:10], e_o)


@pytest.mark.parametrize("shape", [(4, 4, 4), (1, 1, 6), (3, 5, 2), (64, 8, 1), (33, 9, 5), (2, 40, 3)])
def test_small_and_degenerate_shapes_fp64(lbm, orc, shape):
    rho, u = inputs.hit_fields(0, k0=1.0, urms=0.05, seed=2, shape=shape)
    (fg, fo, _), = _run_pair(lbm, orc, 27, shape, rho, u, 1e-4, "kcmp", 7)
    assert rel(fg, fo) < TOL64


@pytest.mark.parametrize("zchunk,tile_y", [(1, 8), (3, 8), (20, 8), (5, 16), (7, 4)])
def test_launch_shapes_fp32_consistent(lbm, orc, zchunk, tile_y):
    """Within one kernel instantiation (the tile height picks it) every z-chunk
    gives the bit-identical FP32 result of the default chunking (the per-cell
    arithmetic does not depend on the decomposition); other tile heights are
    other instantiations and agree with the default launch to FP32 rounding."""
    shape = (40, 24, 20)
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.06, seed=3, shape=shape)
    res = []
    for zc, ty in ((0, 0), (0, tile_y), (zchunk, tile_y)):
        with lbm.Solver(27, shape, 3e-5, closure="kcmp", storage="fp32", zchunk=zc, tile_y=ty) as s:
            s.init_velocity(rho, u)
            s.step(6)
            res.append(s.get_populations())
    assert np.array_equal(res[1], res[2])
    assert rel(res[1], res[0]) < 1e-6


@pytest.mark.parametrize("closure", ["bgk", "kcmp", "kcrb_hermite", "kcrb_raw"])
def test_variants_agree_fp32(lbm, orc, closure):
    """The register-pull (1), split-barrier (8) and asynchronous-copy (13) step
    kernels perform the same per-cell arithmetic: FP32 results agree to FP32 rounding on
    a ragged box; within one variant the z-chunking does not change a bit."""
    shape = (45, 19, 23)
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.07, seed=8, shape=shape)
    res = {}
    for var, zc in [(1, 0), (8, 0), (8, 5), (13, 0), (13, 5)]:
        with lbm.Solver(27, shape, 2e-5, closure=closure, storage="fp32", variant=var, zchunk=zc) as s:
            s.init_velocity(rho, u)
            s.step(8)
            res[(var, zc)] = s.get_populations()
    for v in (8, 13):
        assert rel(res[(v, 0)], res[(1, 0)]) < 1e-6, v
        assert np.array_equal(res[(v, 0)], res[(v, 5)]), v


def test_fp32_hit_64_velocity(lbm, orc):
    """Decaying HIT at 64^3 D3Q27 (k0 = 4, u_rms = 0.04, nu = 1e-4), KC-MP,
    FP32 storage and arithmetic (default launch) vs the FP64 oracle after 50
    steps: velocity to 1e-5, and the dissipation rates of the GPU's FP64
    reduction against the oracle's of its own run.  Tolerance of the rates:
    the velocity error (<= 1e-5 against strains of about 1e-2) moves S:S by
    about 2e-3 relatively at most, and the clipped rate follows tr m_sgs, formed
    from FP32 populations (relative error of m_neq - m_CE about 1e-3): 5e-3 for
    <2 rho nu_eff S:S>, 2.5e-3 for <2 rho nu S:S>."""
    n = 64
    rho, u = inputs.hit_fields(n, k0=4.0, urms=0.04, seed=0)
    with lbm.Solver(27, (n, n, n), 1e-4, closure="kcmp", storage="fp32") as s:
        s.init_velocity(rho, u)
        s.step(50)
        fg = s.get_populations()
        dg = s.diagnostics()
    fo = orc.run(orc.init_equilibrium(27, rho, u), 50, closure=1, nu=1e-4, c_nu=0.035)
    _, ug = orc.fields(fg)
    _, uo = orc.fields(fo)
    err = float(np.abs(ug - uo).max())
    assert err <= 1e-5, err
    do = orc.dissipation(fo, closure=1, nu=1e-4, c_nu=0.035)
    assert dg[8] > dg[9] > 0  # the closure is active
    assert abs(dg[8] - do[0]) <= 5e-3 * do[0], (dg[8], do[0])
    assert abs(dg[9] - do[1]) <= 2.5e-3 * do[1], (dg[9], do[1])


def _spectrum(u):
    """The oracle's E(k) (oracle/spectrum.py, pinned in tests/test_oracle_spectrum.py)."""
    from oracle.spectrum import spectrum

    return spectrum(u)


def test_fp32_hit_64_statistics(lbm, orc):
    """Decaying HIT at 64^3 (k0 = 4, u_rms = 0.04, nu = 1e-4, KC-MP), FP32 GPU
    (default launch) against the FP64 oracle over 300 steps: the energy spectrum
    at steps 200 and 300 to 1e-4 relative L2 over the shells 1..31, the
    kinetic energy to 2e-5 and the dissipation rate -dE_k/dt between them to
    1e-3 relative (FP32 storage rounds each population to 2^-24 relative every
    step; the measured kinetic-energy difference at step 200 is 6e-6)."""
    n = 64
    rho, u = inputs.hit_fields(n, k0=4.0, urms=0.04, seed=0)
    out = _run_pair(lbm, orc, 27, (n, n, n), rho, u, 1e-4, "kcmp", 300, storage="fp32", checkpoints=[200, 300])
    ek = {}
    for (fg, fo, _), step in zip(out, (200, 300)):
        rg, ug = orc.fields(fg)
        ro, uo = orc.fields(fo)
        eg, eo = _spectrum(ug), _spectrum(uo)
        err = np.sqrt(((eg[1:] - eo[1:]) ** 2).sum() / (eo[1:] ** 2).sum())
        assert err < 1e-4, (step, err)
        ek[step] = (float((0.5 * rg * (ug ** 2).sum(0)).mean()), float((0.5 * ro * (uo ** 2).sum(0)).mean()))
        assert abs(ek[step][0] - ek[step][1]) <= 2e-5 * ek[step][1]
    eps_g = (ek[200][0] - ek[300][0]) / 100
    eps_o = (ek[200][1] - ek[300][1]) / 100
    assert eps_o > 0 and abs(eps_g - eps_o) <= 1e-3 * eps_o, (eps_g, eps_o)


def test_hit_256_2000_steps(lbm, orc):
    """Decaying HIT at 256^3 (k0 = 4, u_rms = 0.04, nu = 1e-4, KC-MP, FP32,
    default launch) for 2000 steps: no non-finite flag, mass conserved to FP32
    accumulation (1e-6 relative), kinetic energy decaying every 250 steps."""
    import torch

    n = 256
    rho, u = inputs.hit_fields(n, k0=4.0, urms=0.04, seed=3, device="cuda")
    with lbm.Solver(27, (n, n, n), 1e-4, closure="kcmp", storage="fp32") as s:
        s.init_velocity_device(rho, u)
        r = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
        v = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
        s.moments_device(r, v)
        m0 = float(r.sum())
        ek = [float((0.5 * r * (v ** 2).sum(0)).mean())]
        for _ in range(8):
            s.step(250)
            s.synchronize()
            s.moments_device(r, v)
            ek.append(float((0.5 * r * (v ** 2).sum(0)).mean()))
        assert abs(float(r.sum()) - m0) <= 1e-6 * m0
    assert all(b < a for a, b in zip(ek, ek[1:])), ek
    assert ek[-1] > 0.05 * ek[0]


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("ny", [24, 13, 9])
def test_channel_walls_force_fp64(lbm, orc, q, ny):
    """Halfway bounce-back walls in y, Guo body force in x, one-sided strain
    stencils at the wall layers; ny = 13 and 9 leave one or five rows in the last tile."""
    shape = (20, ny, 6)
    rng = np.random.default_rng(4)
    rho = np.ones((6, ny, 20))
    u = np.zeros((3, 6, ny, 20))
    y = (np.arange(ny) + 0.5) / ny
    u[0] = (0.05 * 4 * y * (1 - y))[None, :, None]
    u += 0.01 * rng.standard_normal(u.shape)
    F = (2e-5, 0.0, 0.0)
    (fg, fo, _), = _run_pair(lbm, orc, q, shape, rho, u, 5e-5, "kcmp", 10, bc=(0, 1, 0), F=F)
    assert rel(fg, fo) < TOL64


def test_ensemble_fp64(lbm, orc):
    """Three independent boxes with different viscosities in one launch."""
    shape = (16, 12, 10)
    nus = np.array([5e-5, 2e-4, 4.5e-4])
    fields = [inputs.hit_fields(0, k0=2.0, urms=0.06, seed=10 + b, shape=shape) for b in range(3)]
    rho = np.stack([f[0] for f in fields])
    u = np.stack([f[1] for f in fields], axis=1)
    with lbm.Solver(27, shape, nus, closure="kcmp", storage="fp64", nbatch=3) as s:
        s.init_velocity(rho, u)
        s.step(8)
        fg = s.get_populations()
    for b in range(3):
        fo = orc.run(orc.init_equilibrium(27, fields[b][0], fields[b][1]), 8, closure=1, nu=nus[b], c_nu=0.035)
        assert rel(fg[b], fo) < TOL64


def test_save_load_resume_bitwise(lbm, orc, tmp_path):
    shape = (24, 16, 12)
    rho, u = inputs.hit_fields(0, k0=2.0, urms=0.05, seed=5, shape=shape)
    p = str(tmp_path / "state.lbm")
    with lbm.Solver(27, shape, 1e-4, closure="kcmp", storage="fp32") as s:
        s.init_velocity(rho, u)
        s.step(10)
        s.save(p)
        s.step(10)
        a = s.get_populations()
        assert s.step_count == 20
    with lbm.Solver(27, shape, 1e-4, closure="kcmp", storage="fp32") as s:
        s.load(p)
        assert s.step_count == 10
        s.step(10)
        b = s.get_populations()
    assert np.array_equal(a, b)
    with lbm.Solver(19, shape, 1e-4, closure="kcmp", storage="fp32") as s:
        with pytest.raises(lbm.LbmError):
            s.load(p)


def test_nonfinite_is_reported(lbm, orc):
    """A NaN injected into the host-side initial field is caught by the step's
    device flag and reported as LBM_ERR_NONFINITE (no device fault involved)."""
    shape = (16, 8, 8)
    rho, u = inputs.hit_fields(0, k0=2.0, urms=0.05, seed=6, shape=shape)
    u[0, 3, 4, 5] = np.nan
    with lbm.Solver(27, shape, 1e-4, closure="kcmp", storage="fp32") as s:
        s.init_velocity(rho, u)
        s.step(2)
        with pytest.raises(lbm.LbmError) as ei:
            s.synchronize()
        assert ei.value.code == lbm.LBM_ERR_NONFINITE
        s.synchronize()  # the flag is cleared once reported


def test_bad_configs_rejected(lbm):
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Solver(19, (8, 8, 8), 1e-4, closure="kcrr")
    assert ei.value.code == lbm.LBM_ERR_UNSUPPORTED
    with pytest.raises(lbm.LbmError):
        lbm.Solver(27, (8, 0, 8), 1e-4)
    with pytest.raises(lbm.LbmError):
        lbm.Solver(27, (8, 8, 8), -1.0)
    with pytest.raises(lbm.LbmError):
        lbm.Solver(27, (8, 8, 8), 1e-4, bc=(1, 0, 0))


def _sampled_cells(n, k, seed):
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, n, size=(k, 3))
    # include the domain corners and tile / chunk edges
    extra = np.array([[0, 0, 0], [n - 1, n - 1, n - 1], [31, 7, 15], [32, 8, 16], [n - 1, 0, n // 2]])
    return np.concatenate([pts, extra])


@pytest.mark.parametrize("n", [256, 512])
def test_full_size_sampled_cells_fp32(lbm, orc, n):
    """Full-size decaying HIT (D3Q27, FP32, KC-MP, nu = 1e-4) in the default launch
    configuration: one GPU step, then sampled cells against the oracle's
    single-cell step evaluated on the GPU's own pre-step populations (FP32
    values are exact in FP64).  Tolerance: 2e-6 x max|f| (FP32 arithmetic of
    ~10^3 operations per cell)."""
    rho, u = inputs.hit_fields(n, k0=4.0, urms=0.04, seed=0)
    pts = _sampled_cells(n, 48, seed=n)
    offs = np.array([(dx, dy, dz) for dz in range(-2, 3) for dy in range(-2, 3) for dx in range(-2, 3)])
    with lbm.Solver(27, (n, n, n), 1e-4, closure="kcmp", storage="fp32") as s:
        # the four-cell kernel on 128 x 8 tiles with the rows' interior staged by TMA
        assert s.launch_config["variant"] == 16 and s.launch_config["tile_y"] == 8
        s.init_velocity(rho, u)
        del rho, u
        s.step(3)
        blocks = s.probe((pts[:, None, :] + offs[None, :, :]).reshape(-1, 3)).reshape(len(pts), 125, 27)
        mass0 = s.diagnostics()[0]
        s.step(1)
        after = s.probe(pts)
        mass1 = s.diagnostics()[0]
    scale = np.abs(after).max()
    for k in range(len(pts)):
        blk = blocks[k].T.reshape(27, 5, 5, 5)
        ref = orc.step_cell(blk, closure=1, nu=1e-4, c_nu=0.035)
        assert np.abs(after[k] - ref).max() <= 2e-6 * scale, (pts[k], np.abs(after[k] - ref).max())
    assert abs(mass1 - mass0) <= 1e-9 * mass0


def test_full_size_sampled_cells_d3q19_fp32(lbm, orc):
    """Full-size D3Q19 HIT (512^3, FP32, KC-MP) in its default launch (the
    four-cell kernel with TMA staging, the D3Q27 positions without the
    corners): one GPU step, then sampled cells against the oracle's single-cell
    step on the GPU's own pre-step populations, as the D3Q27 test."""
    n = 512
    rho, u = inputs.hit_fields(n, k0=4.0, urms=0.04, seed=3)
    pts = _sampled_cells(n, 32, seed=19)
    offs = np.array([(dx, dy, dz) for dz in range(-2, 3) for dy in range(-2, 3) for dx in range(-2, 3)])
    with lbm.Solver(19, (n, n, n), 1e-4, closure="kcmp", storage="fp32") as s:
        assert s.launch_config["variant"] == 16 and s.launch_config["tile_y"] == 8
        s.init_velocity(rho, u)
        del rho, u
        s.step(3)
        blocks = s.probe((pts[:, None, :] + offs[None, :, :]).reshape(-1, 3)).reshape(len(pts), 125, 19)
        mass0 = s.diagnostics()[0]
        s.step(1)
        after = s.probe(pts)
        mass1 = s.diagnostics()[0]
    scale = np.abs(after).max()
    for k in range(len(pts)):
        blk = blocks[k].T.reshape(19, 5, 5, 5)
        ref = orc.step_cell(blk, closure=1, nu=1e-4, c_nu=0.035)
        assert np.abs(after[k] - ref).max() <= 2e-6 * scale, (pts[k], np.abs(after[k] - ref).max())
    assert abs(mass1 - mass0) <= 1e-9 * mass0


def test_full_size_sampled_cells_kcrr(lbm, orc):
    """KC-RR at 256^3 (D3Q27, FP32, its default launch: the four-cell kernel
    with TMA staging, variant 16): one GPU step, then sampled cells against the oracle's
    single-cell KC-RR step on the GPU's own pre-step populations; tolerance as
    for KC-MP (the separable Hermite transforms add ~10^2 operations)."""
    n = 256
    rho, u = inputs.hit_fields(n, k0=4.0, urms=0.04, seed=1)
    pts = _sampled_cells(n, 32, seed=7)
    offs = np.array([(dx, dy, dz) for dz in range(-2, 3) for dy in range(-2, 3) for dx in range(-2, 3)])
    with lbm.Solver(27, (n, n, n), 1e-4, closure="kcrr", c_nu=0.02, storage="fp32") as s:
        assert s.launch_config["variant"] == 16
        s.init_velocity(rho, u)
        del rho, u
        s.step(3)
        blocks = s.probe((pts[:, None, :] + offs[None, :, :]).reshape(-1, 3)).reshape(len(pts), 125, 27)
        s.step(1)
        after = s.probe(pts)
    scale = np.abs(after).max()
    for k in range(len(pts)):
        blk = blocks[k].T.reshape(27, 5, 5, 5)
        ref = orc.step_cell(blk, closure=4, nu=1e-4, c_nu=0.02)
        assert np.abs(after[k] - ref).max() <= 2e-6 * scale, (pts[k], np.abs(after[k] - ref).max())


def test_graph_replay_matches_direct_launches(lbm, orc):
    """lbm_step with nsteps >= 2 replays a captured CUDA graph; the result is
    bit-identical to launching the kernels one by one, for odd and even counts
    and across the graph cache (parities and step counts)."""
    shape = (40, 16, 12)
    rho, u = inputs.hit_fields(0, k0=2.0, urms=0.06, seed=9, shape=shape)
    out = []
    for dis in (True, False):
        with lbm.Solver(27, shape, 5e-5, closure="kcmp", storage="fp32", disable_graphs=dis) as s:
            s.init_velocity(rho, u)
            for n in (3, 4, 3, 1, 7, 4, 4):
                s.step(n)
            assert s.step_count == 26
            out.append(s.get_populations())
    assert np.array_equal(out[0], out[1])


def test_autotune_keeps_state_and_result(lbm, orc):
    shape = (64, 32, 24)
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.05, seed=10, shape=shape)
    with lbm.Solver(27, shape, 1e-4, closure="kcmp", storage="fp32") as s:
        s.init_velocity(rho, u)
        s.step(2)
        before = s.get_populations()
        cfg = s.autotune(trials=2)
        assert cfg["variant"] in (1, 8, 12, 13, 14) and cfg["tile_y"] in (4, 8, 16) and 1 <= cfg["zchunk"] <= 128
        assert np.array_equal(before, s.get_populations())
        s.step(5)
        tuned = s.get_populations()
    with lbm.Solver(27, shape, 1e-4, closure="kcmp", storage="fp32") as s:
        s.init_velocity(rho, u)
        s.step(7)
        ref = s.get_populations()
    assert rel(tuned, ref) < 1e-6


def test_ensemble_and_channel_launch_through_graph(lbm, orc):
    """FP64 ensemble of boxes and a walled channel advanced with graph replay
    match the oracle (the graph path uses the same kernels)."""
    shape = (12, 10, 8)
    nus = np.array([1e-4, 3e-4])
    fields = [inputs.hit_fields(0, k0=2.0, urms=0.05, seed=20 + b, shape=shape) for b in range(2)]
    with lbm.Solver(19, shape, nus, closure="kcmp", storage="fp64", nbatch=2) as s:
        s.init_velocity(np.stack([f[0] for f in fields]), np.stack([f[1] for f in fields], axis=1))
        s.step(9)
        fg = s.get_populations()
    for b in range(2):
        fo = orc.run(orc.init_equilibrium(19, fields[b][0], fields[b][1]), 9, closure=1, nu=nus[b], c_nu=0.035)
        assert rel(fg[b], fo) < TOL64
    rho, u = inputs.channel_fields(16, 11, 6, 0.05, seed=3)
    F = (1e-5, 0.0, 0.0)
    (fg, fo, _), = _run_pair(lbm, orc, 27, (16, 11, 6), rho, u, 2e-3, "kcmp", 6, bc=(0, 1, 0), F=F)
    assert rel(fg, fo) < TOL64


def test_default_variant_selection(lbm):
    """Library default: periodic D3Q27 and D3Q19 with 32- or 16-bit storage and BGK,
    KC-MP or KC-RB takes the four-cell kernel (14) when nx is a multiple of 8
    (tiles 128 x 8, or 64 x 16 for boxes at most 64 wide), for FP32 storage
    with TMA staging (16) where nx is a multiple of the tile width and ny a
    multiple of the tile height or at least eight tile heights; the FP32 channel (D3Q27, D3Q19) with BGK or KC-MP the
    four-cell kernel (14) where (ny - 1) is not a multiple of the tile height,
    with KC-MP under the same conditions as the periodic box with TMA staging
    (16);
    otherwise, for FP32 storage, periodic D3Q27 with KC-MP or KC-RB the
    split-barrier pull with L2 prefetches (12) on z-chunks of at most 16
    planes; KC-RR and the other walls with KC-MP the split-barrier pull
    with asynchronous copies (13); periodic
    D3Q27 otherwise (BGK, FP64, 16-bit storage) the split-barrier pull (8);
    the learned closure on periodic boxes the register pull with the network on
    the tcgen05 tensor cores (15); the rest the register pull (1).  Tiles are
    8 rows, 4 for the learned closure.  An explicitly requested variant that
    is not built for a box is refused."""
    for q, closure, storage, want in ((27, "kcmp", "fp32", 14), (27, "kcrb_hermite", "fp16", 14), (27, "kcmp", "fp64", 8),
                                      (27, "kcrb_raw", "fp32", 14), (27, "kcrr", "fp32", 13),
                                      (27, "bgk", "bf16", 14), (19, "kcmp", "fp32", 14), (19, "bgk", "fp32", 14),
                                      (19, "kcmp", "fp16", 14), (27, "kcrr", "fp64", 8),
                                      (27, "learned", "fp32", 15), (27, "learned", "bf16", 15),
                                      (19, "learned", "fp32", 15)):
        with lbm.Solver(q, (40, 32, 64), 1e-4, closure=closure, storage=storage) as s:
            assert s.launch_config["variant"] == want, (q, closure, storage)
            ty = {14: 16, 15: 4, 1: 4 if closure == "learned" else 8}.get(want, 8)  # nx = 40: 64 x 16 tiles
            assert s.launch_config["tile_y"] == ty, (q, closure, storage)
    with lbm.Solver(27, (256, 36, 64), 1e-4, closure="kcmp", storage="fp32") as s:
        assert s.launch_config["variant"] == 14 and s.launch_config["tile_y"] == 8  # a ragged tile, ny < 8 tile heights
    with lbm.Solver(27, (64, 64, 64), 1e-4, closure="kcmp", storage="fp32", nbatch=2) as s:
        assert s.launch_config["variant"] == 16 and s.launch_config["tile_y"] == 16  # full tiles
    with lbm.Solver(27, (256, 64, 16), 1e-4, closure="kcmp", storage="fp32") as s:
        assert s.launch_config["variant"] == 16 and s.launch_config["tile_y"] == 8
    with lbm.Solver(27, (256, 64, 16), 1e-4, closure="kcrr", storage="fp32") as s:
        assert s.launch_config["variant"] == 16 and s.launch_config["tile_y"] == 8  # KC-RR: TMA staging only
    with lbm.Solver(27, (256, 64, 16), 1e-4, closure="kcmp", storage="fp16") as s:
        assert s.launch_config["variant"] == 14
    for closure, storage, want in (("kcmp", "fp32", 12), ("kcrb_hermite", "fp16", 8), ("bgk", "fp32", 8),
                                   ("learned", "fp32", 15)):
        with lbm.Solver(27, (44, 32, 64), 1e-4, closure=closure, storage=storage) as s:  # nx % 8 != 0
            assert s.launch_config["variant"] == want, (closure, storage)
            if closure == "learned":
                assert s.launch_config["tile_y"] == 4
            if want == 12:
                assert s.launch_config["zchunk"] <= 16
    # walls: the four-cell kernel for D3Q27 FP32 with BGK or KC-MP where the top
    # wall row is not the first row of a tile ((ny - 1) % 8 != 0), else variant 13 / 1
    for q, closure, ny, want in ((27, "kcmp", 32, 14), (27, "bgk", 32, 14), (27, "kcmp", 33, 13),
                                 (19, "kcmp", 32, 14), (19, "kcmp", 33, 13), (27, "kcrb_hermite", 32, 1),
                                 (27, "bgk", 33, 1)):
        with lbm.Solver(q, (40, ny, 16), 1e-4, closure=closure, storage="fp32", bc=(0, 1, 0)) as s:
            assert s.launch_config["variant"] == want, (q, closure, ny, "walls")
    for closure, want in (("kcmp", 16), ("bgk", 14)):  # nx a multiple of 64, ny = 130 spans eight 16-row tiles
        with lbm.Solver(27, (128, 130, 8), 1e-4, closure=closure, storage="fp32", bc=(0, 1, 0)) as s:
            assert s.launch_config["variant"] == want and s.launch_config["tile_y"] == 16, (closure, "walls")
    for retired in (4, 9):  # the TMA-staged and packed-pair kernels are retired
        with pytest.raises(lbm.LbmError):
            lbm.Solver(27, (64, 32, 16), 1e-4, closure="kcmp", storage="fp32", variant=retired)
    with pytest.raises(lbm.LbmError):
        lbm.Solver(27, (40, 32, 16), 1e-4, closure="kcmp", storage="fp64", variant=14)


@pytest.mark.parametrize("shape", [(37, 21, 13), (16, 8, 6)])
def test_kcrr_fp64_matches_oracle(lbm, orc, shape):
    """KC-RR (App. F.4, D3Q27): 17 high-order Hermite modes split into the RR
    reference and the SGS departure, relaxed at omega and omega_s."""
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.08, seed=13, shape=shape)
    nu = 2e-5
    with lbm.Solver(27, shape, nu, closure="kcrr", c_nu=0.02, storage="fp64") as s:
        s.init_velocity(rho, u)
        s.step(10)
        fg = s.get_populations()
    fo = orc.run(orc.init_equilibrium(27, rho, u), 10, closure=4, nu=nu, c_nu=0.02)
    assert rel(fg, fo) < TOL64
    fb = orc.run(orc.init_equilibrium(27, rho, u), 10, closure=0, nu=nu)
    assert np.abs(fo - fb).max() > 1e-7, "the closure must be active"


def test_kcrr_fp32_velocity(lbm, orc):
    n = 32
    rho, u = inputs.hit_fields(n, k0=3.0, urms=0.05, seed=14)
    with lbm.Solver(27, (n, n, n), 5e-5, closure="kcrr", c_nu=0.02, storage="fp32") as s:
        s.init_velocity(rho, u)
        s.step(30)
        fg = s.get_populations()
    fo = orc.run(orc.init_equilibrium(27, rho, u), 30, closure=4, nu=5e-5, c_nu=0.02)
    _, ug = orc.fields(fg)
    _, uo = orc.fields(fo)
    assert np.abs(ug - uo).max() <= 1e-5


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("closure", ["bgk", "kcmp", "kcrb_hermite", "kcrb_raw", "kcrr"])
def test_load_schedule_variants(lbm, orc, storage, closure):
    """Variant 8 (halo and own loads together, split arrive/wait barrier) only
    reschedules the loads and synchronisation of the register pull (variant 1);
    variant 12 adds L2 prefetches to it, variant 13 (32- and 64-bit storage)
    copies the own pulls to shared memory asynchronously one plane ahead.  On a
    ragged box with
    two boxes and several z-chunkings (one and two planes per CTA exercise the
    pipelines' start and drain): FP64 matches the oracle to 1e-12, FP32 matches
    variant 1 to FP32 rounding, 16-bit storage in rho and u to 1e-5 (one 16-bit
    rounding of a population); within a variant the z-chunking changes no bit."""
    shape = (45, 19, 23)
    fields = [inputs.hit_fields(0, k0=3.0, urms=0.07, seed=40 + b, shape=shape) for b in range(2)]
    rho = np.stack([f[0] for f in fields])
    u = np.stack([f[1] for f in fields], axis=1)
    nus = np.array([2e-5, 1e-4])
    variants = (8, 12)
    if storage in ("fp32", "fp64"):
        variants += (13,)
    res = {}
    for var, zc in [(1, 0)] + [(v, z) for v in variants for z in (0, 1, 2, 5)]:
        with lbm.Solver(27, shape, nus, closure=closure, storage=storage, variant=var, zchunk=zc, nbatch=2) as s:
            assert s.launch_config["variant"] == var
            s.init_velocity(rho, u)
            s.step(5)
            res[(var, zc)] = s.get_populations()
    for v in variants:
        for zc in (1, 2, 5):
            assert np.array_equal(res[(v, zc)], res[(v, 0)]), (v, zc)
        if storage == "fp64":
            for b in range(2):
                fo = orc.run(orc.init_equilibrium(27, fields[b][0], fields[b][1]), 5, closure=CL[closure], nu=nus[b],
                             c_nu=CNU[closure])
                assert rel(res[(v, 0)][b], fo) < TOL64
        elif storage == "fp32":
            assert rel(res[(v, 0)], res[(1, 0)]) < 1e-6
        else:
            # a one-ulp difference of a stored population (relative spacing 2^-10
            # for FP16, 2^-7 for BF16, at |f - w| <= gmax) may flip between the
            # kernels' rounding orders and propagate over the five steps
            gmax = np.abs(res[(1, 0)] - orc.lattice(27)[1][None, :, None, None, None]).max()
            tol = 8 * (2.0 ** -10 if storage == "fp16" else 2.0 ** -7) * gmax
            for b in range(2):
                r1, u1 = orc.fields(res[(1, 0)][b])
                rv, uv = orc.fields(res[(v, 0)][b])
                assert np.abs(rv - r1).max() < tol and np.abs(uv - u1).max() < tol, (v, tol)


@pytest.mark.parametrize("shape", [(16, 11, 9), (16, 17, 7)])
@pytest.mark.parametrize("q", [19, 27])
def test_variants_channel(lbm, orc, q, shape):
    """Variants 8, 12 and 13 with bounce-back walls and a body force: FP64
    (variants 8 and 13) against the oracle, FP32 against variant 1 to FP32
    rounding.  With ny = 17 the last tile holds only the wall row y = ny - 1,
    whose one-sided stencil reads the outer halo row two below it."""
    rho, u = inputs.channel_fields(*shape, 0.05, seed=5)
    F = (1e-5, 0.0, 0.0)
    with lbm.Solver(q, shape, 2e-3, closure="kcmp", storage="fp64", bc=(0, 1, 0), force=F, variant=8,
                    zchunk=3) as s:
        s.init_velocity(rho, u)
        s.step(6)
        fg = s.get_populations()
    fo = orc.run(orc.init_equilibrium(q, rho, u), 6, closure=1, nu=2e-3, c_nu=0.035, bc=(0, 1, 0), F=F)
    assert rel(fg, fo) < TOL64
    out = {}
    for var in (1, 8, 12, 13):
        with lbm.Solver(q, shape, 2e-3, closure="kcmp", storage="fp32", bc=(0, 1, 0), force=F,
                        variant=var) as s:
            s.init_velocity(rho, u)
            s.step(6)
            out[var] = s.get_populations()
    for var in (8, 12, 13):
        assert rel(out[var], out[1]) < 1e-6, var
    for var, zc in ((1, 2), (8, 2), (13, 2), (13, 3)):
        with lbm.Solver(q, shape, 2e-3, closure="kcmp", storage="fp64", bc=(0, 1, 0), force=F, variant=var,
                        zchunk=zc) as s:
            s.init_velocity(rho, u)
            s.step(6)
            assert rel(s.get_populations(), fo) < TOL64, (var, zc)


@pytest.mark.parametrize("variant", [1, 8, 13])
def test_channel_ensemble_fp64(lbm, orc, variant):
    """Two channel boxes in one launch (bounce-back walls in y, Guo body force,
    each box its own viscosity and seed): every box against the oracle's
    single-box run to 1e-12 in FP64, with a ragged tile row and z-chunk."""
    shape, F = (16, 13, 7), (1e-5, 0.0, 0.0)
    nus = np.array([2e-3, 6e-4])
    fields = [inputs.channel_fields(*shape, 0.05, seed=80 + b) for b in range(2)]
    rho = np.stack([f[0] for f in fields])
    u = np.stack([f[1] for f in fields], axis=1)
    with lbm.Solver(27, shape, nus, closure="kcmp", storage="fp64", bc=(0, 1, 0), force=F, variant=variant,
                    zchunk=3, nbatch=2) as s:
        assert s.launch_config["variant"] == variant
        s.init_velocity(rho, u)
        s.step(5)
        fg = s.get_populations()
    for b in range(2):
        fo = orc.run(orc.init_equilibrium(27, fields[b][0], fields[b][1]), 5, closure=1, nu=nus[b], c_nu=0.035,
                     bc=(0, 1, 0), F=F)
        assert rel(fg[b], fo) < TOL64, (variant, b)


def test_host_alloc_buffers_transfer_like_ordinary_arrays(lbm):
    """lbm_host_alloc buffers (through lbm.host_empty) carry the fields of
    lbm_init_velocity / lbm_moments exactly like ordinary host arrays, over
    more than one staging chunk, and are released when the arrays go."""
    import gc

    shape = (130, 128, 128)
    rho, u = inputs.hit_fields(0, k0=3.0, urms=0.05, seed=90, shape=shape)
    rho_p, u_p = lbm.host_empty(rho.shape), lbm.host_empty(u.shape)
    rho_p[...] = rho
    u_p[...] = u
    with lbm.Solver(27, shape, 1e-4, closure="kcmp", storage="fp32") as s:
        s.init_velocity(rho, u)
        f_a = s.get_populations()
        lbm.lbm_init_velocity(s.h, rho_p, u_p.reshape(3, -1))
        assert np.array_equal(s.get_populations(), f_a)
        s.step(2)
        r_a, u_a = s.moments()
        r_b, u_b = lbm.host_empty(rho.shape), lbm.host_empty(u.shape)
        lbm.lbm_moments(s.h, r_b, u_b)
        assert np.array_equal(r_b, r_a) and np.array_equal(u_b, u_a)
    del rho_p, u_p, r_b, u_b
    gc.collect()
    with pytest.raises(lbm.LbmError):
        lbm.lbm_host_alloc(0)


def test_bounded_wait_times_out_and_handle_stays_usable(lbm, orc):
    """A device-side wait that nothing completes gives up after its poll limit
    and is reported as LBM_ERR_TIMEOUT (no trap, no fault); the handle then
    steps normally and still matches the oracle."""
    shape = (16, 8, 6)
    rho, u = inputs.hit_fields(0, k0=2.0, urms=0.05, seed=21, shape=shape)
    with lbm.Solver(27, shape, 1e-4, closure="kcmp", storage="fp64") as s:
        s.init_velocity(rho, u)
        assert lbm.lbm_wait_selftest(s.h, 1 << 12) == lbm.LBM_ERR_TIMEOUT
        assert "gave up" in lbm.lbm_last_error()
        s.step(3)
        fg = s.get_populations()
    fo = orc.run(orc.init_equilibrium(27, rho, u), 3, closure=1, nu=1e-4, c_nu=0.035)
    assert rel(fg, fo) < TOL64


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
@pytest.mark.parametrize("shape,nbatch", [((100, 100, 110), 2), ((130, 128, 128), 1)])
def test_host_transfers_in_chunks_match_device_calls(lbm, shape, nbatch, storage):
    """lbm_init_velocity / lbm_moments with host pointers stream the fields
    through two staging slots of 2^21 cells (copy of one chunk overlapped with
    the kernel of the other).  On boxes of more than one chunk, with a chunk
    boundary inside the second box and a ragged last chunk, they give exactly
    what the device-pointer calls give."""
    import torch

    fields = [inputs.hit_fields(0, k0=3.0, urms=0.05, seed=60 + b, shape=shape) for b in range(nbatch)]
    rho = np.stack([f[0] for f in fields])
    u = np.stack([f[1] for f in fields], axis=1)
    assert rho.size > (1 << 21)
    with lbm.Solver(27, shape, 1e-4, closure="kcmp", storage=storage, nbatch=nbatch) as s:
        s.init_velocity(rho, u)
        f_host = s.get_populations()
        s.init_velocity_device(torch.from_numpy(rho).cuda(), torch.from_numpy(np.ascontiguousarray(u)).cuda())
        s.synchronize()
        assert np.array_equal(s.get_populations(), f_host)
        s.step(2)
        r_h, u_h = s.moments()
        r_d = torch.empty(rho.shape, dtype=torch.float64, device="cuda")
        u_d = torch.empty(u.shape, dtype=torch.float64, device="cuda")
        s.moments_device(r_d, u_d)
        s.synchronize()
        assert np.array_equal(np.asarray(r_h).reshape(-1), r_d.cpu().numpy().reshape(-1))
        assert np.array_equal(np.asarray(u_h).reshape(3, -1), u_d.cpu().numpy().reshape(3, -1))


@pytest.mark.parametrize("storage", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("shape,nbatch", [((100, 100, 110), 2), ((130, 128, 128), 1)])
def test_fp32_host_fields_match_fp64_calls(lbm, shape, nbatch, storage):
    """lbm_init_velocity_f32 / lbm_moments_f32 (FP32 host fields through the
    same two staging slots, more than one chunk, a ragged last chunk): the
    populations equal, bit for bit, those lbm_init_velocity makes from the same
    fields held as FP64 (the FP32 and 16-bit equilibria are evaluated in FP32,
    the FP64 one from the same values), and the FP32 moments equal the FP64
    moments rounded to FP32 (both are one rounding of the same sums)."""
    fields = [inputs.hit_fields(0, k0=3.0, urms=0.05, seed=70 + b, shape=shape) for b in range(nbatch)]
    rho32 = np.stack([f[0] for f in fields]).astype(np.float32)
    u32 = np.stack([f[1] for f in fields], axis=1).astype(np.float32)
    assert rho32.size > (1 << 21)
    with lbm.Solver(27, shape, 1e-4, closure="kcmp", storage=storage, nbatch=nbatch) as s:
        s.init_velocity(rho32.astype(np.float64), u32.astype(np.float64))
        f64 = s.get_populations()
        s.init_velocity(rho32, u32)  # float32 arrays: lbm_init_velocity_f32
        assert np.array_equal(s.get_populations(), f64)
        s.step(2)
        r64, v64 = s.moments()
        r32, v32 = s.moments(np.float32)
        assert r32.dtype == np.float32 and v32.dtype == np.float32
        assert np.array_equal(r32, r64.astype(np.float32))
        assert np.array_equal(v32, v64.astype(np.float32))
        # rho only / u only
        r_only = np.empty(rho32.shape, np.float32)
        lbm.lbm_moments_f32(s.h, r_only, None)
        assert np.array_equal(r_only.reshape(r32.shape), r32)
        s.init_velocity(None, u32)
        f_u = s.get_populations()
        s.init_velocity(None, u32.astype(np.float64))
        assert np.array_equal(s.get_populations(), f_u)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("closure", ["bgk", "kcmp", "kcrb_raw"])
def test_load_schedule_variants_d3q19(lbm, orc, storage, closure):
    """The load schedules of the split-barrier kernel on D3Q19 (variant 13
    with its asynchronous halo slot and four-plane ring is the D3Q19 FP32
    default for the closures with a carrier): ragged box, two boxes, several
    z-chunkings; FP64 against the oracle to 1e-12, FP32 against variant 1, and
    within a variant the z-chunking changes no bit."""
    shape = (45, 19, 23)
    fields = [inputs.hit_fields(0, k0=3.0, urms=0.07, seed=70 + b, shape=shape) for b in range(2)]
    rho = np.stack([f[0] for f in fields])
    u = np.stack([f[1] for f in fields], axis=1)
    nus = np.array([2e-5, 1e-4])
    res = {}
    for var, zc in [(1, 0)] + [(v, z) for v in (8, 12, 13) for z in (0, 1, 2, 5)]:
        with lbm.Solver(19, shape, nus, closure=closure, storage=storage, variant=var, zchunk=zc, nbatch=2) as s:
            assert s.launch_config["variant"] == var
            s.init_velocity(rho, u)
            s.step(5)
            res[(var, zc)] = s.get_populations()
    for v in (8, 12, 13):
        for zc in (1, 2, 5):
            assert np.array_equal(res[(v, zc)], res[(v, 0)]), (v, zc)
        if storage == "fp64":
            for b in range(2):
                fo = orc.run(orc.init_equilibrium(19, fields[b][0], fields[b][1]), 5, closure=CL[closure], nu=nus[b],
                             c_nu=CNU[closure])
                assert rel(res[(v, 0)][b], fo) < TOL64, v
        else:
            assert rel(res[(v, 0)], res[(1, 0)]) < 1e-6, v
