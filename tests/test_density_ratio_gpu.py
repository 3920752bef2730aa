"""Density ratio != 1 on the GPU (Sec. 2.3, 3.3: rho(phi) and mu(phi), the mass flux S, the grad rho
terms of H, m2H and P, and the time derivative of S from a stored history) against the FP64
oracle, with both step kernels, inside batches and across checkpoints."""
import numpy as np
import pytest

import oracle
from paper_2408_15654_gb300 import lbm
from paper_2408_15654_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load()
    return torch


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def case(name, n_eps=1e-4):
    """The rising bubble of Sec. 4 at R = 16 (64 x 128, walls, gravity, ratio 10 in density and
    viscosity) and at the paper's resolution R = 60 (240 x 480, 1000 steps); a relaxing slab
    translating along its normal (S parallel to u); a perturbed drop of ratio 5 with the Langmuir
    EOS on a ragged grid between moving walls.  These runs take the unit
    normal only where |grad phi| > 1e-4: with the default threshold (n wherever grad phi is not
    zero) the bulk normal is a rounding artifact and the FP64 oracle itself moves by 5e-5 under a
    single-precision jitter of its inputs (tests/test_conditioning.py).  The arithmetic is the same
    for either threshold; the default one is checked on short runs below."""
    if name == "bubble_R16":
        p, f = W.rising_bubble(16.0)
        return (dict(p, n_eps=n_eps), f), 400
    if name == "bubble_R60":
        p, f = W.rising_bubble(60.0)
        return (dict(p, n_eps=n_eps), f), 1000
    if name == "slab_70x6":
        n = 70
        x = np.arange(n) + 0.5
        ph1 = 0.5 * (np.tanh(2 * (x - n / 4) / 8.0) - np.tanh(2 * (x - 3 * n / 4) / 8.0))
        phi = np.tile(ph1[None, :], (6, 1))
        p = W.base_params(n, 6, rhoA=1.0, rhoB=0.1, muA=0.1, muB=0.05, sigma0=1e-3, E0=0.5, M_phi=0.05,
                          n_eps=n_eps)
        return (p, W.fields(phi, 0.3 * 4 * phi * (1 - phi), ux=0.02)), 300
    p, f = W.shear_drop(45, 19, R=6)
    p = dict(p, rhoA=0.2, rhoB=1.0, muA=p["muA"] * 0.5, n_eps=n_eps)
    return (p, W.perturbed(p, f, seed=7)), 200


NAMES = ["bubble_R16", "bubble_R60", "slab_70x6", "langmuir_45x19"]
_oracle = {}


def oracle_moments(name):
    if name not in _oracle:
        (p, f), steps = case(name)
        o = oracle.Sim(p)
        o.init(**f)
        o.step(steps)
        _oracle[name] = o.moments()
    return _oracle[name]


def errors(m, om):
    e = {k: rel_l2(m[k], om[k]) for k in ("phi", "psi")}
    du = np.hypot(m["ux"] - om["ux"], m["uy"] - om["uy"])
    e["u"] = float(np.linalg.norm(du) / np.linalg.norm(np.hypot(om["ux"], om["uy"])))
    dp = (m["P"] - m["P"].mean()) - (om["P"] - om["P"].mean())
    e["P"] = float(np.abs(dp).max() / max(np.ptp(om["P"]), 1e-30))
    return e


@pytest.mark.parametrize("name", NAMES)
def test_density_ratio_matches_oracle(torch, name):
    """phi and psi within 1e-5 (relative L2) in every case; u within 1e-5 relative L2, except for the
    bubble at R = 60.  After 1000 steps that bubble has run for 0.05 of its time scale R / U_c
    (U_c = 0.175 / R, the velocity scale of the paper's diffusive scaling) and |u| is about 1 % of
    U_c, so a relative L2 of u compares FP32 rounding with a flow that has barely started: its u
    error is held to 1e-5 of U_c (measured 3.4e-7) and to 1e-4 relative L2 (measured 3.9e-5).  The
    same ratio of about 10 between the GPU-oracle difference and the GPU's own spread under a
    single-precision jitter of the inputs holds at R = 16 (4.5e-6 against 5.6e-7) and at R = 60
    (3.9e-5 against 2-3.5e-6), while the FP64 oracle moves by 1.9e-7 under that jitter."""
    (p, f), steps = case(name)
    om = oracle_moments(name)
    g = lbm.Lattice(p)
    g.init(**f)
    g.step(steps)
    m = g.moments()
    e = errors(m, om)
    print(name, {k: f"{v:.2e}" for k, v in e.items()})
    assert e["phi"] <= 1e-5 and e["psi"] <= 1e-5, e
    if name == "bubble_R60":
        du = np.hypot(m["ux"] - om["ux"], m["uy"] - om["uy"])
        u_scale = float(np.sqrt((du ** 2).mean()) / (0.175 / 60.0))
        print(name, f"rms |du| / U_c {u_scale:.2e}")
        assert u_scale <= 1e-5 and e["u"] <= 1e-4, (u_scale, e)
    else:
        assert e["u"] <= 1e-5, e
    assert e["P"] <= 1e-3, e
    assert g.status == 0


@pytest.mark.parametrize("name", ["bubble_R16", "slab_70x6", "langmuir_45x19"])
def test_density_ratio_default_normal_threshold_short_run(torch, name):
    """The same cases for 40 steps with n taken wherever grad phi is not zero."""
    (p, f), _ = case(name, n_eps=1e-12)
    o = oracle.Sim(p)
    o.init(**f)
    o.step(40)
    g = lbm.Lattice(p)
    g.init(**f)
    g.step(40)
    e = errors(g.moments(), o.moments())
    print(name, "n_eps 1e-12, 40 steps", {k: f"{v:.2e}" for k, v in e.items()})
    assert e["phi"] <= 1e-5 and e["psi"] <= 1e-5 and e["u"] <= 1e-5, e
    assert e["P"] <= 1e-3, e


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16_fg"])
def test_density_ratio_pipelined_equals_tile_and_checkpoint(torch, storage):
    (p, f), _ = case("bubble_R16")
    p = dict(p, storage=storage)
    out = []
    for kern in ("tile", "pipelined"):
        g = lbm.Lattice(p)
        g.kernel = kern
        g.init(**f)
        g.step(9)
        blob = g.state()
        g.step(8)
        out.append(g.state())
        h = lbm.Lattice(p)
        h.kernel = kern
        h.init(**W.fields(np.zeros((p["ny"], p["nx"])), 0.0))
        h.restore(blob)
        h.step(8)
        assert h.state() == out[-1], kern  # the mass-flux history travels with the state
        g.close()
        h.close()
    assert out[0] == out[1]


def test_density_ratio_members_in_a_mixed_batch_equal_alone(torch):
    stream = torch.cuda.Stream()
    items = [case(n)[0] for n in NAMES] + [W.shear_drop(96, 40, R=9), W.convected_drop(64, 48, R=10)]
    ref = []
    for p, f in items:
        g = lbm.Lattice(p, stream=stream)
        g.init(**f)
        g.step(13)
        ref.append(g.state())
        g.close()
    lats = []
    for p, f in items:
        g = lbm.Lattice(p, stream=stream)
        g.init(**f)
        lats.append(g)
    b = lbm.Batch(lats, stream)
    b.set_schedule("largest_first", 4)
    b.step(13)
    torch.cuda.synchronize()
    for k, g in enumerate(lats):
        assert g.state() == ref[k], k
    b.close()


@pytest.mark.parametrize("storage", ["fp16", "bf16", "fp16_fg", "bf16_fg"])
def test_density_ratio_16bit_storage_error(torch, storage):
    """The rising bubble in 16-bit storage: stated error after 400 steps (measured on GB300, phi and
    psi: FP16 2.0e-4 and 7.7e-4, FP16_FG 2.0e-4 and 7.1e-4, BF16 1.5e-3 and 5.3e-3, BF16_FG 1.5e-3
    and 6.1e-3)."""
    (p, f), steps = case("bubble_R16")
    om = oracle_moments("bubble_R16")
    g = lbm.Lattice(dict(p, storage=storage))
    g.init(**f)
    g.step(steps)
    e = errors(g.moments(), om)
    print(storage, {k: f"{v:.2e}" for k, v in e.items()})
    bound = 3e-3 if storage.startswith("fp16") else 3e-2
    assert e["phi"] <= bound and e["psi"] <= bound, e
