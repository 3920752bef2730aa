"""16-bit population storage (FP16 / BF16 deviations, FP32 arithmetic) against the FP64 oracle.

The storage error is a stated error, not FP32 round-off: the tolerances below are the measured
errors of each mode with a margin.  Arithmetic is FP32 throughout, so what differs from the FP32
path is only the rounding of the stored populations.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2408_15654_gb300 import lbm
from paper_2408_15654_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# measured errors are written as JSON to the directory named by LBM_RECORD_DIR, if it is set
OUT = os.environ.get("LBM_RECORD_DIR")
_records = {}

# stated relative-L2 error bounds after 1000 steps (128^2 stationary drop, 512x256 shear drop),
# per storage mode and field; measured on GB300 (worst of the two workloads): FP16 phi 9.7e-4,
# psi 1.2e-3, u 5.8e-5; BF16 phi 8.0e-3, psi 8.4e-3, u 3.4e-4; the _fg modes (h in FP32) within
# 5 % of these
BOUND = {
    "fp16": {"phi": 3e-3, "psi": 5e-3, "u": 5e-4},
    "bf16": {"phi": 2e-2, "psi": 3e-2, "u": 2e-3},
}
# f and g in 16 bits with h in FP32: no worse than the all-16-bit mode of the same type
BOUND["fp16_fg"] = BOUND["fp16"]
BOUND["bf16_fg"] = BOUND["bf16"]
HALF = ("fp16", "bf16", "fp16_fg", "bf16_fg")
# 120 steps on a 45 x 19 grid with perturbed fields (every cell near the interface or a wall);
# measured: FP16 phi 6.7e-3, psi 1.5e-2, u 5.2e-4; BF16 phi 7.6e-3, psi 1.8e-2, u 3.6e-3
BOUND_RAGGED = {"phi": 3e-2, "psi": 5e-2, "u": 1e-2}


def _record(name, errs):
    _records[name] = errs
    if not OUT:
        return
    try:
        os.makedirs(OUT, exist_ok=True)
        with open(os.path.join(OUT, "half_store_errors.json"), "w") as f:
            json.dump(_records, f, indent=1)
    except OSError:
        pass


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load()
    yield


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def errors(gm, om, u_scale=None):
    e = {k: rel_l2(gm[k], om[k]) for k in ("phi", "psi")}
    du = np.hypot(gm["ux"] - om["ux"], gm["uy"] - om["uy"])
    un = np.hypot(om["ux"], om["uy"])
    e["u"] = float(np.linalg.norm(du) / (np.linalg.norm(un) if u_scale is None else u_scale * np.sqrt(du.size)))
    dp = (gm["P"] - gm["P"].mean()) - (om["P"] - om["P"].mean())
    e["P"] = float(np.abs(dp).max() / max(np.ptp(om["P"]), 1e-30))
    return e


_oracle_cache = {}


def oracle_moments(key, params, flds, steps):
    if key not in _oracle_cache:
        o = oracle.Sim(params)
        o.init(**flds)
        o.step(steps)
        _oracle_cache[key] = (o.moments(), o.total("phi"), o.total("psi"))
    return _oracle_cache[key]


@pytest.mark.parametrize("storage", HALF)
@pytest.mark.parametrize("case", ["stationary_drop_128", "shear_drop_512x256"])
def test_half_store_error_after_1000_steps(storage, case):
    if case == "stationary_drop_128":
        p, f = W.stationary_drop()
        u_scale = p["sigma0"] / p["muA"]
    else:
        p, f = W.shear_drop()
        u_scale = None
    om, t_phi, t_psi = oracle_moments(case, p, f, 1000)
    q = dict(p, storage=storage)
    g = lbm.Lattice(q)
    g.init(**f)
    g.step(1000)
    e = errors(g.moments(), om, u_scale=u_scale)
    e["sum_phi_rel"] = abs(g.total("phi") - t_phi) / t_phi
    e["sum_psi_rel"] = abs(g.total("psi") - t_psi) / t_psi
    _record(f"{storage}_{case}", e)
    b = BOUND[storage]
    assert e["phi"] <= b["phi"] and e["psi"] <= b["psi"] and e["u"] <= b["u"], e
    # stochastic rounding keeps the storage error unbiased: the totals drift by random walk only
    fp16 = storage.startswith("fp16")
    assert e["sum_phi_rel"] <= (5e-4 if fp16 else 5e-3)
    assert e["sum_psi_rel"] <= (1e-3 if fp16 else 3e-3)
    assert g.status == 0


@pytest.mark.parametrize("storage", HALF)
def test_half_store_ragged_grid_runs_and_conserves(storage):
    """Ragged grid with walls: the 16-bit path of the edge patch and the bounce-back decoding."""
    p, f = W.shear_drop(45, 19, R=6)
    p["sigma0"] = 5e-3
    f = W.perturbed(p, f, seed=11)
    o = oracle.Sim(p)
    o.init(**f)
    o.step(120)
    g = lbm.Lattice(dict(p, storage=storage))
    g.init(**f)
    g.step(120)
    e = errors(g.moments(), o.moments())
    _record(f"{storage}_ragged_45x19", e)
    b = BOUND_RAGGED
    assert e["phi"] <= b["phi"] and e["psi"] <= b["psi"] and e["u"] <= b["u"], e


@pytest.mark.parametrize("storage", HALF)
def test_half_store_checkpoint_is_bitwise(storage):
    p, f = W.shear_drop(80, 48, R=9)
    p["storage"] = storage
    a = lbm.Lattice(p)
    a.init(**f)
    a.step(25)
    blob = a.state()
    a.step(25)
    b = lbm.Lattice(p)
    b.init(**W.fields(np.zeros((48, 80)), 0.0))
    b.restore(blob)
    b.step(25)
    assert a.state() == b.state()


@pytest.mark.parametrize("storage", HALF)
def test_half_store_init_round_trip(storage):
    """Right after initialisation the decoded populations give back the fields to 16-bit precision."""
    p, f = W.shear_drop(40, 24, R=6)
    p["sigma0"] = 0.0
    f = W.perturbed(p, f, seed=3)
    g = lbm.Lattice(dict(p, storage=storage))
    g.init(**f)
    m = g.moments()
    eps = 2.0 ** (-11 if storage.startswith("fp16") else -8)
    np.testing.assert_allclose(m["phi"], f["phi"], atol=9 * eps)
    np.testing.assert_allclose(m["psi"], f["psi"], atol=9 * eps)
    np.testing.assert_allclose(m["ux"], f["ux"], atol=3e-2 * eps * 30)
