"""Many lattices in one launch per step: every member's state is bit for bit what lbm_step gives the
same lattice alone, whatever the schedule, graph length or grouping; members remain usable
through the single-lattice calls; the oracle checks one member directly."""
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


def mixed_cases():
    """Lattices of every group kind: storage modes, walls or periodic, linear or Langmuir EOS,
    ragged sizes (not multiples of the 32 x 8 tile) and a lattice smaller than one tile."""
    out = []
    p, f = W.shear_drop(96, 40, R=9)
    out.append((p, f))                                           # walls, Langmuir, FP32
    p, f = W.stationary_drop(70, 50, R=12)
    out.append((p, W.perturbed(p, f, seed=1)))                   # periodic, linear, FP32, ragged
    p, f = W.shear_drop(45, 19, R=6)
    out.append((dict(p, storage="fp16"), W.perturbed(p, f, seed=2)))
    p, f = W.stationary_drop(64, 64, R=14)
    out.append((dict(p, storage="bf16_fg"), f))
    p, f = W.shear_drop(20, 6, R=2.5)
    out.append((p, W.perturbed(p, f, seed=3)))                   # smaller than one tile
    p, f = W.stationary_drop(33, 9, R=3)
    out.append((dict(p, storage="bf16"), W.perturbed(p, f, seed=4)))
    return out


def make(torch, cases, stream):
    lats = []
    for p, f in cases:
        g = lbm.Lattice(p, stream=stream)
        g.init(**f)
        lats.append(g)
    return lats


def alone_states(torch, cases, steps, stream):
    out = []
    for g in make(torch, cases, stream):
        g.step(steps)
        out.append(g.state())
        g.close()
    return out


@pytest.mark.parametrize("schedule", lbm.SCHEDULES)
@pytest.mark.parametrize("graph_steps", [0, 4])
@pytest.mark.parametrize("kernel", ["auto", "tile", "pipelined"])
def test_batch_bitwise_equals_alone(torch, schedule, graph_steps, kernel):
    """Every schedule, with and without graphs, with each batch kernel; 5 + 8 steps run as graph
    replays and plain launches mixed, which also exercises the alternating tile counters of the
    warp-specialised kernel across replays."""
    stream = torch.cuda.Stream()
    cases = mixed_cases()
    steps = 13  # three 4-step graphs and a remainder
    ref = alone_states(torch, cases, steps, stream)
    lats = make(torch, cases, stream)
    b = lbm.Batch(lats, stream)
    b.kernel = kernel
    assert b.kernel == kernel
    b.set_schedule(schedule, graph_steps)
    b.step(5)
    b.step(steps - 5)
    torch.cuda.synchronize()
    for k, g in enumerate(lats):
        assert g.steps == steps
        assert g.status == 0
        assert g.state() == ref[k], f"member {k}"
    b.close()


def test_batch_launch_count(torch):
    stream = torch.cuda.Stream()
    cases = mixed_cases()
    b = lbm.Batch(make(torch, cases, stream), stream)
    groups = len({(p.get("storage", "fp32"), p.get("walls", False), p.get("eos", "linear")) for p, _ in cases})
    b.set_schedule("largest_first", 0)
    n0 = b.launches
    b.step(7)
    assert b.launches - n0 == 7 * groups + 1
    b.set_schedule("largest_first", 3)
    n0 = b.launches
    b.step(7)  # two graphs of 3 steps (each with its advance kernel) and one plain step
    assert b.launches - n0 == 2 * (3 * groups + 1) + groups + 1
    b.close()


def test_members_mix_with_single_lattice_calls(torch):
    """lbm_step on a member between batch steps, a checkpoint restore, and re-initialisation."""
    stream = torch.cuda.Stream()
    cases = mixed_cases()[:3]
    ref = alone_states(torch, cases, 12, stream)
    lats = make(torch, cases, stream)
    b = lbm.Batch(lats, stream)
    b.set_schedule("edges_first", 4)
    b.step(4)
    lats[1].step(3)       # member 1 runs ahead alone
    blob = lats[2].state()
    lats[2].step(2)
    lats[2].restore(blob)  # and member 2 goes back
    b.step(5)             # members: 9, 12, 9 steps
    lats[0].step(3)
    lats[2].step(3)
    torch.cuda.synchronize()
    for k, g in enumerate(lats):
        assert g.steps == 12
        assert g.state() == ref[k], f"member {k}"
    b.close()


def test_member_list_changes(torch):
    stream = torch.cuda.Stream()
    cases = mixed_cases()
    ref = alone_states(torch, cases, 6, stream)
    lats = make(torch, cases, stream)
    b = lbm.Batch(lats[:2], stream, capacity=len(lats), max_tiles=lbm.lbm_batch_tiles([g.handle for g in lats]))
    b.step(2)
    b.set_members(lats[1:])   # lattice 0 leaves, the others join
    b.step(4)
    b.set_members([])
    b.step(3)                 # an empty batch does nothing
    lats[0].step(4)           # lattice 0: 2 in the batch + 4 alone
    for g in lats[2:]:        # the joiners: 4 in the batch + 2 alone
        g.step(2)
    torch.cuda.synchronize()
    assert [g.steps for g in lats] == [6, 6] + [6] * (len(lats) - 2)
    for k, g in enumerate(lats):
        assert g.state() == ref[k], f"member {k}"
    b.close()


def test_batch_member_validation(torch):
    stream = torch.cuda.Stream()
    cases = mixed_cases()[:2]
    lats = make(torch, cases, stream)
    b = lbm.Batch(lats, stream)
    with pytest.raises(lbm.LBMError):
        b.set_members([lats[0], lats[0]])            # duplicate
    with pytest.raises(lbm.LBMError):
        b.set_members(lats + lats[:1])               # above capacity
    other = lbm.Lattice(cases[0][0], stream=torch.cuda.Stream())
    with pytest.raises(lbm.LBMError):
        b.set_members([other])                       # another stream
    big = lbm.Lattice(W.stationary_drop(256, 256)[0], stream=stream)
    with pytest.raises(lbm.LBMError):
        b.set_members([big])                         # more tiles than max_tiles
    with pytest.raises(lbm.LBMError):
        b.set_schedule(7, 0)
    fresh = lbm.Lattice(cases[0][0], stream=stream)
    b.set_members([fresh])
    with pytest.raises(lbm.LBMError):
        b.step(1)                                    # member without state
    b.close()


def test_autotune_keeps_results_exact(torch):
    stream = torch.cuda.Stream()
    cases = mixed_cases()
    lats = make(torch, cases, stream)
    b = lbm.Batch(lats, stream)
    sched, k = b.autotune(trial_steps=8)
    assert sched in lbm.SCHEDULES and k in (0, 16)
    b.step(3)
    torch.cuda.synchronize()
    steps = lats[0].steps
    assert all(g.steps == steps for g in lats)
    assert steps == 4 * (16 + 16) + 1 + 8 + 3
    ref = alone_states(torch, cases, steps, stream)
    for i, g in enumerate(lats):
        assert g.state() == ref[i], f"member {i}"
    b.close()


def test_batch_member_against_oracle(torch):
    """A member of a mixed batch after 200 steps against the FP64 oracle (FP32 parity bound).  The
    unit normal is taken only where |grad phi| > 1e-4: the perturbed members compress the flat bulk,
    where grad phi is of rounding size and its direction is set by rounding (with the default
    threshold, member 1 differs by 4.3e-5 in psi; with this one by 1.4e-7)."""
    stream = torch.cuda.Stream()
    cases = [(dict(p, n_eps=1e-4), f) for p, f in mixed_cases()]
    lats = make(torch, cases, stream)
    b = lbm.Batch(lats, stream)
    b.set_schedule("row_interleaved", 8)
    b.step(200)
    torch.cuda.synchronize()
    for k in (0, 1, 4):
        p, f = cases[k]
        o = oracle.Sim(p)
        o.init(**f)
        o.step(200)
        om, gm = o.moments(), lats[k].moments()
        for fld in ("phi", "psi"):
            err = np.linalg.norm(gm[fld] - om[fld]) / np.linalg.norm(om[fld])
            assert err <= 1e-5, (k, fld, err)
    b.close()


def test_config4_batch_sampled_members(torch):
    """The 64-lattice mix (sizes 128^2 .. 1024x512) for 20 steps: sampled members equal alone."""
    stream = torch.cuda.Stream()
    inst = W.batch_instances(64, seed=0)
    lats = make(torch, inst, stream)
    b = lbm.Batch(lats, stream)
    b.set_schedule("largest_first", 8)
    b.step(20)
    torch.cuda.synchronize()
    assert all(g.status == 0 for g in lats)
    for k in (0, 17, 63):
        assert lats[k].state() == alone_states(torch, [inst[k]], 20, stream)[0]
    b.close()


@pytest.mark.parametrize("kernel", ["tile", "pipelined"])
def test_batch_interior_tiles_of_uneven_members(torch, kernel):
    """Members of different sizes with interior tiles (cells and ring at least two cells from every
    edge, which take the kernels' interior path): a CTA must decide the path from its own member's
    grid, whichever member an SM ran before.  Every member equals the lattice stepped alone."""
    cases = []
    for (nx, ny), st in (((256, 128), "fp32"), ((96, 64), "fp32"), ((160, 48), "fp32"), ((200, 72), "fp16"),
                         ((128, 96), "fp16"), ((64, 40), "fp32")):
        p, f = W.shear_drop(nx, ny, R=min(nx, ny) / 5)
        cases.append((dict(p, storage=st), W.perturbed(p, f, seed=nx + ny)))
    stream = torch.cuda.Stream()
    ref = alone_states(torch, cases, 6, stream)
    lats = make(torch, cases, stream)
    b = lbm.Batch(lats, stream)
    b.kernel = kernel
    b.step(6)
    torch.cuda.synchronize()
    for k, g in enumerate(lats):
        assert g.status == lbm.LBM_OK, k
        assert g.state() == ref[k], k
    b.close()
    for g in lats:
        g.close()
