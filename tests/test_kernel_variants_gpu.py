"""The two step kernels (one CTA per tile; persistent CTAs with a double-buffered TMA pipeline)
compute the same step bit for bit, in every storage mode and flow variant, on ragged and full-size
grids; the comparison covers the whole state, ghost frame included.  The 16-bit modes update two
horizontally adjacent cells per thread, so odd widths (a thread whose second cell lies beyond the
grid) are among the cases, with walls and with periodic images in y."""
import pytest

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


def cases():
    p, f = W.shear_drop(96, 40, R=9)
    yield "shear_96x40", p, f
    p, f = W.stationary_drop(70, 50, R=12)
    yield "periodic_70x50_perturbed", p, W.perturbed(p, f, seed=1)
    p, f = W.shear_drop(45, 19, R=6)
    yield "walls_45x19_perturbed", p, W.perturbed(p, f, seed=2)
    p, f = W.shear_drop(20, 6, R=2.5)
    yield "below_one_tile", p, f
    # a width that is a multiple of the tile width: every tile column is whole
    p, f = W.stationary_drop(64, 37, R=10)
    yield "periodic_64x37_perturbed", p, W.perturbed(p, f, seed=5)
    # odd width, periodic in y: the last thread of a row has one cell, and its images wrap in y
    p, f = W.stationary_drop(45, 21, R=7)
    yield "periodic_45x21_perturbed", p, W.perturbed(p, f, seed=7)
    p, f = W.rising_bubble(7.0)
    yield "density_ratio_walls_28x56_perturbed", p, W.perturbed(p, f, seed=3)
    p, f = W.rising_bubble(8.0)
    yield "density_ratio_walls_32x64_perturbed", p, W.perturbed(p, f, seed=6)
    yield "density_ratio_periodic_32x64_perturbed", dict(p, walls=False), W.perturbed(p, f, seed=4)
    p, f = W.convected_drop(70, 45, R=10)
    yield "prescribed_70x45", p, f
    p, f = W.convected_drop(64, 45, R=10)
    yield "prescribed_64x45", p, f


def run(torch, p, f, kernel, steps):
    g = lbm.Lattice(p)
    g.kernel = kernel
    g.init(**f)
    g.step(steps)
    torch.cuda.synchronize()
    assert g.kernel == kernel
    s = g.state()
    g.close()
    return s


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16", "fp16_fg", "bf16_fg"])
def test_pipelined_equals_tile(torch, storage):
    for name, p, f in cases():
        q = dict(p, storage=storage)
        g = lbm.Lattice(q)
        try:
            g.kernel = "pipelined"
        except lbm.LBMError:
            pytest.skip(f"the pipelined kernel does not fit for {storage}")
        finally:
            g.close()
        assert run(torch, q, f, "tile", 9) == run(torch, q, f, "pipelined", 9), name


@pytest.mark.parametrize("storage", ["fp16", "bf16_fg"])
def test_pipelined_equals_tile_full_size(torch, storage):
    """2048 x 1024: every persistent CTA takes 13 or 14 tiles through both pipeline stages."""
    p, f = W.shear_drop_large()
    q = dict(p, storage=storage)
    assert run(torch, q, f, "tile", 5) == run(torch, q, f, "pipelined", 5)


def test_default_kernel_per_storage(torch):
    p, f = W.stationary_drop(64, 64, R=14)
    got = {}
    for st in ("fp32", "fp16", "bf16", "fp16_fg", "bf16_fg"):
        g = lbm.Lattice(dict(p, storage=st))
        got[st] = g.kernel
        g.kernel = "auto"
        assert g.kernel == got[st]
        g.close()
    # at uniform density: FP32 is bandwidth-bound either way and keeps the one-tile kernel; the
    # 16-bit modes take the warp-specialised kernel, which stages one tile ahead
    assert got == {"fp32": "tile", "fp16": "pipelined", "bf16": "pipelined", "fp16_fg": "pipelined",
                   "bf16_fg": "pipelined"}
    # with a prescribed velocity (no flow populations) the same choice
    p, f = W.convected_drop(64, 64, R=10.0)
    for st, kn in (("fp32", "tile"), ("fp16", "pipelined"), ("bf16_fg", "pipelined")):
        g = lbm.Lattice(dict(p, storage=st))
        assert g.kernel == kn, st
        g.close()
    # a density ratio != 1 takes the warp-specialised kernel in every storage mode
    p, f = W.rising_bubble(8.0)
    for st in ("fp32", "fp16", "bf16_fg"):
        g = lbm.Lattice(dict(p, storage=st))
        assert g.kernel == "pipelined", st
        g.close()


def smallest_grids():
    """The smallest grids the library accepts (nx = ny = 2, or two fluid rows between walls), and a
    width of three: every cell is an edge cell and writes its periodic images or wall ghosts on
    several sides, and one tile covers the grid many times over."""
    p, f = W.stationary_drop(2, 2, R=0.6)
    yield "periodic_2x2", p, W.perturbed(p, f, seed=11)
    p, f = W.shear_drop(2, 2, R=0.6)
    yield "walls_2x2", p, W.perturbed(p, f, seed=12)
    p, f = W.shear_drop(3, 2, R=0.6)
    yield "walls_3x2", p, W.perturbed(p, f, seed=13)
    p, f = W.convected_drop(2, 3, R=0.6)
    yield "prescribed_2x3", p, f
    # density ratio 10 with gravity (the rising bubble's parameters at R = 8) on the smallest grids
    pb, _ = W.rising_bubble(8.0)
    for nx, ny, walls in ((2, 4, True), (3, 2, True), (2, 2, False)):
        q = dict(pb, nx=nx, ny=ny, walls=walls)
        _, g0 = W.stationary_drop(nx, ny, R=0.6)
        yield f"density_ratio_{'walls' if walls else 'periodic'}_{nx}x{ny}", q, W.perturbed(q, g0, seed=14 + nx + ny)


@pytest.mark.parametrize("kernel", ["tile", "pipelined"])
def test_smallest_grids_match_oracle(torch, kernel):
    """FP32 storage on the smallest grids against the FP64 oracle after 100 steps (the FP32 parity
    bound of the larger cases), through both kernels.  The unit normal is taken only where
    |grad phi| > 1e-4, as in the other long parity runs: on the 2 x 2 channel the gradients are of
    rounding size, and with the default threshold the oracle's own u moves by up to 1.5e-6 when its
    inputs are perturbed at FP32 rounding size (6e-8 relative), against 2e-10 with this one."""
    import numpy as np
    import oracle
    for name, p, f in smallest_grids():
        p = dict(p, n_eps=1e-4)
        g = lbm.Lattice(p)
        g.kernel = kernel
        g.init(**f)
        g.step(100)
        torch.cuda.synchronize()
        assert g.status == lbm.LBM_OK, name
        gm = g.moments()
        g.close()
        o = oracle.Sim(p)
        o.init(**f)
        o.step(100)
        om = o.moments()
        for k in ("phi", "psi"):
            err = np.linalg.norm(gm[k] - om[k]) / np.linalg.norm(om[k])
            assert err <= 1e-5, (name, k, err)
        du = np.hypot(gm["ux"] - om["ux"], gm["uy"] - om["uy"]).max()
        assert du <= 1e-5 * max(np.hypot(om["ux"], om["uy"]).max(), 1e-3), (name, du)


@pytest.mark.parametrize("storage", ["fp16", "bf16_fg"])
def test_smallest_grids_16bit_kernels_agree(torch, storage):
    """16-bit storage on the smallest grids: both kernels give the same state bit for bit, the run
    stays stable, and the total of phi moves only by the stochastic rounding's random walk."""
    for name, p, f in smallest_grids():
        q = dict(p, storage=storage)
        assert run(torch, q, f, "tile", 50) == run(torch, q, f, "pipelined", 50), name
        g = lbm.Lattice(q)
        g.init(**f)
        t0 = g.total("phi")
        g.step(50)
        torch.cuda.synchronize()
        assert g.status == lbm.LBM_OK, name
        assert abs(g.total("phi") - t0) <= 1e-2 * abs(t0), name
        g.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_smallest_grids_in_a_batch_equal_alone(torch, storage):
    """The smallest grids as members of one batch (one launch per group and step, both batch
    kernels): every member equals the lattice stepped alone, bit for bit."""
    cases = [(dict(p, storage=storage), f) for _, p, f in smallest_grids()]
    ref = []
    for p, f in cases:
        g = lbm.Lattice(p)
        g.init(**f)
        g.step(20)
        torch.cuda.synchronize()
        ref.append(g.state())
        g.close()
    for kernel in ("tile", "pipelined"):
        stream = torch.cuda.Stream()
        lats = []
        for p, f in cases:
            g = lbm.Lattice(p, stream=stream)
            g.init(**f)
            lats.append(g)
        b = lbm.Batch(lats, stream)
        b.kernel = kernel
        b.step(20)
        torch.cuda.synchronize()
        for k, g in enumerate(lats):
            assert g.status == lbm.LBM_OK, (kernel, k)
            assert g.state() == ref[k], (kernel, k)
        b.close()
        for g in lats:
            g.close()
