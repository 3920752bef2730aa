"""lbm_reduce_noalloc, the FP64 sum for callers that cannot allocate device memory, checked
against lbm_reduce through the C ABI (needs a GPU).

Such a caller (a plugin whose host application owns all device memory, or code that must not
allocate while other work is in flight) hands the library a population buffer it already holds;
the partial sums then live in a fixed device array inside the library.  This file is collected
last so that a run stopping at the first failure has already run every other test; it also runs
on its own in a fresh process, where its first call performs the per-device set-up.
"""
import numpy as np
import pytest

from paper_2408_15654_gb300 import lbm
from paper_2408_15654_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load()
    yield


def current_buffer(sim: "lbm.Lattice") -> int:
    """Device address of the handle's current population buffer (layout of lbm_workspace_bytes)."""
    pitch = (sim.nx + 10 + 31) // 32 * 32  # the grid inside its ghost frame
    buf = (26 * (sim.ny + 4) * pitch * 4 + 255) // 256 * 256
    return sim.workspace.data_ptr() + (sim.steps % 2) * buf


@pytest.mark.parametrize("nx,ny,steps", [(96, 40, 7), (64, 1500, 4)])
def test_noalloc_sum_matches_lbm_reduce_on_two_calls(nx, ny, steps):
    p, f = W.shear_drop(nx, ny, R=min(nx, ny) / 4)
    f = W.perturbed(p, f, seed=9)
    sim = lbm.Lattice(p)
    sim.init(**f)
    sim.step(steps)
    stream = sim.stream.cuda_stream
    for what in (lbm.LBM_SUM_PHI, lbm.LBM_SUM_PSI):
        expect = lbm.lbm_reduce(sim.handle, what)
        first = lbm.lbm_reduce_noalloc(current_buffer(sim), nx, ny, what, stream)
        second = lbm.lbm_reduce_noalloc(current_buffer(sim), nx, ny, what, stream)
        assert first == second  # the second call starts from the first call's scratch contents
        assert first == pytest.approx(expect, rel=1e-12, abs=1e-12)
    # the state is untouched: the handle keeps stepping and its own sum still agrees
    sim.step(1)
    assert lbm.lbm_reduce_noalloc(current_buffer(sim), nx, ny, lbm.LBM_SUM_PHI, stream) == pytest.approx(
        lbm.lbm_reduce(sim.handle, lbm.LBM_SUM_PHI), rel=1e-12)
    sim.close()


def test_noalloc_rejects_grids_beyond_its_fixed_scratch():
    p, f = W.stationary_drop(32, 32, R=8)
    sim = lbm.Lattice(p)
    sim.init(**f)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_reduce_noalloc(current_buffer(sim), 32, lbm.LBM_NOALLOC_MAX_ROWS + 1, lbm.LBM_SUM_PHI,
                               sim.stream.cuda_stream)
    assert ei.value.code == lbm.LBM_EINVAL
    assert "fixed scratch" in str(ei.value)
    assert np.isfinite(lbm.lbm_reduce_noalloc(current_buffer(sim), 32, 32, lbm.LBM_SUM_PSI, sim.stream.cuda_stream))
    sim.close()
