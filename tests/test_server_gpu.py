"""The lattice server: every job's final fields are bit for bit those of the same lattice stepped
alone (whatever else shares its rounds), admission follows the policy, a failing job ends alone
with its status, and the counters add up."""
import time

import numpy as np
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


def jobs_mix():
    out = []
    p, f = W.shear_drop(96, 40, R=9)
    out.append((p, f, 37))
    p, f = W.stationary_drop(70, 50, R=12)
    out.append((dict(p, storage="fp16"), W.perturbed(p, f, seed=1), 50))
    p, f = W.shear_drop(45, 19, R=6)
    out.append((dict(p, storage="bf16_fg"), W.perturbed(p, f, seed=2), 23))
    p, f = W.stationary_drop(64, 64, R=14)
    out.append((p, f, 64))
    p, f = W.shear_drop(20, 6, R=2.5)
    out.append((p, W.perturbed(p, f, seed=3), 11))
    return out


def alone(torch, p, f, steps):
    g = lbm.Lattice(p, stream=torch.cuda.Stream())
    g.init(**f)
    g.step(steps)
    m = g.moments()
    g.close()
    return m


def collect(srv, n, timeout=120.0):
    res = []
    t0 = time.time()
    while len(res) < n and time.time() - t0 < timeout:
        res += srv.poll(64, timeout=1.0)
    assert len(res) == n, f"{len(res)} of {n} results"
    return res


@pytest.mark.parametrize("policy,max_jobs,chunk,graph", [("fcfs", 2, 7, 0), ("shortest_first", 3, 16, 4),
                                                         ("fcfs", 8, 1000, 8)])
def test_server_results_equal_alone(torch, policy, max_jobs, chunk, graph):
    srv = lbm.Server(64 << 20, torch.cuda.Stream(), policy=policy, max_jobs=max_jobs, chunk_steps=chunk,
                     graph_steps=graph)
    jobs = jobs_mix()
    ids = [srv.submit(p, f, n) for p, f, n in jobs]
    res = {r["id"]: r for r in collect(srv, len(jobs))}
    for jid, (p, f, n) in zip(ids, jobs):
        r = res[jid]
        assert r["status"] == lbm.LBM_OK, r["message"]
        assert r["steps"] == n and r["t_submit"] <= r["t_admit"] <= r["t_done"]
        ref = alone(torch, p, f, n)
        for k in lbm.FIELDS:
            assert np.array_equal(r["moments"][k], ref[k]), (jid, k)
    st = srv.stats()
    assert st["completed"] == st["submitted"] == len(jobs)
    assert st["queued"] == 0 and st["active"] == 0
    assert st["lattice_updates"] == sum(p["nx"] * p["ny"] * n for p, _, n in jobs)
    assert st["kernel_launches"] > 0
    srv.close()


def test_policies_order_completions(torch):
    """One job at a time: FCFS finishes in submission order, shortest-first by work."""
    p, f = W.stationary_drop(64, 64, R=14)
    steps = [60, 10, 30, 20]
    for policy in ("fcfs", "shortest_first"):
        srv = lbm.Server(64 << 20, torch.cuda.Stream(), policy=policy, max_jobs=1, chunk_steps=8)
        # hold the worker on a long first job so that the others queue up behind it
        first = srv.submit(*W.stationary_drop(128, 128)[:2], 400, outputs=False)
        t0 = time.time()
        while srv.stats()["active"] == 0 and time.time() - t0 < 30.0:
            time.sleep(0.001)
        ids = [srv.submit(p, f, n, outputs=False) for n in steps]
        order = [r["id"] for r in collect(srv, 5)]
        assert order[0] == first
        want = ids if policy == "fcfs" else [ids[k] for k in np.argsort(steps)]
        assert order[1:] == want, policy
        srv.close()


def test_failing_jobs_end_alone(torch):
    srv = lbm.Server(64 << 20, torch.cuda.Stream(), max_jobs=4, chunk_steps=10)
    good_p, good_f = W.stationary_drop(64, 64, R=14)
    bad_f = dict(good_f, phi=np.full((64, 64), np.nan))               # rejected at initialisation
    fast_p, fast_f = W.stationary_drop(40, 24, R=6)
    fast_f = dict(fast_f, ux=np.full((24, 40), 0.35))                 # |u| >= 0.3: unstable
    ids = [srv.submit(good_p, good_f, 30), srv.submit(good_p, bad_f, 30), srv.submit(fast_p, fast_f, 5),
           srv.submit(good_p, good_f, 40)]
    res = {r["id"]: r for r in collect(srv, 4)}
    assert res[ids[0]]["status"] == lbm.LBM_OK and res[ids[3]]["status"] == lbm.LBM_OK
    assert res[ids[1]]["status"] == lbm.LBM_EINVAL and res[ids[1]]["message"]
    assert res[ids[2]]["status"] == lbm.LBM_EUNSTABLE
    ref = alone(torch, good_p, good_f, 40)
    assert np.array_equal(res[ids[3]]["moments"]["phi"], ref["phi"])
    srv.close()


def test_submit_rejects_jobs_that_never_fit(torch):
    srv = lbm.Server(1 << 20, torch.cuda.Stream(), max_tiles=64)
    p, f = W.stationary_drop(128, 128)
    with pytest.raises(lbm.LBMError):
        srv.submit(p, f, 10)             # 3.7 MB workspace > 1 MB arena
    p, f = W.stationary_drop(16, 16, R=4)
    with pytest.raises(lbm.LBMError):
        srv.submit(p, f, 0)
    bad = dict(p, W=0.0)
    with pytest.raises(lbm.LBMError):
        srv.submit(bad, f, 10)
    srv.close()


def test_close_with_work_pending_returns(torch):
    srv = lbm.Server(256 << 20, torch.cuda.Stream(), max_jobs=1, chunk_steps=50)
    p, f = W.stationary_drop(256, 256)
    for _ in range(3):
        srv.submit(p, f, 100000, outputs=False)
    time.sleep(0.5)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 30.0
