"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (same names, argument marshalling only).

Every step of the method runs in the CUDA library ``liblbm.so``; this module only converts
arguments.  PyTorch supplies device memory (the workspace and optional device field arrays) and
the CUDA stream.  If the library cannot be built or loaded, every call raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE = range(7)
LBM_BC_PERIODIC, LBM_BC_WALLS = 0, 1
LBM_EOS_LINEAR, LBM_EOS_LANGMUIR = 0, 1
LBM_STORE_FP32, LBM_STORE_FP16, LBM_STORE_BF16, LBM_STORE_FP16_FG, LBM_STORE_BF16_FG = 0, 1, 2, 3, 4
STORAGE = {"fp32": LBM_STORE_FP32, "fp16": LBM_STORE_FP16, "bf16": LBM_STORE_BF16,
           "fp16_fg": LBM_STORE_FP16_FG, "bf16_fg": LBM_STORE_BF16_FG}
LBM_MEM_HOST, LBM_MEM_DEVICE = 0, 1
LBM_VELOCITY_SOLVED, LBM_VELOCITY_PRESCRIBED = 0, 1
LBM_PHI, LBM_PSI, LBM_UX, LBM_UY, LBM_P = 1, 2, 4, 8, 16
LBM_SUM_PHI, LBM_SUM_PSI = 0, 1
LBM_NOALLOC_MAX_ROWS = 8192
LBM_SCHED_MEMBER_ORDER, LBM_SCHED_LARGEST_FIRST, LBM_SCHED_EDGES_FIRST, LBM_SCHED_ROW_INTERLEAVED = 0, 1, 2, 3
SCHEDULES = ("member_order", "largest_first", "edges_first", "row_interleaved")
LBM_SERVE_FCFS, LBM_SERVE_SHORTEST_FIRST = 0, 1
LBM_KERNEL_AUTO, LBM_KERNEL_TILE, LBM_KERNEL_PIPELINED = 0, 1, 2
KERNELS = {"auto": LBM_KERNEL_AUTO, "tile": LBM_KERNEL_TILE, "pipelined": LBM_KERNEL_PIPELINED}
POLICIES = {"fcfs": LBM_SERVE_FCFS, "shortest_first": LBM_SERVE_SHORTEST_FIRST}
FIELDS = ("phi", "psi", "ux", "uy", "P")

# Symbols declared in include/lbm.h (checked by the tests against the header and the library).
EXPORTS = ("lbm_workspace_bytes", "lbm_create", "lbm_init_fields", "lbm_step", "lbm_get_moments",
           "lbm_reduce", "lbm_reduce_noalloc", "lbm_status", "lbm_state_bytes", "lbm_get_state", "lbm_set_state",
           "lbm_steps_taken", "lbm_destroy", "lbm_last_error", "lbm_set_kernel", "lbm_get_kernel", "lbm_batch_tiles", "lbm_batch_workspace_bytes",
           "lbm_batch_create", "lbm_batch_set_members", "lbm_batch_set_schedule", "lbm_batch_step",
           "lbm_batch_autotune", "lbm_batch_launches", "lbm_batch_destroy", "lbm_server_workspace_bytes",
           "lbm_server_create", "lbm_server_submit", "lbm_server_poll", "lbm_server_get_stats",
           "lbm_server_destroy", "lbm_selftest_wait", "lbm_batch_set_kernel", "lbm_batch_get_kernel")


class lbm_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("bc_y", C.c_int32), ("eos", C.c_int32),
        ("storage", C.c_int32), ("velocity", C.c_int32),
        ("u_top", C.c_double), ("u_bot", C.c_double),
        ("phiA", C.c_double), ("phiB", C.c_double), ("rhoA", C.c_double), ("rhoB", C.c_double),
        ("muA", C.c_double), ("muB", C.c_double), ("W", C.c_double), ("M_phi", C.c_double),
        ("D", C.c_double), ("sigma0", C.c_double), ("E0", C.c_double), ("gx", C.c_double),
        ("gy", C.c_double), ("n_eps", C.c_double),
        ("s_f", C.c_double * 5), ("s_g", C.c_double * 5), ("s_h", C.c_double * 5),
    ]


class lbm_server_config(C.Structure):
    _fields_ = [("policy", C.c_int32), ("max_jobs", C.c_int32), ("max_cells", C.c_int64), ("max_tiles", C.c_int64),
                ("chunk_steps", C.c_int64), ("graph_steps", C.c_int32), ("schedule", C.c_int32)]


class lbm_job_result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("storage", C.c_int32), ("nx", C.c_int32),
                ("ny", C.c_int32), ("steps", C.c_int64), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("message", C.c_char * 128)]


class lbm_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("queued", C.c_int64), ("active", C.c_int64),
                ("lattice_updates", C.c_int64), ("rounds", C.c_int64), ("kernel_launches", C.c_int64),
                ("busy_seconds", C.c_double), ("now", C.c_double)]


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lbm error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str | None = None):
    """Load liblbm.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    lib = C.CDLL(path or _build.build())
    vp, dp, sz = C.c_void_p, C.POINTER(C.c_double), C.c_size_t
    P = C.POINTER(lbm_params)
    sig = {
        "lbm_workspace_bytes": [P, C.POINTER(sz)],
        "lbm_create": [P, vp, sz, vp, C.POINTER(vp)],
        "lbm_init_fields": [vp, vp, vp, vp, vp, vp, C.c_int],
        "lbm_step": [vp, C.c_int64],
        "lbm_get_moments": [vp, C.c_uint, C.POINTER(vp), C.c_int],
        "lbm_reduce": [vp, C.c_int, dp],
        "lbm_reduce_noalloc": [vp, C.c_int, C.c_int, C.c_int, vp, dp],
        "lbm_status": [vp],
        "lbm_state_bytes": [vp, C.POINTER(sz)],
        "lbm_get_state": [vp, vp, sz],
        "lbm_set_state": [vp, vp, sz],
        "lbm_steps_taken": [vp, C.POINTER(C.c_int64)],
        "lbm_destroy": [vp],
        "lbm_last_error": [],
        "lbm_set_kernel": [vp, C.c_int],
        "lbm_get_kernel": [vp, C.POINTER(C.c_int)],
        "lbm_batch_tiles": [C.POINTER(vp), C.c_int, C.POINTER(C.c_int64)],
        "lbm_batch_workspace_bytes": [C.c_int, C.c_int64, C.POINTER(sz)],
        "lbm_batch_create": [C.c_int, C.c_int64, vp, sz, vp, C.POINTER(vp)],
        "lbm_batch_set_members": [vp, C.POINTER(vp), C.c_int],
        "lbm_batch_set_schedule": [vp, C.c_int, C.c_int],
        "lbm_batch_step": [vp, C.c_int64],
        "lbm_batch_autotune": [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "lbm_batch_launches": [vp, C.POINTER(C.c_int64)],
        "lbm_batch_destroy": [vp],
        "lbm_server_workspace_bytes": [C.POINTER(lbm_server_config), sz, C.POINTER(sz)],
        "lbm_server_create": [C.POINTER(lbm_server_config), vp, sz, vp, C.POINTER(vp)],
        "lbm_server_submit": [vp, P, vp, vp, vp, vp, vp, C.c_int64, C.POINTER(vp), C.POINTER(C.c_int64)],
        "lbm_server_poll": [vp, C.POINTER(lbm_job_result), C.c_int, C.c_double, C.POINTER(C.c_int)],
        "lbm_server_get_stats": [vp, C.POINTER(lbm_server_stats)],
        "lbm_server_destroy": [vp],
        "lbm_selftest_wait": [vp, vp],
        "lbm_batch_set_kernel": [vp, C.c_int],
        "lbm_batch_get_kernel": [vp, C.POINTER(C.c_int)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_char_p if name == "lbm_last_error" else C.c_int
    if path is None:
        _lib = lib
    return lib


def lbm_last_error() -> str:
    return load().lbm_last_error().decode()


def _check(rc: int):
    if rc != LBM_OK:
        raise LBMError(rc, lbm_last_error())


def make_params(p: dict) -> lbm_params:
    """Marshal a workload parameter dict into ``lbm_params``."""
    q = lbm_params()
    q.nx, q.ny = int(p["nx"]), int(p["ny"])
    q.bc_y = LBM_BC_WALLS if p.get("walls", False) else LBM_BC_PERIODIC
    q.eos = LBM_EOS_LANGMUIR if p.get("eos", "linear") == "langmuir" else LBM_EOS_LINEAR
    st = p.get("storage", LBM_STORE_FP32)
    q.storage = STORAGE[st] if isinstance(st, str) else int(st)
    v = p.get("velocity", "solved")
    q.velocity = int(v) if not isinstance(v, str) else {"solved": LBM_VELOCITY_SOLVED,
                                                        "prescribed": LBM_VELOCITY_PRESCRIBED}[v]
    for k in ("u_top", "u_bot", "phiA", "phiB", "rhoA", "rhoB", "muA", "muB", "W", "M_phi", "D",
              "sigma0", "E0", "gx", "gy", "n_eps"):
        setattr(q, k, float(p[k]))
    for k in ("s_f", "s_g", "s_h"):
        arr = getattr(q, k)
        for i, v in enumerate(p[k]):
            arr[i] = float(v)
    return q


def lbm_workspace_bytes(params: lbm_params) -> int:
    n = C.c_size_t()
    _check(load().lbm_workspace_bytes(C.byref(params), C.byref(n)))
    return n.value


def lbm_create(params: lbm_params, workspace_ptr: int, nbytes: int, stream_ptr: int) -> int:
    h = C.c_void_p()
    _check(load().lbm_create(C.byref(params), C.c_void_p(workspace_ptr), nbytes, C.c_void_p(stream_ptr),
                             C.byref(h)))
    return h.value


def _ptr(a, mem: int):
    if mem == LBM_MEM_HOST:
        assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
        return C.c_void_p(a.ctypes.data)
    return C.c_void_p(a.data_ptr())


def lbm_init_fields(h: int, phi, psi, ux, uy, P, mem: int = LBM_MEM_HOST):
    _check(load().lbm_init_fields(C.c_void_p(h), *[_ptr(a, mem) for a in (phi, psi, ux, uy, P)], mem))


def lbm_step(h: int, n: int):
    _check(load().lbm_step(C.c_void_p(h), int(n)))


def lbm_get_moments(h: int, mask: int, outs, mem: int = LBM_MEM_HOST):
    arr = (C.c_void_p * 5)(*[(_ptr(o, mem) if o is not None else None) for o in outs])
    _check(load().lbm_get_moments(C.c_void_p(h), mask, arr, mem))


def lbm_reduce(h: int, what: int) -> float:
    v = C.c_double()
    _check(load().lbm_reduce(C.c_void_p(h), what, C.byref(v)))
    return v.value


def lbm_reduce_noalloc(d_pops: int, nx: int, ny: int, what: int, stream_ptr: int) -> float:
    v = C.c_double()
    _check(load().lbm_reduce_noalloc(C.c_void_p(d_pops), int(nx), int(ny), int(what), C.c_void_p(stream_ptr),
                                     C.byref(v)))
    return v.value


def lbm_selftest_wait(d_word: int, stream_ptr: int) -> int:
    """The failure-detection self-test (a bounded wait that must give up); returns the status code."""
    return load().lbm_selftest_wait(C.c_void_p(d_word), C.c_void_p(stream_ptr))


def lbm_status(h: int) -> int:
    return load().lbm_status(C.c_void_p(h))


def lbm_state_bytes(h: int) -> int:
    n = C.c_size_t()
    _check(load().lbm_state_bytes(C.c_void_p(h), C.byref(n)))
    return n.value


def lbm_get_state(h: int) -> bytes:
    n = lbm_state_bytes(h)
    buf = C.create_string_buffer(n)
    _check(load().lbm_get_state(C.c_void_p(h), buf, n))
    return buf.raw


def lbm_set_state(h: int, blob: bytes):
    _check(load().lbm_set_state(C.c_void_p(h), C.c_char_p(blob), len(blob)))


def lbm_steps_taken(h: int) -> int:
    v = C.c_int64()
    _check(load().lbm_steps_taken(C.c_void_p(h), C.byref(v)))
    return v.value


def lbm_destroy(h: int):
    _check(load().lbm_destroy(C.c_void_p(h)))


class Lattice:
    """One simulation on the current CUDA device: a torch-allocated workspace plus a handle.

    ``params`` is a workload dict (see ``workloads``); ``stream`` a torch CUDA stream (default:
    the current stream)."""

    def __init__(self, params: dict, stream=None):
        import torch

        self.params = dict(params)
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self._p = make_params(params)
        nbytes = lbm_workspace_bytes(self._p)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = lbm_create(self._p, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            lbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi, psi, ux, uy, P):
        arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (self.ny, self.nx)))
                for a in (phi, psi, ux, uy, P)]
        lbm_init_fields(self.handle, *arrs, mem=LBM_MEM_HOST)

    def step(self, n: int = 1):
        lbm_step(self.handle, n)

    def moments(self, mask: int = 31) -> dict:
        outs = [np.zeros((self.ny, self.nx)) if mask & (1 << k) else None for k in range(5)]
        lbm_get_moments(self.handle, mask, outs, LBM_MEM_HOST)
        return {FIELDS[k]: outs[k] for k in range(5) if outs[k] is not None}

    def total(self, what: str) -> float:
        return lbm_reduce(self.handle, LBM_SUM_PHI if what == "phi" else LBM_SUM_PSI)

    @property
    def status(self) -> int:
        return lbm_status(self.handle)

    def state(self) -> bytes:
        return lbm_get_state(self.handle)

    def restore(self, blob: bytes):
        lbm_set_state(self.handle, blob)

    @property
    def steps(self) -> int:
        return lbm_steps_taken(self.handle)

    @property
    def kernel(self) -> str:
        v = C.c_int()
        _check(load().lbm_get_kernel(C.c_void_p(self.handle), C.byref(v)))
        return {LBM_KERNEL_TILE: "tile", LBM_KERNEL_PIPELINED: "pipelined"}[v.value]

    @kernel.setter
    def kernel(self, name: str):
        _check(load().lbm_set_kernel(C.c_void_p(self.handle), KERNELS[name]))


def _handles(members):
    return (C.c_void_p * max(1, len(members)))(*[C.c_void_p(m) for m in members])


def lbm_batch_tiles(members) -> int:
    v = C.c_int64()
    _check(load().lbm_batch_tiles(_handles(members), len(members), C.byref(v)))
    return v.value


def lbm_batch_workspace_bytes(max_members: int, max_tiles: int) -> int:
    n = C.c_size_t()
    _check(load().lbm_batch_workspace_bytes(int(max_members), int(max_tiles), C.byref(n)))
    return n.value


def lbm_batch_create(max_members: int, max_tiles: int, workspace_ptr: int, nbytes: int, stream_ptr: int) -> int:
    b = C.c_void_p()
    _check(load().lbm_batch_create(int(max_members), int(max_tiles), C.c_void_p(workspace_ptr), nbytes,
                                   C.c_void_p(stream_ptr), C.byref(b)))
    return b.value


def lbm_batch_set_members(b: int, members):
    _check(load().lbm_batch_set_members(C.c_void_p(b), _handles(members), len(members)))


def lbm_batch_set_schedule(b: int, schedule: int, graph_steps: int):
    _check(load().lbm_batch_set_schedule(C.c_void_p(b), int(schedule), int(graph_steps)))


def lbm_batch_step(b: int, n: int):
    _check(load().lbm_batch_step(C.c_void_p(b), int(n)))


def lbm_batch_autotune(b: int, trial_steps: int):
    s, k = C.c_int(), C.c_int()
    _check(load().lbm_batch_autotune(C.c_void_p(b), int(trial_steps), C.byref(s), C.byref(k)))
    return s.value, k.value


def lbm_batch_set_kernel(b: int, variant: int):
    _check(load().lbm_batch_set_kernel(C.c_void_p(b), int(variant)))


def lbm_batch_get_kernel(b: int) -> int:
    v = C.c_int()
    _check(load().lbm_batch_get_kernel(C.c_void_p(b), C.byref(v)))
    return v.value


def lbm_batch_launches(b: int) -> int:
    v = C.c_int64()
    _check(load().lbm_batch_launches(C.c_void_p(b), C.byref(v)))
    return v.value


def lbm_batch_destroy(b: int):
    _check(load().lbm_batch_destroy(C.c_void_p(b)))


class Batch:
    """Many ``Lattice`` objects advanced together (one launch per step and member group).

    All members must use the batch's stream.  ``capacity`` bounds the member count and
    ``max_tiles`` the total tile count (default: exactly what ``lattices`` need)."""

    def __init__(self, lattices, stream, capacity=None, max_tiles=None):
        import torch

        self.lattices = list(lattices)
        handles = [m.handle for m in self.lattices]
        capacity = capacity or max(1, len(handles))
        max_tiles = max_tiles or max(1, lbm_batch_tiles(handles))
        nbytes = lbm_batch_workspace_bytes(capacity, max_tiles)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream
        self.handle = lbm_batch_create(capacity, max_tiles, self.workspace.data_ptr(), nbytes, stream.cuda_stream)
        lbm_batch_set_members(self.handle, handles)

    def set_members(self, lattices):
        self.lattices = list(lattices)
        lbm_batch_set_members(self.handle, [m.handle for m in self.lattices])

    def set_schedule(self, schedule, graph_steps=0):
        if isinstance(schedule, str):
            schedule = SCHEDULES.index(schedule)
        lbm_batch_set_schedule(self.handle, schedule, graph_steps)

    def step(self, n: int = 1):
        lbm_batch_step(self.handle, n)

    def autotune(self, trial_steps: int = 32):
        s, k = lbm_batch_autotune(self.handle, trial_steps)
        return SCHEDULES[s], k

    @property
    def launches(self) -> int:
        return lbm_batch_launches(self.handle)

    @property
    def kernel(self) -> str:
        return {v: k for k, v in KERNELS.items()}[lbm_batch_get_kernel(self.handle)]

    @kernel.setter
    def kernel(self, name: str):
        lbm_batch_set_kernel(self.handle, KERNELS[name])

    def close(self):
        if getattr(self, "handle", None):
            lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_server_workspace_bytes(cfg: lbm_server_config, job_arena_bytes: int) -> int:
    n = C.c_size_t()
    _check(load().lbm_server_workspace_bytes(C.byref(cfg), int(job_arena_bytes), C.byref(n)))
    return n.value


def lbm_server_create(cfg: lbm_server_config, workspace_ptr: int, nbytes: int, stream_ptr: int) -> int:
    h = C.c_void_p()
    _check(load().lbm_server_create(C.byref(cfg), C.c_void_p(workspace_ptr), nbytes, C.c_void_p(stream_ptr),
                                    C.byref(h)))
    return h.value


def lbm_server_submit(s: int, params: lbm_params, fields, steps: int, outs) -> int:
    v = C.c_int64()
    arr = (C.c_void_p * 5)(*[(C.c_void_p(o.ctypes.data) if o is not None else None) for o in outs])
    _check(load().lbm_server_submit(C.c_void_p(s), C.byref(params), *[C.c_void_p(a.ctypes.data) for a in fields],
                                    int(steps), arr, C.byref(v)))
    return v.value


def lbm_server_poll(s: int, max_results: int, timeout_s: float):
    buf = (lbm_job_result * max(1, max_results))()
    n = C.c_int()
    _check(load().lbm_server_poll(C.c_void_p(s), buf, int(max_results), float(timeout_s), C.byref(n)))
    return [buf[k] for k in range(n.value)]


def lbm_server_get_stats(s: int) -> dict:
    st = lbm_server_stats()
    _check(load().lbm_server_get_stats(C.c_void_p(s), C.byref(st)))
    return {f: getattr(st, f) for f, _ in lbm_server_stats._fields_}


def lbm_server_destroy(s: int):
    _check(load().lbm_server_destroy(C.c_void_p(s)))


class Server:
    """A lattice server on the current device: jobs run by a native worker thread in one
    continuously re-formed batch.  ``arena_bytes`` of device memory hold the job workspaces."""

    def __init__(self, arena_bytes: int, stream, policy="fcfs", max_jobs=64, max_cells=1 << 24,
                 max_tiles=1 << 20, chunk_steps=100, graph_steps=16, schedule="largest_first"):
        import torch

        cfg = lbm_server_config()
        cfg.policy = POLICIES[policy] if isinstance(policy, str) else int(policy)
        cfg.max_jobs, cfg.max_cells, cfg.max_tiles = int(max_jobs), int(max_cells), int(max_tiles)
        cfg.chunk_steps, cfg.graph_steps = int(chunk_steps), int(graph_steps)
        cfg.schedule = SCHEDULES.index(schedule) if isinstance(schedule, str) else int(schedule)
        nbytes = lbm_server_workspace_bytes(cfg, arena_bytes)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream
        self.handle = lbm_server_create(cfg, self.workspace.data_ptr(), nbytes, stream.cuda_stream)
        self._jobs = {}

    def submit(self, params: dict, fields: dict, steps: int, outputs: bool = True) -> int:
        ny, nx = int(params["ny"]), int(params["nx"])
        ins = [np.ascontiguousarray(np.broadcast_to(np.asarray(fields[k], dtype=np.float64), (ny, nx)))
               for k in FIELDS]
        outs = [np.empty((ny, nx)) for _ in FIELDS] if outputs else [None] * 5
        jid = lbm_server_submit(self.handle, make_params(params), ins, steps, outs)
        self._jobs[jid] = (ins, outs)  # kept alive until the result is polled
        return jid

    def poll(self, max_results: int = 64, timeout: float = 0.0) -> list:
        out = []
        for r in lbm_server_poll(self.handle, max_results, timeout):
            ins, outs = self._jobs.pop(r.id)
            d = {f: getattr(r, f) for f, _ in lbm_job_result._fields_ if f != "message"}
            d["message"] = r.message.decode(errors="replace")
            d["moments"] = {FIELDS[k]: outs[k] for k in range(5) if outs[k] is not None}
            out.append(d)
        return out

    def stats(self) -> dict:
        return lbm_server_get_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            lbm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
