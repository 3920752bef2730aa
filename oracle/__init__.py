"""FP64 CPU oracle of the three-population lattice-Boltzmann step (arXiv 2408.15654).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` load it; the CUDA library never does.  The C source (``lbm_oracle.c``) follows the
paper's Secs. 2-4 step by step in double precision; this module compiles it with gcc on first use
and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_HDR = os.path.join(_HERE, "lbm_oracle.h")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

EOS_LINEAR = 0
EOS_LANGMUIR = 1


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("walls", C.c_int), ("eos", C.c_int),
        ("u_top", C.c_double), ("u_bot", C.c_double),
        ("phiA", C.c_double), ("phiB", C.c_double), ("rhoA", C.c_double), ("rhoB", C.c_double),
        ("muA", C.c_double), ("muB", C.c_double),
        ("W", C.c_double), ("M_phi", C.c_double), ("D", C.c_double),
        ("sigma0", C.c_double), ("E0", C.c_double),
        ("gx", C.c_double), ("gy", C.c_double), ("rho0", C.c_double), ("n_eps", C.c_double),
        ("s_f", C.c_double * 5), ("s_g", C.c_double * 5), ("s_h", C.c_double * 5),
        ("prescribed", C.c_int),
    ]


class CellIn(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "phi", "psi", "ux", "uy", "P", "rho", "nx", "ny", "Fx", "Fy", "Sx", "Sy",
        "drho_x", "drho_y", "dt_phiux", "dt_phiuy", "dt_psiux", "dt_psiuy",
        "dt_m2_xx", "dt_m2_xy", "dt_m2_yy")]


class CellOut(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "phi", "psi", "ux", "uy", "P", "gpx", "gpy", "lap", "gsx", "gsy", "Fx", "Fy", "Fmx", "Fmy")]


_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP) into ``oracle/_build``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD_DIR)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_variant(name: str, substitutions) -> str:
    """Compile a copy of the oracle with text substitutions [(old, new), ...] into
    ``oracle/_build/variants/<name>`` and return its path.  Tests use it to plant a mistake in the
    oracle and show that a pin catches it; nothing else loads a variant."""
    src = open(_SRC).read()
    for old, new in substitutions:
        if old not in src:
            raise ValueError(f"variant {name}: text to replace not found: {old!r}")
        src = src.replace(old, new)
    d = os.path.join(_BUILD_DIR, "variants", name)
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, "lbm_oracle.c"), "w") as fh:
        fh.write(src)
    out = os.path.join(d, "liboracle.so")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-I", os.path.dirname(_HDR), "-o", out, os.path.join(d, "lbm_oracle.c"), "-lm"]
    subprocess.run(cmd, check=True)
    return out


_variants = {}


def _load(path: str | None = None):
    global _lib
    if path is not None:
        if path not in _variants:
            _variants[path] = _bind(C.CDLL(path))
        return _variants[path]
    if _lib is not None:
        return _lib
    _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(lib):
    dp = C.POINTER(C.c_double)
    lib.orc_create.restype = C.c_void_p
    lib.orc_create.argtypes = [C.POINTER(_Params)]
    lib.orc_destroy.argtypes = [C.c_void_p]
    lib.orc_init.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
    lib.orc_step.argtypes = [C.c_void_p, C.c_long]
    lib.orc_moments.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
    lib.orc_fields.argtypes = [C.c_void_p, C.POINTER(CellOut)]
    lib.orc_sum.restype = C.c_double
    lib.orc_sum.argtypes = [C.c_void_p, C.c_int]
    lib.orc_populations.argtypes = [C.c_void_p, dp, dp, dp]
    lib.orc_status.argtypes = [C.c_void_p]
    lib.orc_steps.restype = C.c_long
    lib.orc_steps.argtypes = [C.c_void_p]
    lib.orc_set_threads.argtypes = [C.c_int]
    lib.orc_cell_distributions.argtypes = [C.POINTER(_Params), C.POINTER(CellIn)] + [dp] * 6
    lib.orc_operators.argtypes = [dp, dp, dp]
    lib.orc_moment_matrix.argtypes = [dp]
    lib.orc_lattice.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(p: dict) -> _Params:
    """Marshal a workload parameter dict (see ``paper_2408_15654_gb300.workloads``)."""
    q = _Params()
    q.nx, q.ny = int(p["nx"]), int(p["ny"])
    q.walls = 1 if p.get("walls", False) else 0
    q.eos = EOS_LANGMUIR if p.get("eos", "linear") == "langmuir" else EOS_LINEAR
    q.prescribed = 1 if p.get("velocity", "solved") == "prescribed" else 0
    for k in ("u_top", "u_bot", "phiA", "phiB", "rhoA", "rhoB", "muA", "muB", "W", "M_phi", "D",
              "sigma0", "E0", "gx", "gy", "rho0", "n_eps"):
        setattr(q, k, float(p[k]))
    for k in ("s_f", "s_g", "s_h"):
        arr = getattr(q, k)
        for i, v in enumerate(p[k]):
            arr[i] = float(v)
    return q


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of the oracle (0 keeps the current); returns the count in use."""
    return _load().orc_set_threads(int(n))


def lattice():
    lib = _load()
    cx = (C.c_int * 9)()
    cy = (C.c_int * 9)()
    w = np.zeros(9)
    lib.orc_lattice(cx, cy, _dp(w))
    return np.array(cx[:]), np.array(cy[:]), w


def moment_matrix() -> np.ndarray:
    m = np.zeros(81)
    _load().orc_moment_matrix(_dp(m))
    return m.reshape(9, 9)


def operators(s5) -> tuple[np.ndarray, np.ndarray]:
    """(Lambda, source operator) = (M^-1 S M, M^-1 (I - S/2) M) for rates (s0..s4)."""
    s = np.ascontiguousarray(s5, dtype=np.float64)
    lam = np.zeros(81)
    src = np.zeros(81)
    _load().orc_operators(_dp(s), _dp(lam), _dp(src))
    return lam.reshape(9, 9), src.reshape(9, 9)


def cell_distributions(p: dict, **cell) -> dict:
    """Equilibrium and source distributions of one cell (f_eq, F, g_eq, G, h_eq, H)."""
    q = make_params(p)
    c = CellIn()
    for k, v in cell.items():
        setattr(c, k, float(v))
    outs = [np.zeros(9) for _ in range(6)]
    _load().orc_cell_distributions(C.byref(q), C.byref(c), *[_dp(o) for o in outs])
    return dict(zip(("feq", "F", "geq", "G", "heq", "H"), outs))


class Sim:
    """One oracle simulation: populations on an (ny, nx) grid in FP64."""

    def __init__(self, params: dict, lib_path: str | None = None):
        self._lib = _load(lib_path)
        self.params = dict(params)
        self._p = make_params(params)
        self.nx, self.ny = self._p.nx, self._p.ny
        self._h = self._lib.orc_create(C.byref(self._p))
        if not self._h:
            raise RuntimeError("oracle: invalid parameters or out of memory")

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _field(self, a) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != (self.ny, self.nx):
            a = np.broadcast_to(a, (self.ny, self.nx)).copy()
        return a

    def init(self, phi, psi, ux, uy, P):
        arrs = [self._field(a) for a in (phi, psi, ux, uy, P)]
        self._lib.orc_init(self._h, *[_dp(a) for a in arrs])

    def step(self, n: int = 1) -> int:
        return self._lib.orc_step(self._h, int(n))

    def moments(self) -> dict:
        outs = [np.zeros((self.ny, self.nx)) for _ in range(5)]
        self._lib.orc_moments(self._h, *[_dp(o) for o in outs])
        return dict(zip(("phi", "psi", "ux", "uy", "P"), outs))

    def fields(self) -> dict:
        n = self.nx * self.ny
        buf = (CellOut * n)()
        self._lib.orc_fields(self._h, buf)
        raw = np.ctypeslib.as_array(C.cast(buf, C.POINTER(C.c_double)), shape=(n, len(CellOut._fields_)))
        return {name: raw[:, j].reshape(self.ny, self.nx).copy()
                for j, (name, _) in enumerate(CellOut._fields_)}

    def total(self, what: str) -> float:
        return self._lib.orc_sum(self._h, 0 if what == "phi" else 1)

    def populations(self):
        f = np.zeros((9, self.ny, self.nx))
        g = np.zeros_like(f)
        h = np.zeros_like(f)
        self._lib.orc_populations(self._h, _dp(f), _dp(g), _dp(h))
        return f, g, h

    @property
    def status(self) -> int:
        return self._lib.orc_status(self._h)

    @property
    def steps(self) -> int:
        return self._lib.orc_steps(self._h)
