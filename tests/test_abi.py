"""The C-ABI library builds for sm_103a, loads, and exports what include/lbm.h declares (no GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2408_15654_gb300 import lbm
from paper_2408_15654_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(lbm_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = lbm.load()
    names = declared_functions()
    assert len(names) >= 27
    assert sorted(lbm.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lbm._build.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_\w+)", out))
    assert set(names) <= exported


@pytest.mark.parametrize("name", ["lbm_params", "lbm_server_config", "lbm_job_result", "lbm_server_stats"])
def test_struct_layout_matches_header(tmp_path, name):
    """Compile a probe against the header with gcc and compare sizeof/offsetof with ctypes."""
    cls = getattr(lbm, name)
    fields = [f[0] for f in cls._fields_]
    src = tmp_path / "probe.c"
    body = "\n".join(f'printf("{f} %zu\\n", offsetof({name}, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\nint main(void){'
                   f'printf("size %zu\\n", sizeof({name}));{body}return 0;}}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), "-o", str(exe), str(src)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n") if line)
    assert int(got["size"]) == C.sizeof(cls)
    for f in fields:
        assert int(got[f]) == getattr(cls, f).offset, f


def test_workspace_bytes_without_gpu():
    p, _ = W.shear_drop(512, 256)
    n = lbm.lbm_workspace_bytes(lbm.make_params(p))
    # planes of (256 + 4) rows x pitch cells, pitch = 512 + 10 rounded up to 32 (the ghost frame)
    pitch, rows = 544, 260
    cells = pitch * rows
    # two buffers of 26 float planes, two (u_x, u_y) history buffers, status and partials
    assert n >= 2 * 26 * cells * 4 + 2 * cells * 8
    assert n < 2 * 26 * cells * 4 + 2 * cells * 8 + 64 * 1024
    # 16-bit storage halves the population buffers
    p["storage"] = "fp16"
    n16 = lbm.lbm_workspace_bytes(lbm.make_params(p))
    assert n16 >= 2 * 13 * cells * 4 + 2 * cells * 8
    assert n16 < 2 * 13 * cells * 4 + 2 * cells * 8 + 64 * 1024
    # f and g in 16 bits, h in FP32: 68 bytes per cell and buffer
    p["storage"] = "bf16_fg"
    nfg = lbm.lbm_workspace_bytes(lbm.make_params(p))
    assert nfg >= 2 * 68 * cells + 2 * cells * 8
    assert nfg < 2 * 68 * cells + 2 * cells * 8 + 64 * 1024


def test_prescribed_velocity_workspace_has_no_flow_planes():
    p, _ = W.convected_drop(512, 256)
    full = lbm.lbm_workspace_bytes(lbm.make_params(dict(p, velocity="solved")))
    pres = lbm.lbm_workspace_bytes(lbm.make_params(p))
    assert full - pres == 2 * 8 * 4 * 260 * 544


@pytest.mark.parametrize("bad", [dict(nx=1), dict(ny=0), dict(rhoB=0.0), dict(W=0.0), dict(M_phi=-1.0),
                                 dict(D=0.0), dict(muA=0.0), dict(s_f=(1, 1, 2.5, 1, 1)),
                                 dict(sigma0=float("nan")), dict(storage=7),
                                 dict(velocity=2)])
def test_parameter_validation(bad):
    p, _ = W.stationary_drop(32, 32, R=8)
    p.update(bad)
    q = lbm.make_params(p)
    n = C.c_size_t()
    rc = lbm.load().lbm_workspace_bytes(C.byref(q), C.byref(n))
    assert rc == lbm.LBM_EINVAL
    assert lbm.lbm_last_error()


def test_calls_reject_null_handle():
    lib = lbm.load()
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_reduce(None, 0, None) == lbm.LBM_EINVAL
    assert lib.lbm_destroy(None) == lbm.LBM_OK


def test_density_ratio_workspace_has_a_mass_flux_history():
    p, _ = W.rising_bubble(16.0)
    var = lbm.lbm_workspace_bytes(lbm.make_params(p))
    uni = lbm.lbm_workspace_bytes(lbm.make_params(dict(p, rhoB=p["rhoA"])))
    pitch, rows = (64 + 10 + 31) // 32 * 32, 128 + 4
    assert var - uni == 2 * ((pitch * rows * 8 + 255) // 256 * 256)


@pytest.mark.parametrize("storage,pair_bytes", [("fp32", 104), ("fp16", 52), ("bf16_fg", 68)])
def test_grid_size_limits(storage, pair_bytes):
    """The smallest grid (2 x 2) and grids of exactly 2^30 cells are accepted, with at least the two
    population buffers in the workspace (the size query allocates nothing); one cell row or column
    beyond 2^30 cells, more than 524280 rows (65535 rows of 8-row tiles), or a dimension below 2,
    is rejected."""
    lib = lbm.load()
    n = C.c_size_t()
    for nx, ny, ok in ((2, 2, True), (1 << 15, 1 << 15, True), (1 << 12, 1 << 18, True), (1 << 29, 2, True),
                       (2048, 524280, True), (2048, 524281, False), (2, 1 << 29, False),
                       (1 << 15, (1 << 15) + 1, False), ((1 << 29) + 1, 2, False), (2, 1, False), (1, 2, False)):
        p, _ = W.stationary_drop(8, 8, R=2)
        p.update(nx=nx, ny=ny, storage=storage)
        rc = lib.lbm_workspace_bytes(C.byref(lbm.make_params(p)), C.byref(n))
        assert (rc == lbm.LBM_OK) == ok, (nx, ny, rc)
        if ok:
            assert n.value >= 2 * pair_bytes * nx * ny, (nx, ny, n.value)
        else:
            assert lbm.lbm_last_error()


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16", "fp16_fg"])
def test_population_buffers_hold_the_staged_fields(storage):
    """Each population buffer also stages the five FP64 fields of lbm_init_fields and
    lbm_get_moments (40 bytes per cell), also where 16-bit storage with a prescribed velocity needs
    fewer bytes for its populations."""
    lib = lbm.load()
    n = C.c_size_t()
    for nx, ny in ((512, 512), (2048, 1024), (100, 100)):
        p, _ = W.convected_drop(nx, ny, R=nx / 8)
        p["storage"] = storage
        assert lib.lbm_workspace_bytes(C.byref(lbm.make_params(p)), C.byref(n)) == lbm.LBM_OK
        assert n.value >= 2 * 40 * nx * ny + 2 * 8 * nx * ny, (nx, ny, n.value)
