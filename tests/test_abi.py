"""CPU checks of the C ABI library: it loads without a GPU, exports every
entry point include/glasma.h declares, and its host-side validation and
workspace sizing behave as documented.  No compute call is made here."""
import ctypes
import math
import os
import re

import pytest

import paper_2303_05599_gb300 as G
from paper_2303_05599_gb300 import _binding as B
from paper_2303_05599_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_05599_gb300 import build
    build.build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "glasma.h")).read()
    return re.findall(r"^(?:size_t|gl_status|const char\*)\s+(\w+)\(", src, re.M)


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert len(names) >= 13
    L = ctypes.CDLL(B.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(B.SIGNATURES)


def test_batch_obs_row_bytes():
    # GL_MAX_SPECIES x 7 per-species values and 7 field check values, FP64;
    # host only, so it is called here without a GPU
    n = B.lib().gl_batch_obs_row_bytes()
    assert n == 8 * (B.GL_MAX_SPECIES * 7 + 7)
    assert n <= ctypes.sizeof(B.gl_obs)


def test_struct_sizes_match_header():
    # gl_config: 4 int32 + 5 double + uint64 + 2 int32; gl_species: 2 double + int64 + 2 int32 + 2 double
    assert ctypes.sizeof(B.gl_config) == 16 + 40 + 8 + 8 + 8
    assert ctypes.sizeof(B.gl_species) == 16 + 8 + 8 + 16
    assert ctypes.sizeof(B.gl_obs) == 8 + 8 + 8 + 8 * 8 + 6 * 8 * 8 + 7 * 8


def test_workspace_bytes_and_validation():
    w = W.config_small()
    n64 = G.gl_workspace_bytes(w)
    w32 = W.config_small()
    w32.precision = W.FP32_2ROW
    n32 = G.gl_workspace_bytes(w32)
    assert n64 > 0 and 0 < n32 < n64
    # FP64 field buffers: 2 x (2 links x 9 + 4 algebra planes x 4) x 16 B per site
    V = w.N * w.N
    assert n64 >= 2 * V * (18 + 16) * 16
    bad = W.config_small()
    bad.N = 2
    assert G.gl_workspace_bytes(bad) == 0
    bad = W.config_small()
    bad.species[0].rep = 5
    assert G.gl_workspace_bytes(bad) == 0


def test_create_rejects_bad_workspace_without_touching_the_gpu():
    L = B.lib()
    w = W.config_small()
    cfg = B.make_config(w)
    sp = B.make_species(w)
    ctx = ctypes.c_void_p()
    # misaligned pointer
    st = L.gl_create(ctypes.byref(cfg), sp, 1, ctypes.c_void_p(0x1001), 1 << 30, None, ctypes.byref(ctx))
    assert st == B.GL_ERR_ARG and not ctx.value
    assert b"aligned" in L.gl_error_string(None)
    # too small
    st = L.gl_create(ctypes.byref(cfg), sp, 1, ctypes.c_void_p(0x10000), 1024, None, ctypes.byref(ctx))
    assert st == B.GL_ERR_SIZE
    # host-only creation/destruction with a fake device address works
    need = L.gl_workspace_bytes(ctypes.byref(cfg), sp, 1)
    st = L.gl_create(ctypes.byref(cfg), sp, 1, ctypes.c_void_p(0x100000), need, None, ctypes.byref(ctx))
    assert st == B.GL_OK and ctx.value
    # wong_push before any field step is refused before any launch
    assert L.wong_push(ctx) == B.GL_ERR_STATE
    assert L.gl_destroy(ctx) == B.GL_OK


def test_lattice_units_match_workload_module():
    w = W.config_n256()
    assert abs(w.a_fm - 10.0 / 256) < 1e-15
    assert w.n_steps == 205
    assert W.config_small().n_steps == 86
    m, tf, p0, p1 = w.lattice_species()[0]
    assert abs(m - 1.27 * w.a_GeVinv) < 1e-15 and abs(tf - 0.06 / w.a_fm) < 1e-12
    assert math.isinf(w.lattice_species()[1][0])


def test_native_snapshot_sizes_and_checks_without_touching_the_gpu():
    """gl_native_bytes from the configuration alone; a wrong size or an
    unknown part is refused before any copy."""
    L = B.lib()
    w = W.config_small()
    cfg = B.make_config(w)
    sp = B.make_species(w)
    ctx = ctypes.c_void_p()
    need = L.gl_workspace_bytes(ctypes.byref(cfg), sp, 1)
    assert L.gl_create(ctypes.byref(cfg), sp, 1, ctypes.c_void_p(0x100000), need, None, ctypes.byref(ctx)) == B.GL_OK
    n = w.n_particles
    a256 = lambda b: (b + 255) // 256 * 256
    if w.precision == W.FP64:
        per_site = 34 * 16
        parts = 3 * a256(16 * n) + a256(64 * n) + 2 * a256(4 * n) + 2 * a256(8 * n)
    else:
        per_site = 14 * 16
        parts = a256(16 * n) + a256(8 * n) + a256(32 * n) + 3 * a256(4 * n) + a256(8 * n)
    assert L.gl_native_bytes(ctx, B.GL_NATIVE_FIELDS) == w.N * w.N * per_site
    assert L.gl_native_bytes(ctx, B.GL_NATIVE_PARTICLES) == parts
    assert L.gl_native_bytes(ctx, 5) == 0 and L.gl_native_bytes(None, B.GL_NATIVE_FIELDS) == 0
    buf = (ctypes.c_uint8 * 64)()
    assert L.gl_upload_native(ctx, B.GL_NATIVE_FIELDS, buf, 64) == B.GL_ERR_SIZE
    assert L.gl_download_native(ctx, B.GL_NATIVE_PARTICLES, buf, 64) == B.GL_ERR_SIZE
    assert L.gl_upload_native(ctx, 9, buf, 64) == B.GL_ERR_ARG
    assert L.gl_download_native(None, B.GL_NATIVE_FIELDS, buf, 64) == B.GL_ERR_ARG
    assert L.gl_destroy(ctx) == B.GL_OK
