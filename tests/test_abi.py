"""CPU checks of the C ABI: the library loads, exports every function that
include/t2sh.h declares, and its host-only entry points behave (no GPU calls)."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1809_04195_gb300 import build as B
from paper_1809_04195_gb300 import t2sh


@pytest.fixture(scope="module")
def lib():
    B.build()
    return t2sh.lib()


def test_exports_every_declared_symbol(lib):
    declared = t2sh.header_symbols()
    assert len(declared) >= 12
    nm = subprocess.run(["nm", "-D", "--defined-only", t2sh.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in nm.splitlines() if ln.strip()}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert getattr(lib, s) is not None


C_PROGRAM = r"""
#include <stdio.h>
#include "t2sh.h"
int main(void) {
  t2sh_dims d = {0};
  d.ny = 256; d.nz = 160; d.ncoils = 12; d.nmaps = 1; d.nechoes = 80; d.nbasis = 4;
  d.nslices = 320; d.block = 8; d.lambda = 0.005f; d.iters = 100; d.seed = 1; d.precision = T2SH_FP32;
  size_t ws = 0;
  int32_t sh[4];
  if (t2sh_workspace_bytes(&d, &ws) != T2SH_OK) { fprintf(stderr, "%s\n", t2sh_last_error()); return 1; }
  if (t2sh_shifts(1809, 2, 8, sh) != T2SH_OK) return 2;
  d.ny = 63;
  if (t2sh_workspace_bytes(&d, &ws) == T2SH_OK) return 3;
  printf("%d %zu %d %d %d %d\n", t2sh_version(), ws, sh[0], sh[1], sh[2], sh[3]);
  return 0;
}
"""


def test_header_is_c99_and_links_from_c(lib, tmp_path):
    """A plain C99 program (-pedantic -Werror) includes the header, links the library and
    gets the same host-only results as the binding and the oracle."""
    import os
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "main.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "main"
    libdir = os.path.dirname(t2sh.LIB_PATH)
    inc = os.path.join(os.path.dirname(libdir), "include")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, str(src),
                        "-L", libdir, "-l:libt2sh.so", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.pathsep.join(p for p in ("/usr/local/cuda/lib64", env.get("LD_LIBRARY_PATH", "")) if p)
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env)
    assert r.returncode == 0, r.stderr
    ver, ws, *sh = (int(v) for v in r.stdout.split())
    assert ver == t2sh.version()
    assert ws == t2sh.workspace_bytes(t2sh.make_dims(256, 160, 12, 80, 4, nslices=320, block=8, iters=100,
                                                     lam=0.005, seed=1))
    assert sh == [int(v) for v in O.llr_shifts(1809, 2, 8).ravel()]


def test_version(lib):
    assert t2sh.version() == 100


@pytest.mark.parametrize("seed,b", [(1809, 8), (1810, 8), (0, 12), (2**63 + 12345, 5), (7, 1)])
def test_shift_table_bit_exact_with_oracle(lib, seed, b):
    got = t2sh.shifts(seed, 300, b)
    ref = O.llr_shifts(seed, 300, b)
    assert np.array_equal(got.astype(np.int64), ref)


def test_workspace_bytes_formula(lib):
    d = t2sh.make_dims(256, 160, 12, 80, 4, nslices=320, block=8, iters=100)
    N = 256 * 160
    vec = 320 * 1 * 4 * N * 8
    expect = (320 * 12 * 1 * N * 8 + 10 * N * 4 + 80 * 4 * 4 + 80 * N + 4 * vec + 320 * 12 * 4 * N * 8
              + (256 + 160) * 8 + 8 * 2 * 100 + 64)
    assert t2sh.workspace_bytes(d) == expect


@pytest.mark.parametrize("kw,status", [
    (dict(ny=63), t2sh.EINVAL),          # odd
    (dict(nz=14 * 7), t2sh.EINVAL),      # 98 = 2 * 7^2: 7 is not a radix of the FFT passes
    (dict(ny=2 * 11 * 5), t2sh.EINVAL),  # 110: 11 neither
    (dict(ny=4), t2sh.EINVAL),           # too small
    (dict(nbasis=9), t2sh.EINVAL),
    (dict(nmaps=3), t2sh.EINVAL),
    (dict(block=0), t2sh.EINVAL),
    (dict(nechoes=3), t2sh.EINVAL),      # T < K
    (dict(precision=2), t2sh.EINVAL),     # neither FP32 nor MIXED_BF16
    (dict(flags=0x80), t2sh.EINVAL),
    (dict(flags=0x10), t2sh.EINVAL),
    (dict(ny=1024), t2sh.EINVAL),        # above the largest slice matrix, 512
    (dict(block=17), t2sh.EINVAL),       # above the largest block, 16
    (dict(nslices=0), t2sh.EINVAL),      # an empty batch of slices
    (dict(nslices=65536), t2sh.EINVAL),  # above the largest batch
    (dict(ncoils=0), t2sh.EINVAL),
    (dict(iters=-1), t2sh.EINVAL),
    (dict(lam=-0.1), t2sh.EINVAL),
    (dict(lam=float("nan")), t2sh.EINVAL),
    (dict(step=float("inf")), t2sh.EINVAL),
    # an LLR band of K x b x nz = 4 x 16 x 512 complex values (262 KB) exceeds shared memory
    (dict(ny=512, nz=512, block=16), t2sh.EUNSUPPORTED),
])
def test_invalid_dims_rejected(lib, kw, status):
    base = dict(ny=64, nz=48, ncoils=8, nechoes=32, nbasis=4, nslices=1, block=8, iters=10)
    base.update(kw)
    d = t2sh.make_dims(**base)
    n = ctypes.c_size_t(0)
    assert lib.t2sh_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == status
    assert len(t2sh.last_error()) > 0


def test_largest_supported_shapes_accepted(lib):
    """512 x 512 with a band that fits: K = 4 with 8-row blocks, K = 2 with 16-row blocks."""
    for kw in (dict(nbasis=4, block=8), dict(nbasis=2, block=16)):
        d = t2sh.make_dims(512, 512, 2, 8, nslices=1, iters=4, **kw)
        n = ctypes.c_size_t(0)
        assert lib.t2sh_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == t2sh.OK


def test_paper_slice_matrix_accepted(lib):
    """Table I: 260 x 240 slices (260 = 4 * 5 * 13), C = 7, M = 2, b = 12."""
    d = t2sh.make_dims(260, 240, 7, 80, 4, nslices=288, nmaps=2, block=12, iters=250, lam=0.0125)
    n = ctypes.c_size_t(0)
    assert lib.t2sh_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == t2sh.OK
    assert n.value > 0


def test_mixed_precision_dims_accepted(lib):
    d = t2sh.make_dims(256, 160, 12, 80, 4, nslices=2, block=8, iters=10, precision=t2sh.MIXED_BF16)
    n = ctypes.c_size_t(0)
    assert lib.t2sh_workspace_bytes(ctypes.byref(d), ctypes.byref(n)) == t2sh.OK
    assert n.value == t2sh.workspace_bytes(t2sh.make_dims(256, 160, 12, 80, 4, nslices=2, block=8, iters=10))


def test_null_arguments_rejected(lib):
    assert lib.t2sh_workspace_bytes(None, None) == t2sh.EINVAL
    assert lib.t2sh_normal_op(None, None, None) == t2sh.EINVAL
    assert lib.t2sh_destroy(None) == t2sh.OK
    out = ctypes.c_void_p(0)
    assert lib.t2sh_plan(None, None, None, None, None, ctypes.byref(out)) == t2sh.EINVAL and not out.value
    assert lib.t2sh_forward(None, None, None, t2sh.KSPACE_TE) == t2sh.EINVAL
    assert lib.t2sh_adjoint(None, None, t2sh.KSPACE_TE, None) == t2sh.EINVAL
    assert lib.t2sh_llr_prox(None, None, 0.1, 0, 0) == t2sh.EINVAL
    assert lib.t2sh_solve(None, None, t2sh.KSPACE_PROJ, None, None) == t2sh.EINVAL
    assert lib.t2sh_solve_admm(None, None, t2sh.KSPACE_PROJ, None, 1.0, 3, None) == t2sh.EINVAL
    assert lib.t2sh_objective(None, None, t2sh.KSPACE_PROJ, None, None) == t2sh.EINVAL
    assert lib.t2sh_postprocess(None, None, None, 0, 0.65, None) == t2sh.EINVAL
    assert lib.t2sh_sync(None) == t2sh.EINVAL
    assert lib.t2sh_configure(None, 0, 0) == t2sh.EINVAL
    assert lib.t2sh_wait_selftest(None, 1000) == t2sh.EINVAL
    assert lib.t2sh_autotune(None, 3, None, None) == t2sh.EINVAL
    assert lib.t2sh_solve_begin(None, None, t2sh.KSPACE_PROJ) == t2sh.EINVAL
    assert lib.t2sh_solve_iterate(None, 1, None) == t2sh.EINVAL
    assert lib.t2sh_solve_end(None, None, None) == t2sh.EINVAL
