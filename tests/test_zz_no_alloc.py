"""The allocation-free normal operator (t2sh_normal_op_noalloc) against the planned one.

Some callers cannot let a library allocate device memory: code that runs where
cudaMalloc is not permitted, or an application that owns every byte of device memory
itself.  For them the library offers y = A^H A x with all scratch in a static device
array.  This test calls it through the C ABI twice in a row, with different inputs each
time (so stale scratch from the first call would show up in the second), and compares
each result with t2sh_normal_op of a plan built from the same inputs, within the
operator tolerance of the parity tests (NRMSE <= 1e-5; 1e-4 for the mixed-precision
column pass), that a call allocates no device memory, that y may alias x, that a size
beyond the static array is refused with EINVAL, and that a bounded device wait which
runs out on this path is reported by t2sh_noalloc_sync as T2SH_ETIMEOUT (the wait is on
a barrier nothing completes, with a limit of a few milliseconds: no fault is involved),
after which the entry point works and matches again.  The file name makes pytest
collect it last.
"""
import ctypes

import numpy as np
import pytest

import t2sh_synth as synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_04195_gb300 import build as B
    B.build()
    from paper_1809_04195_gb300 import t2sh
    return t2sh


def problem(seed, S, ny, nz, C, Tn, K, M):
    rng = np.random.default_rng(seed)
    phi = torch.from_numpy(synth.t2_basis(Tn, K).astype(np.float32)).cuda()
    mask = torch.from_numpy(synth.vd_masks(Tn, ny, nz, 0.2, rng)).cuda()
    maps = torch.from_numpy(np.stack([synth.coil_maps(C, ny, nz, rng, M=M) for _ in range(S)])
                            .astype(np.complex64)).cuda()
    x = torch.from_numpy((rng.standard_normal((S, M, K, ny, nz)) + 1j * rng.standard_normal((S, M, K, ny, nz)))
                         .astype(np.complex64)).cuda()
    return phi, mask, maps, x


def nrmse(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def planned(T, d, phi, mask, maps, x):
    with T.Plan(d, phi, mask, maps) as p:
        return p.normal_op(x)


def test_noalloc_normal_op_matches_planned_twice(T):
    cases = [(1, 2, 64, 48, 6, 20, 4, 1), (2, 3, 60, 36, 4, 12, 3, 2)]
    for seed, S, ny, nz, C, Tn, K, M in cases:
        phi, mask, maps, x = problem(seed, S, ny, nz, C, Tn, K, M)
        d = T.make_dims(ny, nz, C, Tn, K, nslices=S, nmaps=M)
        ref = planned(T, d, phi, mask, maps, x)
        got = T.normal_op_noalloc(d, phi, mask, maps, x)
        T.noalloc_sync()
        e = nrmse(got, ref)
        assert e <= OP_TOL, (seed, e)


def test_noalloc_allocates_nothing_and_allows_aliasing(T):
    S, ny, nz, C, Tn, K, M = 2, 64, 48, 6, 20, 4, 1
    phi, mask, maps, x = problem(5, S, ny, nz, C, Tn, K, M)
    d = T.make_dims(ny, nz, C, Tn, K, nslices=S, nmaps=M)
    ref = planned(T, d, phi, mask, maps, x)
    out = torch.empty_like(x)
    T.normal_op_noalloc(d, phi, mask, maps, x, out=out)  # loads the module and its array
    T.noalloc_sync()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    T.normal_op_noalloc(d, phi, mask, maps, x, out=out)
    T.noalloc_sync()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert nrmse(out, ref) <= OP_TOL
    xin = x.clone()  # y == x: the result overwrites its own input
    T.normal_op_noalloc(d, phi, mask, maps, xin, out=xin)
    T.noalloc_sync()
    assert nrmse(xin, ref) <= OP_TOL


def test_noalloc_mixed_precision_matches_planned(T):
    S, ny, nz, C, Tn, K, M = 2, 64, 48, 6, 20, 4, 1
    phi, mask, maps, x = problem(7, S, ny, nz, C, Tn, K, M)
    d = T.make_dims(ny, nz, C, Tn, K, nslices=S, nmaps=M, precision=T.MIXED_BF16)
    ref = planned(T, T.make_dims(ny, nz, C, Tn, K, nslices=S, nmaps=M), phi, mask, maps, x)
    for _ in range(2):
        got = T.normal_op_noalloc(d, phi, mask, maps, x)
        T.noalloc_sync()
        assert nrmse(got, ref) <= MIXED_TOL


def test_noalloc_reports_a_wait_that_ran_out(T):
    S, ny, nz, C, Tn, K, M = 2, 64, 48, 6, 20, 4, 1
    phi, mask, maps, x = problem(9, S, ny, nz, C, Tn, K, M)
    d = T.make_dims(ny, nz, C, Tn, K, nslices=S, nmaps=M)
    ref = planned(T, d, phi, mask, maps, x)
    T.noalloc_sync()  # nothing pending
    T.noalloc_wait_selftest(5_000_000)  # 5 ms on a barrier that nothing completes
    with pytest.raises(T.T2shError) as ei:
        T.noalloc_sync()
    assert ei.value.status == T.ETIMEOUT
    # a later call does not hide a timeout: the flag survives until it is read
    T.noalloc_wait_selftest(5_000_000)
    got = T.normal_op_noalloc(d, phi, mask, maps, x)
    with pytest.raises(T.T2shError) as ei:
        T.noalloc_sync()
    assert ei.value.status == T.ETIMEOUT
    # read once, the flag is clear: the next call succeeds and matches the planned operator
    got = T.normal_op_noalloc(d, phi, mask, maps, x)
    T.noalloc_sync()
    assert nrmse(got, ref) <= OP_TOL


def test_noalloc_rejects_sizes_beyond_the_static_array(T):
    # 320 knee slices need gigabytes of scratch
    d = T.make_dims(256, 160, 12, 80, 4, nslices=320)
    lib = T.lib()
    one = torch.zeros(1, device="cuda")
    p = ctypes.c_void_p(one.data_ptr())
    st = lib.t2sh_normal_op_noalloc(ctypes.byref(d), p, p, p, p, p, None)
    assert st == T.EINVAL
    assert "static array" in T.last_error()
