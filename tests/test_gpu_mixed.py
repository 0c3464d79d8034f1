"""GPU parity of the mixed-precision path (precision = T2SH_MIXED_BF16): the column pass
of the normal operator runs as split-BF16 DFT-as-GEMM on the tensor cores (FP32
accumulation), everything else as in the FP32 path.

Tolerances: a split-BF16 product carries about 16 significant bits (relative error
~2^-17 per term, the dropped lo x lo term ~2^-18), so a column DFT pair plus Psi is
expected near 1e-5 NRMSE; the operator bound is 1e-4.  The solve bound is the stated
1e-3 per slice for the mixed-precision path.
"""
import numpy as np
import pytest

import oracle as O
import t2sh_synth as synth

from t2sh_cases import crandn, proj_scan, te_case
from test_gpu_parity import T, c64, host, make_plan, nrmse, r32, random_problem  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_OP_TOL = 1e-4
MIXED_SOLVE_TOL = 1e-3

MIXED_SHAPES = [
    # S, ny, nz, C, T, K, M   (ny = 16 R1; nz % 4 == 0; K <= 4)
    (1, 64, 48, 8, 32, 4, 1),     # R1 = 4, one K-step in stage 1
    (1, 256, 160, 2, 16, 4, 1),   # the knee slice matrix, R1 = 16
    (1, 240, 128, 3, 12, 4, 1),   # R1 = 15
    (2, 96, 64, 2, 8, 2, 1),      # K = 2 (one 128-row block per stage)
    (1, 192, 192, 2, 12, 4, 2),   # two map sets, R1 = 12
    (2, 48, 40, 3, 12, 3, 1),     # R1 = 3, K = 3 (padded rows)
    (1, 160, 96, 2, 8, 1, 1),     # K = 1, R1 = 10
    (1, 128, 36, 2, 8, 4, 1),     # R1 = 8, nz = 36
    (1, 60, 36, 2, 8, 4, 1),      # ny = 60 is not 16 R1: the FP32 column pass serves it
]


@pytest.mark.parametrize("S,ny,nz,C,Tn,K,M", MIXED_SHAPES)
def test_mixed_normal_op_matches_oracle(T, S, ny, nz, C, Tn, K, M):
    rng, phi, mask, maps = random_problem(500 + ny + K, S, ny, nz, C, Tn, K, M)
    x = crandn(rng, S, M, K, ny, nz)
    with make_plan(T, phi, mask, maps, precision=T.MIXED_BF16) as p:
        got = host(p.normal_op(c64(x)))
        p.sync()
    with make_plan(T, phi, mask, maps) as p:
        got32 = host(p.normal_op(c64(x)))
    psi = O.space_time_kernel(mask, phi)
    xs = x.astype(np.complex64).astype(np.complex128)
    for s in range(S):
        ref = O.normal(xs[s], maps[s], psi)
        e, e32 = nrmse(got[s], ref), nrmse(got32[s], ref)
        print(f"{ny}x{nz} K={K} M={M}: mixed {e:.2e}, fp32 {e32:.2e}")
        assert e < MIXED_OP_TOL


def test_mixed_solve_single_slice_64x48(T):
    sh = synth.SINGLE_SLICE_64x48
    phi, mask, maps, y = te_case(sh)
    phi, maps = r32(phi, maps)
    ys = y.astype(np.complex64).astype(np.complex128)
    ref = O.fista(ys, "te", maps, mask, phi, sh.lam, sh.block, sh.iters, sh.seed)
    with make_plan(T, phi, mask, maps[None], block=sh.block, lam=sh.lam, iters=sh.iters, seed=sh.seed,
                   precision=T.MIXED_BF16) as p:
        got = host(p.solve(c64(y[None]), T.KSPACE_TE))[0]
        p.sync()
    e = nrmse(got, ref)
    print("mixed single-slice NRMSE", e)
    assert e < MIXED_SOLVE_TOL


def test_mixed_solve_knee_slices(T):
    """Knee slices (256 x 160, C = 12, T = 80, 5 %/echo, 100 iterations), projected input:
    the mixed-precision solve against the oracle, next to the FP32 solve."""
    sh = synth.KNEE_320x256x160
    sl = [0, 160]
    phi, mask, maps, ytil = proj_scan(sh, sl)
    phi, maps = r32(phi, maps)
    kw = dict(block=sh.block, lam=sh.lam, iters=sh.iters, seed=sh.seed)
    with make_plan(T, phi, mask, maps, precision=T.MIXED_BF16, **kw) as p:
        got = host(p.solve(c64(ytil), T.KSPACE_PROJ))
        p.sync()
    with make_plan(T, phi, mask, maps, **kw) as p:
        got32 = host(p.solve(c64(ytil), T.KSPACE_PROJ))
    ys = ytil.astype(np.complex64).astype(np.complex128)
    for i in range(len(sl)):
        ref = O.fista(ys[i], "proj", maps[i], mask, phi, sh.lam, sh.block, sh.iters, sh.seed)
        e, e32 = nrmse(got[i], ref), nrmse(got32[i], ref)
        print(f"knee slice {sl[i]}: mixed NRMSE {e:.2e}, fp32 {e32:.2e}")
        assert e < MIXED_SOLVE_TOL


def test_mixed_batch_and_autotune(T):
    """A mixed-precision plan keeps its tensor-core column pass through autotuning and
    batching, and the batch equals the single solve.  The batch plans take the tuned choice
    from the process's tuning cache, so all three run the same kernels (the fused row form,
    if the timing picked it, agrees with the separate kernels only to rounding)."""
    rng, phi, mask, maps = random_problem(21, 2, 64, 48, 4, 16, 4, 1)
    y = crandn(rng, 2, 4, 4, 64, 48) * 0.1
    kw = dict(block=8, lam=0.01, iters=6, seed=3, precision=T.MIXED_BF16)
    with make_plan(T, phi, mask, maps, **kw) as p:
        var, fused = p.autotune(2)
        assert var == 3
        one = host(p.solve(c64(y), T.KSPACE_PROJ))
    with make_plan(T, phi, mask, maps, **kw) as p1, make_plan(T, phi, mask, maps, **kw) as p2:
        assert p1.autotune(2) == (var, fused) and p2.autotune(2) == (var, fused)
        outs = T.solve_batch([p1, p2], [c64(y), c64(y)], [T.KSPACE_PROJ, T.KSPACE_PROJ])
        for o in outs:
            assert np.array_equal(host(o), one)
