"""GPU parity of the ADMM solver loop (t2sh_solve_admm: CG alpha-updates with per-slice
float64 dot products, LLR prox on v, scaled dual) against the oracle's admm(), which
states the same iteration step by step in float64.

Tolerance: the float32 solve bar, per-slice NRMSE <= 1e-4.  A few CG steps per outer
iteration from the same warm start keep the float32 Krylov directions within ~1e-6 of
the float64 ones, and the ADMM outer map is non-expansive, so the gap does not grow.
"""
import numpy as np
import pytest

import oracle as O
import t2sh_synth as synth

from t2sh_cases import crandn, proj_scan, te_case
from test_gpu_parity import T, c64, host, make_plan, nrmse, r32, random_problem  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-4


@pytest.mark.parametrize("rho,cg_iters", [(0.5, 3), (0.2, 1), (1.0, 5)])
def test_admm_single_slice_64x48(T, rho, cg_iters):
    sh = synth.SINGLE_SLICE_64x48
    phi, mask, maps, y = te_case(sh)
    phi, maps = r32(phi, maps)
    ys = y.astype(np.complex64).astype(np.complex128)
    it = 30
    ref = O.admm(ys, "te", maps, mask, phi, sh.lam, sh.block, it, sh.seed, rho, cg_iters)
    with make_plan(T, phi, mask, maps[None], block=sh.block, lam=sh.lam, iters=it, seed=sh.seed) as p:
        got, res = p.solve_admm(c64(y[None]), T.KSPACE_TE, rho=rho, cg_iters=cg_iters, residual=True)
        got = host(got)[0]
        p.sync()
    e = nrmse(got, ref)
    print(f"ADMM rho={rho} cg={cg_iters}: NRMSE {e:.2e}, last residual {res[-1]:.2e}")
    assert e < SOLVE_TOL
    assert np.all(np.isfinite(res)) and res[-1] < res[1]


def test_admm_knee_slices_projected(T):
    sh = synth.KNEE_320x256x160
    sl = [0, 160]
    phi, mask, maps, ytil = proj_scan(sh, sl)
    phi, maps = r32(phi, maps)
    it, rho, cg_iters = 12, 0.5, 3
    with make_plan(T, phi, mask, maps, block=sh.block, lam=sh.lam, iters=it, seed=sh.seed) as p:
        got = host(p.solve_admm(c64(ytil), T.KSPACE_PROJ, rho=rho, cg_iters=cg_iters))
    ys = ytil.astype(np.complex64).astype(np.complex128)
    for i in range(len(sl)):
        ref = O.admm(ys[i], "proj", maps[i], mask, phi, sh.lam, sh.block, it, sh.seed, rho, cg_iters)
        e = nrmse(got[i], ref)
        print("ADMM knee slice", sl[i], "NRMSE", e)
        assert e < SOLVE_TOL


def test_admm_two_maps_partial_blocks_no_shift(T):
    rng, phi, mask, maps = random_problem(31, 2, 60, 36, 4, 24, 4, 2, frac=0.2)
    y = crandn(rng, 2, 4, 24, 60, 36) * mask[None, None] * 0.1
    ys = y.astype(np.complex64).astype(np.complex128)
    it, rho, cg_iters, lam, b = 15, 0.4, 4, 0.02, 8
    with make_plan(T, phi, mask, maps, block=b, lam=lam, iters=it, seed=9, flags=T.NO_SHIFT) as p:
        got = host(p.solve_admm(c64(y), T.KSPACE_TE, rho=rho, cg_iters=cg_iters))
    for s in range(2):
        ref = O.admm(ys[s], "te", maps[s], mask, phi, lam, b, it, 9, rho, cg_iters, shifts=False)
        assert nrmse(got[s], ref) < SOLVE_TOL


def test_admm_edge_cases(T):
    rng, phi, mask, maps = random_problem(32, 1, 32, 32, 2, 8, 4, 1)
    y = crandn(rng, 1, 2, 8, 32, 32) * mask[None, None]
    with make_plan(T, phi, mask, maps, block=8, lam=0.1, iters=4) as p:
        assert np.all(host(p.solve_admm(c64(y), T.KSPACE_TE, rho=0.5, cg_iters=0)) == 0)  # alpha stays 0
        with pytest.raises(T.T2shError):
            p.solve_admm(c64(y), T.KSPACE_TE, rho=0.0, cg_iters=2)
        with pytest.raises(T.T2shError):
            p.solve_admm(c64(y), T.KSPACE_TE, rho=float("nan"), cg_iters=2)
        # the plan still solves with FISTA afterwards
        p.solve(c64(y), T.KSPACE_TE)
        p.sync()


def test_admm_host_io_matches_device(T):
    sh = synth.SINGLE_SLICE_64x48
    phi, mask, maps, y = te_case(sh)
    kw = dict(block=sh.block, lam=sh.lam, iters=8, seed=sh.seed)
    with make_plan(T, phi, mask, maps[None], **kw) as p:
        dev_out = host(p.solve_admm(c64(y[None]), T.KSPACE_TE, rho=0.5, cg_iters=3))
    d = T.make_dims(64, 48, 8, 32, 4, flags=T.HOST_IO, **kw)
    with T.Plan(d, phi.astype(np.float32), mask.astype(np.uint8), maps[None].astype(np.complex64)) as p:
        host_out = p.solve_admm(y[None].astype(np.complex64), T.KSPACE_TE, rho=0.5, cg_iters=3)
    assert np.array_equal(host_out.astype(np.complex128), dev_out)
