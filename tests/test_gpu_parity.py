"""GPU parity: every C-ABI entry point against the FP64 oracle on seeded inputs.

Tolerances (float32 arithmetic against float64):
  * single operators (A, A^H, A^H A, LLR prox): NRMSE <= 1e-5.  A 2D FFT pair
    accumulates about log2(ny nz) ~ 12-16 roundings of u = 6e-8 per stage, plus the
    K-term Psi and C-term coil sums: expected ~1e-6, bound 1e-5.
  * the FISTA solve: per-slice NRMSE <= 1e-4 (the stated requirement of the fp32 path).
"""
import numpy as np
import pytest

import oracle as O
import t2sh_synth as synth

from t2sh_cases import crandn, proj_scan, te_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
SOLVE_TOL = 1e-4


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_04195_gb300 import build as B
    B.build()
    from paper_1809_04195_gb300 import t2sh
    return t2sh


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def c64(a):
    return dev(np.asarray(a, np.complex64))


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def nrmse(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def make_plan(T, phi, mask, maps, **kw):
    S, C, M, ny, nz = maps.shape
    Tn, K = phi.shape
    d = T.make_dims(ny, nz, C, Tn, K, nslices=S, nmaps=M, **kw)
    return T.Plan(d, dev(phi.astype(np.float32)), dev(mask.astype(np.uint8)), c64(maps))


def r32(phi=None, maps=None):
    """The inputs as the float32 / complex64 values the GPU receives, widened back."""
    out = []
    if phi is not None:
        out.append(phi.astype(np.float32).astype(np.float64))
    if maps is not None:
        out.append(maps.astype(np.complex64).astype(np.complex128))
    return out


def random_problem(seed, S, ny, nz, C, T_, K, M, frac=0.15):
    rng = np.random.default_rng(seed)
    phi = synth.t2_basis(T_, K)
    mask = synth.vd_masks(T_, ny, nz, frac, rng)
    maps = np.stack([synth.coil_maps(C, ny, nz, rng, M=M) for _ in range(S)])
    phi, maps = r32(phi, maps)
    return rng, phi, mask, maps


SHAPES = [
    # S, ny, nz, C, T, K, M
    (1, 64, 48, 8, 32, 4, 1),
    (3, 40, 24, 3, 12, 4, 2),
    (2, 60, 36, 4, 10, 3, 1),   # radix-3/5 passes, K < 4
    (2, 48, 30, 2, 14, 6, 1),   # K > 4 path
    (1, 256, 160, 2, 16, 4, 1),  # the knee slice matrix
    (1, 240, 128, 3, 12, 4, 1),  # size-specialised passes with 4-row bands
    (1, 192, 192, 2, 12, 4, 2),  # two map sets on the specialised passes
    (2, 96, 64, 2, 8, 2, 1),     # K = 2 on the specialised passes
    (1, 260, 240, 7, 16, 4, 2),  # Table I slice matrix: radix-13 passes, C = 7, M = 2
    (1, 260, 48, 2, 8, 2, 1),    # 260-point columns (two tensor-map boxes) with K = 2
    (2, 64, 240, 3, 8, 2, 2),    # two-row row-pass bands for two map sets at nz = 240, K = 2
    (1, 512, 512, 2, 8, 4, 1),   # the largest slice matrix (generic passes)
    (1, 32, 24, 2, 16, 8, 1),    # K = 8, the largest basis
    (2, 8, 8, 1, 4, 2, 1),       # the smallest matrix, one coil
    (1, 26, 52, 2, 8, 3, 1),     # radix 13 on the generic passes
]


@pytest.mark.parametrize("S,ny,nz,C,Tn,K,M", SHAPES)
def test_operators_match_oracle(T, S, ny, nz, C, Tn, K, M):
    rng, phi, mask, maps = random_problem(100 + ny + K, S, ny, nz, C, Tn, K, M)
    with make_plan(T, phi, mask, maps, block=8) as p:
        x = crandn(rng, S, M, K, ny, nz)
        y = crandn(rng, S, C, Tn, ny, nz)
        ytil = crandn(rng, S, C, K, ny, nz)
        g_fwd_te = host(p.forward(c64(x), T.KSPACE_TE))
        g_fwd_pr = host(p.forward(c64(x), T.KSPACE_PROJ))
        g_adj_te = host(p.adjoint(c64(y), T.KSPACE_TE))
        g_adj_pr = host(p.adjoint(c64(ytil), T.KSPACE_PROJ))
        g_nrm = host(p.normal_op(c64(x)))
        torch.cuda.synchronize()
    psi = O.space_time_kernel(mask, phi)
    xs = x.astype(np.complex64).astype(np.complex128)
    ys = y.astype(np.complex64).astype(np.complex128)
    yts = ytil.astype(np.complex64).astype(np.complex128)
    for s in range(S):
        assert nrmse(g_fwd_te[s], O.forward(xs[s], maps[s], mask, phi)) < OP_TOL
        assert nrmse(g_fwd_pr[s], O.project(O.forward(xs[s], maps[s], mask, phi), mask, phi)) < OP_TOL
        assert nrmse(g_adj_te[s], O.adjoint(ys[s], maps[s], mask, phi)) < OP_TOL
        assert nrmse(g_adj_pr[s], O.adjoint_projected(yts[s], maps[s])) < OP_TOL
        assert nrmse(g_nrm[s], O.normal(xs[s], maps[s], psi)) < OP_TOL


def test_adjoint_identity_on_gpu(T):
    rng, phi, mask, maps = random_problem(7, 2, 64, 48, 4, 16, 4, 1)
    with make_plan(T, phi, mask, maps) as p:
        x = c64(crandn(rng, 2, 1, 4, 64, 48))
        y = c64(crandn(rng, 2, 4, 16, 64, 48) * mask[None, None])
        ax = p.forward(x, T.KSPACE_TE)
        ahy = p.adjoint(y, T.KSPACE_TE)
        lhs = torch.vdot(y.flatten().to(torch.complex128), ax.flatten().to(torch.complex128)).item()
        rhs = torch.vdot(ahy.flatten().to(torch.complex128), x.flatten().to(torch.complex128)).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_step_matches_oracle(T):
    _, phi, mask, maps = random_problem(9, 3, 64, 48, 6, 20, 4, 2)
    with make_plan(T, phi, mask, maps) as p:
        mu = p.step
    L = max(O.lipschitz(maps[s], O.space_time_kernel(mask, phi)) for s in range(3))
    assert abs(mu - 1.0 / L) <= 1e-5 / L


def test_plan_step_is_shared_by_its_slices(T):
    """A plan's slices share one step, 1/L with L the largest Lipschitz bound over its slices
    (a valid step for each of them).  With coil maps of a different scale in every slice the
    library takes that smallest step, and the oracle's FISTA given the same step agrees
    slice by slice."""
    rng, phi, mask, maps = random_problem(14, 3, 48, 40, 3, 16, 4, 1, frac=0.3)
    (maps,) = r32(maps=maps * np.array([1.0, 0.6, 1.5])[:, None, None, None, None])
    y = crandn(rng, 3, 3, 16, 48, 40) * mask[None, None] * 0.1
    ys = y.astype(np.complex64).astype(np.complex128)
    psi = O.space_time_kernel(mask, phi)
    L = max(O.lipschitz(maps[s], psi) for s in range(3))
    with make_plan(T, phi, mask, maps, block=8, lam=0.02, iters=15, seed=3) as p:
        assert abs(p.step - 1.0 / L) <= 1e-5 / L
        got = host(p.solve(c64(y), T.KSPACE_TE))
    for s in range(3):
        ref = O.fista(ys[s], "te", maps[s], mask, phi, 0.02, 8, 15, 3, step=1.0 / L)
        assert nrmse(got[s], ref) < SOLVE_TOL


@pytest.mark.parametrize("ny,nz,b,sy,sz,M,K", [
    (64, 48, 8, 3, 5, 1, 4),
    (60, 36, 8, 7, 2, 1, 4),    # partial blocks on both axes
    (40, 24, 6, 5, 0, 2, 4),    # two map sets
    (48, 30, 8, 1, 6, 1, 6),    # K > 4
    (256, 160, 8, 0, 0, 1, 4),
    (260, 240, 12, 7, 11, 2, 4),  # Table I: 12 x 12 blocks, 260 mod 12 = 8, two map sets
    (8, 8, 16, 13, 9, 1, 2),      # a block larger than the image: shifts beyond its size
    (512, 512, 16, 15, 7, 1, 2),  # the largest matrix and block (K = 2: the band fits shared memory)
    (32, 24, 8, 5, 3, 1, 8),      # K = 8
])
def test_llr_prox_matches_oracle(T, ny, nz, b, sy, sz, M, K):
    rng, phi, mask, maps = random_problem(ny * nz + b, 2, ny, nz, 2, max(K, 8), K, M)
    x = crandn(rng, 2, M, K, ny, nz)
    # blocks with a decaying spectrum so that some singular values fall under tau
    x[..., ::2, :] *= 0.3
    tau = 0.8
    with make_plan(T, phi, mask, maps, block=b) as p:
        xg = c64(x)
        p.llr_prox(xg, tau, sy, sz)
        got = host(xg)
    xs = x.astype(np.complex64).astype(np.complex128)
    for s in range(2):
        ref = O.llr_prox(xs[s], b, tau, sy, sz)
        assert nrmse(got[s], ref) < OP_TOL


def test_solve_largest_matrix(T):
    """512 x 512 slice, K = 4, 8 x 8 blocks, a few iterations against the oracle."""
    rng, phi, mask, maps = random_problem(512, 1, 512, 512, 2, 8, 4, 1)
    y = crandn(rng, 1, 2, 8, 512, 512) * mask[None, None] * 0.1
    with make_plan(T, phi, mask, maps, block=8, lam=0.02, iters=4, seed=9) as p:
        got = host(p.solve(c64(y), T.KSPACE_TE))
        p.sync()
    ref = O.fista(y[0].astype(np.complex64).astype(np.complex128), "te", maps[0], mask, phi, 0.02, 8, 4, 9)
    assert nrmse(got[0], ref) < SOLVE_TOL


def test_llr_prox_limits(T):
    rng, phi, mask, maps = random_problem(3, 1, 32, 32, 2, 8, 4, 1)
    x = crandn(rng, 1, 1, 4, 32, 32)
    with make_plan(T, phi, mask, maps, block=8) as p:
        a = c64(x)
        p.llr_prox(a, 0.0, 2, 3)
        assert nrmse(host(a), x.astype(np.complex64)) < 1e-6
        p.llr_prox(a, 1e6, 2, 3)
        assert float(a.abs().max()) == 0.0


@pytest.mark.parametrize("eig64,fused", [(False, False), (True, False), (False, True), (True, True)])
def test_solve_single_slice_64x48(T, eig64, fused):
    """The 64 x 48, C=8, T=32, K=4, 10 %/echo, lambda=0.01, 50-iteration single slice,
    per-echo (TE-form) input, against the oracle's FISTA; float32 and float64 LLR
    eigendecompositions."""
    sh = synth.SINGLE_SLICE_64x48
    phi, mask, maps, y = te_case(sh)
    phi, maps = r32(phi, maps)
    ys = y.astype(np.complex64).astype(np.complex128)
    ref = O.fista(ys, "te", maps, mask, phi, sh.lam, sh.block, sh.iters, sh.seed)
    flags = (T.EIG_FP64 if eig64 else 0) | (T.FUSED_ROWS if fused else 0)
    with make_plan(T, phi, mask, maps[None], block=sh.block, lam=sh.lam, iters=sh.iters, seed=sh.seed,
                   flags=flags) as p:
        got, res = p.solve(c64(y[None]), T.KSPACE_TE, residual=True)
        got = host(got)[0]
    e = nrmse(got, ref)
    print("single-slice NRMSE", e)
    assert e < SOLVE_TOL
    assert np.all(np.isfinite(res)) and res[-1] < res[1]


def test_solve_batch_ragged_two_maps(T):
    """Several slices at once, partial LLR blocks (60 x 36, b = 8), M = 2, projected input."""
    rng, phi, mask, maps = random_problem(11, 3, 60, 36, 4, 24, 4, 2, frac=0.2)
    psi = O.space_time_kernel(mask, phi)
    a_true = crandn(rng, 3, 2, 4, 60, 36) * 0.05
    ytil = np.stack([O.apply_psi(O.fft2c(O.sense(a_true[s], maps[s])), psi) for s in range(3)])
    ytil += 0.001 * crandn(rng, *ytil.shape) * (psi[..., 0, 0] > 0)
    ys = ytil.astype(np.complex64).astype(np.complex128)
    lam, b, it, seed = 0.02, 8, 30, 77
    with make_plan(T, phi, mask, maps, block=b, lam=lam, iters=it, seed=seed) as p:
        got = host(p.solve(c64(ytil), T.KSPACE_PROJ))
    for s in range(3):
        ref = O.fista(ys[s], "proj", maps[s], mask, phi, lam, b, it, seed)
        assert nrmse(got[s], ref) < SOLVE_TOL


def test_solve_no_shift_and_fixed_step(T):
    rng, phi, mask, maps = random_problem(12, 2, 48, 40, 3, 16, 3, 1, frac=0.3)
    y = crandn(rng, 2, 3, 16, 48, 40) * mask[None, None] * 0.1
    ys = y.astype(np.complex64).astype(np.complex128)
    with make_plan(T, phi, mask, maps, block=8, lam=0.05, iters=20, seed=5, step=0.7, flags=T.NO_SHIFT) as p:
        assert abs(p.step - 0.7) < 1e-7
        got = host(p.solve(c64(y), T.KSPACE_TE))
    for s in range(2):
        ref = O.fista(ys[s], "te", maps[s], mask, phi, 0.05, 8, 20, 5, step=0.7, shifts=False)
        assert nrmse(got[s], ref) < SOLVE_TOL


def test_solve_host_io_matches_device(T):
    sh = synth.SINGLE_SLICE_64x48
    phi, mask, maps, y = te_case(sh)
    kw = dict(block=sh.block, lam=sh.lam, iters=10, seed=sh.seed)
    with make_plan(T, phi, mask, maps[None], **kw) as p:
        dev_out = host(p.solve(c64(y[None]), T.KSPACE_TE))
    d = T.make_dims(64, 48, 8, 32, 4, flags=T.HOST_IO, **kw)
    with T.Plan(d, phi.astype(np.float32), mask.astype(np.uint8), maps[None].astype(np.complex64)) as p:
        host_out = p.solve(y[None].astype(np.complex64), T.KSPACE_TE)
    assert np.array_equal(host_out.astype(np.complex128), dev_out)


def test_solve_host_io_pipelined_matches_device(T):
    """A host-buffer solve of several slices runs in chunks of slices with the copies
    overlapping the work; every slice's result is bitwise the device-buffer solve's, and
    the convergence monitor (a sum over slices, in another order) agrees to rounding."""
    rng, phi, mask, maps = random_problem(41, 11, 48, 40, 3, 16, 4, 1)
    y = crandn(rng, 11, 3, 16, 48, 40) * mask[None, None] * 0.1
    kw = dict(block=8, lam=0.02, iters=12, seed=4)
    with make_plan(T, phi, mask, maps, **kw) as p:
        dev_out, dev_res = p.solve(c64(y), T.KSPACE_TE, residual=True)
        dev_out = host(dev_out)
    d = T.make_dims(48, 40, 3, 16, 4, nslices=11, flags=T.HOST_IO, **kw)
    with T.Plan(d, phi.astype(np.float32), mask.astype(np.uint8), maps.astype(np.complex64)) as p:
        host_out, host_res = p.solve(y.astype(np.complex64), T.KSPACE_TE, residual=True)
        again = p.solve(y.astype(np.complex64), T.KSPACE_TE)   # the plan's stage and streams are reused
    assert np.array_equal(host_out.astype(np.complex128), dev_out)
    assert np.array_equal(again, host_out)
    assert np.allclose(host_res, dev_res, rtol=1e-6, atol=0)


def test_plans_made_on_another_thread_during_a_solve(T):
    """The bench's pipelined host-buffer loop: while one host thread solves scan i through
    host buffers, another makes scan i+1's host-buffer plan on its own stream.  Every result
    equals the same solve made one scan after the other, bitwise."""
    import threading
    import torch
    rng, phi, mask, maps = random_problem(47, 16, 64, 48, 4, 16, 4, 1)
    ys = [(crandn(rng, 16, 4, 4, 64, 48) * 0.05).astype(np.complex64) for _ in range(3)]
    kw = dict(block=8, lam=0.01, iters=10, seed=6)
    d = T.make_dims(64, 48, 4, 16, 4, nslices=16, flags=T.HOST_IO, **kw)
    args = (phi.astype(np.float32), mask.astype(np.uint8), maps.astype(np.complex64))
    ref = []
    for y in ys:
        with T.Plan(d, *args) as p:
            ref.append(p.solve(y, T.KSPACE_PROJ))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    made, errors = {}, []

    def make(i):
        try:
            torch.cuda.set_device(0)
            made[i] = T.Plan(d, *args, stream=streams[i % 2])
        except Exception as e:  # reported on the main thread
            errors.append(e)

    got = []
    worker = threading.Thread(target=make, args=(0,))
    worker.start()
    for i, y in enumerate(ys):
        worker.join()
        assert not errors, errors
        p = made.pop(i)
        if i + 1 < len(ys):
            worker = threading.Thread(target=make, args=(i + 1,))
            worker.start()
        got.append(p.solve(y, T.KSPACE_PROJ))
        p.close()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_solve_zero_iterations_and_empty_mask(T):
    rng, phi, mask, maps = random_problem(13, 1, 32, 32, 2, 8, 4, 1)
    zero_mask = np.zeros_like(mask)
    with make_plan(T, phi, zero_mask, maps, block=8, lam=0.1, iters=5) as p:
        assert p.step == 1.0
        out = host(p.solve(c64(crandn(rng, 1, 2, 8, 32, 32)), T.KSPACE_TE))
    assert np.all(out == 0)
    with make_plan(T, phi, mask, maps, block=8, lam=0.1, iters=0) as p:
        out = host(p.solve(c64(crandn(rng, 1, 2, 8, 32, 32)), T.KSPACE_TE))
    assert np.all(out == 0)


def test_solve_knee_slices_projected(T):
    """Four slices of the 256 x 160, C = 12, T = 80, 5 %/echo knee scan (3D ellipsoid
    phantom, projected input, lambda = 0.005, 100 iterations) against the oracle."""
    sh = synth.KNEE_320x256x160
    sl = [0, 101, 160, 319]
    phi, mask, maps, ytil = proj_scan(sh, sl)
    phi, maps = r32(phi, maps)
    with make_plan(T, phi, mask, maps, block=sh.block, lam=sh.lam, iters=sh.iters, seed=sh.seed) as p:
        got = host(p.solve(c64(ytil), T.KSPACE_PROJ))
    with make_plan(T, phi, mask, maps, block=sh.block, lam=sh.lam, iters=sh.iters, seed=sh.seed,
                   flags=T.FUSED_ROWS) as p:
        got_fused = host(p.solve(c64(ytil), T.KSPACE_PROJ))
    assert nrmse(got_fused, got) < 1e-5
    ys = ytil.astype(np.complex64).astype(np.complex128)
    for i in (0, 3):
        ref = O.fista(ys[i], "proj", maps[i], mask, phi, sh.lam, sh.block, sh.iters, sh.seed)
        e = nrmse(got[i], ref)
        print("knee slice", sl[i], "NRMSE", e)
        assert e < SOLVE_TOL


def full_launch(T, sh, sl, **kw):
    """A whole scan of shape `sh` as one plan (the bench's launch configuration): the listed
    slices from the oracle's own seeded inputs, every other slice a copy of one of them with
    maps and k-space at half scale, so that the plan's shared step 1 / max_s L_s is set by
    the listed slices.  Returns (plan, device k-space, oracle inputs, step)."""
    phi, mask, maps_l, ytil_l = proj_scan(sh, sl)
    phi, maps_l = r32(phi, maps_l)
    S = sh.nslices
    maps_d = torch.empty((S,) + maps_l.shape[1:], dtype=torch.complex64, device="cuda")
    y_d = torch.empty((S,) + ytil_l.shape[1:], dtype=torch.complex64, device="cuda")
    ml, yl = c64(maps_l), c64(ytil_l)
    for s_ in range(S):
        i = sl.index(s_) if s_ in sl else s_ % len(sl)
        f = 1.0 if s_ in sl else 0.5
        maps_d[s_].copy_(ml[i] * f)
        y_d[s_].copy_(yl[i] * f)
    psi = O.space_time_kernel(mask, phi)
    mu = 1.0 / max(O.lipschitz(maps_l[i], psi) for i in range(len(sl)))
    d = T.make_dims(sh.ny, sh.nz, sh.ncoils, sh.nechoes, sh.nbasis, nslices=S, nmaps=sh.nmaps, block=sh.block,
                    lam=sh.lam, iters=sh.iters, seed=sh.seed, **kw)
    p = T.Plan(d, dev(phi.astype(np.float32)), dev(mask.astype(np.uint8)), maps_d)
    assert abs(p.step - mu) <= 1e-5 * mu
    ys = ytil_l.astype(np.complex64).astype(np.complex128)
    return p, y_d, (phi, mask, maps_l, ys), mu


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_full_knee_launch_sampled_slices_match_oracle(T, precision):
    """The knee scan in the launch configuration the bench times: all 320 slices of
    256 x 160 (C = 12, K = 4) in one plan, 100 FISTA iterations, in FP32 and with the
    tensor-core column pass; slices 0 and 319 against the oracle given the plan's step
    (NRMSE <= 1e-4 in FP32, <= 1e-3 mixed)."""
    sh = synth.KNEE_320x256x160
    sl = [0, 101, 160, 319]
    tol = SOLVE_TOL if precision == "fp32" else 1e-3
    p, y_d, (phi, mask, maps_l, ys), mu = full_launch(
        T, sh, sl, precision=T.FP32 if precision == "fp32" else T.MIXED_BF16)
    with p:
        got = p.solve(y_d, T.KSPACE_PROJ)
        out = {s_: host(got[s_]) for s_ in (sl[0], sl[3])}
    for i in (0, 3):
        ref = O.fista(ys[i], "proj", maps_l[i], mask, phi, sh.lam, sh.block, sh.iters, sh.seed, step=mu)
        e = nrmse(out[sl[i]], ref)
        print(f"full knee launch ({precision}), slice", sl[i], "NRMSE", e)
        assert e < tol


def test_full_batch_of_three_scans_sampled_slices_match_oracle(T):
    """The batched workload at full size: 320 x 256x160 C = 12, 288 x 240x128 C = 8 and
    256 x 192x192 C = 16 (100 iterations each) in one batched solve; the last slice of
    every scan against the oracle given its plan's step."""
    plans, ks, cases = [], [], []
    for sh in synth.BATCH_SCANS:
        sl = [sh.nslices // 2, sh.nslices - 1]
        p, y_d, case, mu = full_launch(T, sh, sl)
        plans.append(p)
        ks.append(y_d)
        cases.append((sh, sl, case, mu))
    outs = T.solve_batch(plans, ks)
    last = [host(o[sh.nslices - 1]) for o, (sh, _, _, _) in zip(outs, cases)]
    for p in plans:
        p.close()
    for got, (sh, sl, (phi, mask, maps_l, ys), mu) in zip(last, cases):
        ref = O.fista(ys[1], "proj", maps_l[1], mask, phi, sh.lam, sh.block, sh.iters, sh.seed, step=mu)
        e = nrmse(got, ref)
        print(f"full batch, {sh.ny}x{sh.nz} C={sh.ncoils} slice {sh.nslices - 1} NRMSE {e:.2e}")
        assert e < SOLVE_TOL


def test_solve_paper_shape_slices(T):
    """Two slices of the Table I scan (260 x 240, C = 7, T = 80, K = 4, M = 2 soft-SENSE
    map sets, 12 x 12 LLR blocks, lambda = 0.0125, 1/139 of k-space per echo), projected
    input, the full 250 FISTA iterations of Table I, against the oracle: the iteration
    count at which float32 drift under FISTA's momentum would show."""
    sh = synth.PAPER_288x260x240
    sl = [0, 144]
    phi, mask, maps, ytil = proj_scan(sh, sl)
    phi, maps = r32(phi, maps)
    it = sh.iters
    with make_plan(T, phi, mask, maps, block=sh.block, lam=sh.lam, iters=it, seed=sh.seed) as p:
        got = host(p.solve(c64(ytil), T.KSPACE_PROJ))
    ys = ytil.astype(np.complex64).astype(np.complex128)
    assert np.all(np.isfinite(got))
    i = 1  # the central slice: the oracle needs about half a minute for 250 iterations
    ref = O.fista(ys[i], "proj", maps[i], mask, phi, sh.lam, sh.block, it, sh.seed)
    e = nrmse(got[i], ref)
    print("paper-shape slice", sl[i], "NRMSE", e)
    assert e < SOLVE_TOL


def test_resumable_solve_equals_one_call(T):
    rng, phi, mask, maps = random_problem(31, 2, 64, 48, 4, 16, 4, 1, frac=0.2)
    y = c64(crandn(rng, 2, 4, 16, 64, 48) * mask[None, None] * 0.1)
    kw = dict(block=8, lam=0.02, iters=25, seed=9)
    with make_plan(T, phi, mask, maps, **kw) as p:
        one = host(p.solve(y, T.KSPACE_TE))
        p.solve_begin(y, T.KSPACE_TE)
        assert p.solve_iterate(10) == 10
        assert p.solve_iterate(4) == 14
        assert p.solve_iterate(100) == 25
        parts, res = p.solve_end(residual=True)
        parts = host(parts)
    assert np.array_equal(parts, one)
    assert res.shape == (25,) and np.all(res > 0)


def test_batch_of_uneven_scans_matches_single_solves(T):
    """Three scans of different shapes in one batched solve: bitwise equal to their single
    solves, and the last slice of every scan against the oracle's FISTA."""
    shapes = [(2, 64, 48, 4, 16, 4, 1), (3, 96, 64, 3, 12, 4, 1), (1, 48, 48, 6, 10, 3, 2)]
    plans, ks, singles, refs = [], [], [], []
    for i, (S, ny, nz, C, Tn, K, M) in enumerate(shapes):
        rng, phi, mask, maps = random_problem(200 + i, S, ny, nz, C, Tn, K, M, frac=0.25)
        ytil = c64(crandn(rng, S, C, K, ny, nz) * 0.05)
        kw = dict(block=8, lam=0.01, iters=12 + 3 * i, seed=5 + i)
        p = make_plan(T, phi, mask, maps, **kw)
        singles.append(host(p.solve(ytil, T.KSPACE_PROJ)))
        plans.append(p)
        ks.append(ytil)
        refs.append(O.fista(host(ytil)[S - 1], "proj", maps[S - 1], mask, phi, kw["lam"], kw["block"], kw["iters"],
                            kw["seed"]))
    for per_scan in (False, True):  # the LLR work list, then one LLR launch per scan
        T.batch_schedule(per_scan)
        try:
            outs = T.solve_batch(plans, ks)
        finally:
            T.batch_schedule(False)
        for o, ref, oref in zip(outs, singles, refs):
            got = host(o)
            assert np.array_equal(got, ref)
            e = nrmse(got[-1], oref)
            print("batch scan vs oracle NRMSE", e)
            assert e < SOLVE_TOL
    for p in plans:
        p.close()


def test_batch_with_table1_bands_matches_single_solves(T):
    """A scan with Table I's LLR bands (260 x 240, 12-row bands, two map sets: only two band
    CTAs fit an SM, so the LLR runs 512-thread CTAs) batched with a small scan: the work-list
    launch takes the large band's CTA shape for both; results equal the single solves (each
    with its own CTA shape) bitwise, and the large scan's last slice matches the oracle."""
    shapes = [(2, 260, 240, 2, 12, 4, 2, 12), (2, 64, 48, 3, 12, 4, 1, 8)]
    plans, ks, singles = [], [], []
    ref = None
    for i, (S, ny, nz, C, Tn, K, M, b) in enumerate(shapes):
        rng, phi, mask, maps = random_problem(260 + i, S, ny, nz, C, Tn, K, M, frac=0.25)
        ytil = c64(crandn(rng, S, C, K, ny, nz) * 0.05)
        kw = dict(block=b, lam=0.01, iters=6, seed=7 + i)
        p = make_plan(T, phi, mask, maps, **kw)
        singles.append(host(p.solve(ytil, T.KSPACE_PROJ)))
        plans.append(p)
        ks.append(ytil)
        if i == 0:
            ref = O.fista(host(ytil)[S - 1], "proj", maps[S - 1], mask, phi, kw["lam"], b, kw["iters"], kw["seed"])
    outs = T.solve_batch(plans, ks)
    for o, single in zip(outs, singles):
        assert np.array_equal(host(o), single)
    e = nrmse(host(outs[0])[-1], ref)
    print("Table I bands in a batch vs oracle NRMSE", e)
    assert e < SOLVE_TOL
    for p in plans:
        p.close()


def test_batch_mixing_llr_variants_falls_back_to_per_scan_launches(T):
    """A batch whose plans take different LLR variants (float64 eigen-step in one of them)
    runs one LLR launch per scan; results still equal the single solves bitwise."""
    plans, ks, singles = [], [], []
    for i, flags in enumerate((0, T.EIG_FP64)):
        rng, phi, mask, maps = random_problem(230 + i, 2, 64, 48, 3, 12, 4, 1, frac=0.25)
        ytil = c64(crandn(rng, 2, 3, 4, 64, 48) * 0.05)
        p = make_plan(T, phi, mask, maps, block=8, lam=0.01, iters=8, seed=11 + i, flags=flags)
        singles.append(host(p.solve(ytil, T.KSPACE_PROJ)))
        plans.append(p)
        ks.append(ytil)
    outs = T.solve_batch(plans, ks)
    for o, ref in zip(outs, singles):
        assert np.array_equal(host(o), ref)
    for p in plans:
        p.close()


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_batch_of_the_three_scan_shapes_matches_oracle(T, precision):
    """The batched-scan workload's three shapes (256x160 with C = 12, 240x128 with C = 8,
    192x192 with C = 16; T = 80, K = 4, 5 %/echo, lambda = 0.005) in one batched solve,
    two slices of each scan, 15 FISTA iterations, every slice against the oracle:
    NRMSE <= 1e-4 in FP32, <= 1e-3 with the tensor-core column pass."""
    it = 15
    tol = SOLVE_TOL if precision == "fp32" else 1e-3
    prec = T.FP32 if precision == "fp32" else T.MIXED_BF16
    plans, ks, cases = [], [], []
    for sh in synth.BATCH_SCANS:
        sl = [sh.nslices // 2, sh.nslices - 1]
        phi, mask, maps, ytil = proj_scan(sh, sl)
        phi, maps = r32(phi, maps)
        plans.append(make_plan(T, phi, mask, maps, block=sh.block, lam=sh.lam, iters=it, seed=sh.seed,
                               precision=prec))
        ks.append(c64(ytil))
        cases.append((sh, phi, mask, maps, ytil.astype(np.complex64).astype(np.complex128)))
    outs = T.solve_batch(plans, ks)
    for o, (sh, phi, mask, maps, ys) in zip(outs, cases):
        got = host(o)
        for i in range(got.shape[0]):
            ref = O.fista(ys[i], "proj", maps[i], mask, phi, sh.lam, sh.block, it, sh.seed)
            e = nrmse(got[i], ref)
            print(f"{sh.ny}x{sh.nz} C={sh.ncoils} slice {i} ({precision}) NRMSE {e:.2e}")
            assert e < tol
    for p in plans:
        p.close()


def test_autotuned_plan_still_matches_oracle(T):
    sh = synth.SINGLE_SLICE_64x48
    phi, mask, maps, y = te_case(sh)
    phi, maps = r32(phi, maps)
    ys = y.astype(np.complex64).astype(np.complex128)
    ref = O.fista(ys, "te", maps, mask, phi, sh.lam, sh.block, sh.iters, sh.seed)
    with make_plan(T, phi, mask, maps[None], block=sh.block, lam=sh.lam, iters=sh.iters, seed=sh.seed) as p:
        var, fused = p.autotune(probe_iters=-1)
        assert var in (0, 1, 2, 4) and fused in (False, True)
        got = host(p.solve(c64(y[None]), T.KSPACE_TE))[0]
        p.sync()
    assert nrmse(got, ref) < SOLVE_TOL


@pytest.mark.parametrize("variant", [0, 1, 2, 4])
@pytest.mark.parametrize("ny,nz,K", [(256, 160, 4), (256, 160, 2), (260, 240, 4), (260, 40, 3), (240, 128, 3),
                                     (64, 48, 4), (96, 36, 2), (192, 64, 4), (240, 96, 4), (48, 40, 4), (128, 24, 4),
                                     (96, 16, 4), (160, 8, 4)])
def test_column_variants_match_oracle(T, variant, ny, nz, K):
    """Every normal-operator column-pass variant (TMA x8, cp.async x8, cp.async x4, TMA x4)
    on every size-specialised column length; nz = 36 is not a multiple of 8, so the
    8-column variants fall back there.  At 260 rows the TMA variants copy each column as two
    boxes and the cp.async variants run the 20 x 13 kernel."""
    rng, phi, mask, maps = random_problem(300 + ny + variant, 2, ny, nz, 3, 12, K, 1)
    x = crandn(rng, 2, 1, K, ny, nz)
    with make_plan(T, phi, mask, maps) as p:
        p.configure(variant)
        got = host(p.normal_op(c64(x)))
        p.sync()
    psi = O.space_time_kernel(mask, phi)
    xs = x.astype(np.complex64).astype(np.complex128)
    for s in range(2):
        assert nrmse(got[s], O.normal(xs[s], maps[s], psi)) < OP_TOL
