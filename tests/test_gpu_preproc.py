"""GPU parity of the pre-processing steps (t2sh_coil_compression, t2sh_preprocess) against
the oracle, from a sparse array of readout lines in a shuffled order.

Tolerances: compression matrix entries within 1e-4 (float32 calibration sums feeding a
float64 eigensolver; eigenvalues well separated); projected k-space NRMSE <= 1e-5 (a
Ctot-term compression, one float32 DFT along x, a few-term projection); masks bit-exact."""
import numpy as np
import pytest

import oracle as O
import t2sh_synth as synth

from t2sh_cases import crandn
from test_gpu_parity import T, c64, dev, host, make_plan, nrmse  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sparse_scan(seed, nchan, nx, ny, nz, Tn, frac, ncoil_rank=4):
    """Lines of a synthetic acquisition: channel data of rank ncoil_rank plus noise (so the
    channel covariance has well separated leading eigenvalues), sampled at a random mask,
    shuffled.  Returns float32-representable lines [n][nchan][nx] and the indices."""
    rng = np.random.default_rng(seed)
    mask = (rng.random((Tn, ny, nz)) < frac).astype(np.uint8)
    mask[:, ny // 2 - 2:ny // 2 + 2, nz // 2 - 2:nz // 2 + 2] = 1   # a sampled centre
    t, a, b = np.nonzero(mask)
    order = rng.permutation(len(t))
    t, a, b = t[order], a[order], b[order]
    B = crandn(rng, ncoil_rank, nchan) * np.geomspace(4.0, 0.5, ncoil_rank)[:, None]
    src = crandn(rng, len(t), ncoil_rank, nx)
    lines = np.einsum("jrx,rc->jcx", src, B) + 0.05 * crandn(rng, len(t), nchan, nx)
    lines = lines.astype(np.complex64).astype(np.complex128)
    return lines, t.astype(np.int32), a.astype(np.int32), b.astype(np.int32), mask


@pytest.mark.parametrize("nchan,nx,ny,nz,win,ncomp", [(8, 24, 20, 16, 8, 4), (16, 288, 26, 24, 12, 7),
                                                       (12, 260, 20, 18, 10, 5)])
def test_coil_compression_matches_oracle(T, nchan, nx, ny, nz, win, ncomp):
    """The channel data have rank ncomp + 1 with geometrically spaced energies (plus weak
    noise), so the ncomp leading eigenvectors are well separated and defined to float
    precision; beyond the signal rank they would span a near-degenerate noise subspace."""
    lines, t, a, b, mask = sparse_scan(nchan + nx, nchan, nx, ny, nz, 10, 0.3, ncoil_rank=ncomp + 1)
    W = T.coil_compression(c64(lines), t, a, b, ny, nz, 10, window=win, ncomp=ncomp)
    torch.cuda.synchronize()
    ref = O.compression_matrix(O.calibration_average(lines, a, b, ny, nz, win), ncomp)
    got = host(W)
    print(f"nchan={nchan} nx={nx}: max |W - W_ref| = {np.abs(got - ref).max():.2e}")
    assert np.abs(got - ref).max() < 1e-4
    assert np.abs(got.conj().T @ got - np.eye(ncomp)).max() < 1e-5
    assert np.abs(got @ got.conj().T - ref @ ref.conj().T).max() < 1e-4


@pytest.mark.parametrize("nchan,ncomp,nx,ny,nz,Tn,K", [(8, 4, 24, 20, 16, 10, 3), (16, 7, 288, 26, 24, 12, 4),
                                                       (6, 6, 260, 14, 12, 8, 4)])
def test_preprocess_matches_oracle(T, nchan, ncomp, nx, ny, nz, Tn, K):
    lines, t, a, b, mask = sparse_scan(3 * nx + nchan, nchan, nx, ny, nz, Tn, 0.25)
    rng = np.random.default_rng(nx)
    W = np.linalg.qr(crandn(rng, nchan, ncomp))[0].astype(np.complex64).astype(np.complex128)
    phi = synth.t2_basis(Tn, K).astype(np.float32).astype(np.float64)
    ytil, m = T.preprocess(c64(lines), t, a, b, c64(W), dev(phi.astype(np.float32)), ny, nz)
    ref, mref = O.preprocess(lines, t, a, b, W, phi, ny, nz)
    assert np.array_equal(m.cpu().numpy(), mref)
    assert np.array_equal(mref, mask)
    e = nrmse(host(ytil), ref)
    print(f"preprocess nx={nx}: NRMSE {e:.2e}")
    assert e < 1e-5


def test_preprocess_repeated_lines_add(T):
    lines, t, a, b, mask = sparse_scan(7, 4, 16, 8, 8, 4, 0.3)
    lines2 = np.concatenate([lines, lines[:5]])
    t2, a2, b2 = (np.concatenate([v, v[:5]]) for v in (t, a, b))
    W = np.eye(4, 2, dtype=np.complex128)
    phi = synth.t2_basis(4, 2).astype(np.float32).astype(np.float64)
    ytil, _ = T.preprocess(c64(lines2), t2, a2, b2, c64(W), dev(phi.astype(np.float32)), 8, 8)
    ref, _ = O.preprocess(lines2, t2, a2, b2, W, phi, 8, 8)
    assert nrmse(host(ytil), ref) < 1e-5


def test_sparse_lines_to_reconstruction(T):
    """Chain: sparse lines of a synthetic scan (fully sampled readout, per-echo masks) ->
    coil compression -> decoupling and projection -> FISTA on three readout slices, against
    the oracle's chain on the same lines."""
    rng = np.random.default_rng(44)
    nchan, C, nx, ny, nz, Tn, K = 8, 4, 16, 48, 40, 16, 4
    phi = synth.t2_basis(Tn, K)
    mask = synth.vd_masks(Tn, ny, nz, 0.15, rng)
    # a 3D scene: per readout position x, a 2D decay series seen by nchan smooth coils
    maps3 = np.stack([synth.coil_maps(nchan, ny, nz, rng) for _ in range(nx)])   # [x][Ctot][1][y][z]
    rho, t2 = synth.ellipse_phantom(ny, nz, rng)
    xt = synth.decay_series(rho, t2, synth.echo_times_ms(Tn))                     # [T][y][z]
    img = np.einsum("xcyz,tyz->ctxyz", maps3[:, :, 0], xt)                        # [Ctot][T][x][y][z]
    k3 = np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(img, axes=(2, 3, 4)), axes=(2, 3, 4), norm="ortho"),
                         axes=(2, 3, 4))
    t, a, b = np.nonzero(mask)
    lines = np.stack([k3[:, t[j], :, a[j], b[j]] for j in range(len(t))])
    lines = lines / np.abs(lines).max()
    lines = lines.astype(np.complex64).astype(np.complex128)
    t, a, b = t.astype(np.int32), a.astype(np.int32), b.astype(np.int32)
    W = T.coil_compression(c64(lines), t, a, b, ny, nz, Tn, window=12, ncomp=C)
    ytil, m = T.preprocess(c64(lines), t, a, b, W, dev(phi.astype(np.float32)), ny, nz)
    Wh = host(W)
    ref_y, ref_m = O.preprocess(lines, t, a, b, Wh, phi.astype(np.float32).astype(np.float64), ny, nz)
    assert np.array_equal(m.cpu().numpy(), ref_m)
    assert nrmse(host(ytil), ref_y) < 1e-5
    # maps of the virtual coils: the compressed physical maps, normalised per pixel
    sl = [3, 8, 12]
    vm = np.einsum("xcyz,cd->xdyz", maps3[sl, :, 0], Wh)
    vm = vm / np.sqrt((np.abs(vm) ** 2).sum(1, keepdims=True))
    vm = vm[:, :, None].astype(np.complex64).astype(np.complex128)
    phi32 = phi.astype(np.float32).astype(np.float64)
    with make_plan(T, phi32, mask, vm, block=8, lam=0.01, iters=15, seed=2) as p:
        got = host(p.solve(ytil[sl].contiguous(), T.KSPACE_PROJ))
    ys = host(ytil)[sl]
    for i in range(len(sl)):
        ref = O.fista(ys[i], "proj", vm[i], mask, phi32, 0.01, 8, 15, 2)
        assert nrmse(got[i], ref) < 1e-4


def test_preprocess_rejects_bad_input(T):
    lines, t, a, b, mask = sparse_scan(5, 4, 16, 8, 8, 4, 0.3)
    L = c64(lines)
    bad = a.copy()
    bad[0] = 8
    with pytest.raises(T.T2shError):
        T.coil_compression(L, t, bad, b, 8, 8, 4, window=4, ncomp=2)
    with pytest.raises(T.T2shError):   # no line in a 1 x 1 x 1 window at an unsampled centre?  use ncomp > nchan
        T.coil_compression(L, t, a, b, 8, 8, 4, window=4, ncomp=5)
    phi = dev(synth.t2_basis(4, 2).astype(np.float32))
    with pytest.raises(T.T2shError):   # nx = 14 = 2 * 7 is not a product of 2, 3, 5, 13
        l14 = c64(lines[:, :, :14].copy())
        T.preprocess(l14, t, a, b, c64(np.eye(4, 2)), phi, 8, 8)
