"""GPU parity of the wavelet soft-threshold of the coefficient volume (t2sh_wavelet_denoise:
orthonormal 3D Haar pyramid over (slice, y, z), complex soft threshold of the details,
inverse) against the oracle's wavelet_denoise().  Inputs are random complex volumes and
the seeded phantom's coefficient images, both built on the host without the library.

Tolerance: at most 2 x levels float32 butterfly passes of three additions each and one
threshold per coefficient: NRMSE <= 1e-6 (soft thresholding is continuous, so a
coefficient near tau moves the result by a rounding error at most)."""
import numpy as np
import pytest

import oracle as O
import t2sh_synth as synth

from t2sh_cases import crandn
from test_gpu_parity import T, c64, make_plan, nrmse, random_problem  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WAV_TOL = 1e-6


def detail_scale(a, levels):
    """A threshold that zeroes some detail coefficients and shrinks the others: the median
    magnitude of the finest-level details of the first image."""
    c = O.haar3(a[:, 0, 0], 1)
    n = [m // 2 for m in c.shape]
    return float(np.median(np.abs(c[n[0]:, :, :])))


@pytest.mark.parametrize("S,M,K,ny,nz,levels", [
    (8, 1, 4, 16, 24, 1),
    (8, 2, 3, 16, 24, 2),
    (8, 1, 2, 16, 24, 3),
    (16, 1, 1, 16, 16, 4),   # one approximation coefficient per image
    (4, 2, 4, 64, 48, 2),
])
def test_wavelet_denoise_matches_oracle(T, S, M, K, ny, nz, levels):
    rng, phi, mask, maps = random_problem(900 + S + ny + levels, S, ny, nz, 2, 8, K, M)
    a = crandn(rng, S, M, K, ny, nz)
    a32 = a.astype(np.complex64).astype(np.complex128)
    tau = detail_scale(a32, levels)
    with make_plan(T, phi, mask, maps) as p:
        x = c64(a)
        p.wavelet_denoise(x, tau, levels)
        got = x.cpu().numpy().astype(np.complex128)
        p.sync()
    ref = O.wavelet_denoise(a32, float(np.float32(tau)), levels)
    e = nrmse(got, ref)
    print(f"wavelet {S}x{ny}x{nz} M={M} K={K} L={levels}: NRMSE {e:.2e}")
    assert e < WAV_TOL
    with make_plan(T, phi, mask, maps) as p:  # tau = 0: the identity up to rounding
        x = c64(a)
        p.wavelet_denoise(x, 0.0, levels)
        assert nrmse(x.cpu().numpy().astype(np.complex128), a32) < WAV_TOL


def test_wavelet_denoise_phantom_coefficients(T):
    """The coefficient images Phi^T x of 16 slices of the seeded 3D knee phantom (x the
    echo series), three levels, tau at the detail median."""
    sh = synth.KNEE_320x256x160
    phi, mask, te = synth.scan_common(sh)
    vol = synth.EllipsoidVolume.draw(synth.rng_for(sh.seed, 4, 0))
    sl = range(152, 168)
    a = np.zeros((len(sl), 1, sh.nbasis, sh.ny, sh.nz), np.complex128)
    maps = []
    for i, s in enumerate(sl):
        st = synth.slice_structure(sh, s, volume=vol)
        a[i, 0] = np.einsum("tk,tyz->kyz", phi, synth.decay_series(st.rho, st.t2, te))
        maps.append(st.maps)
    a32 = a.astype(np.complex64).astype(np.complex128)
    tau = detail_scale(a32, 3)
    with make_plan(T, phi, mask, np.stack(maps)) as p:
        x = c64(a)
        p.wavelet_denoise(x, tau, 3)
        got = x.cpu().numpy().astype(np.complex128)
    ref = O.wavelet_denoise(a32, float(np.float32(tau)), 3)
    e = nrmse(got, ref)
    print("phantom coefficients NRMSE", e)
    assert e < WAV_TOL
    assert 0.0 < nrmse(ref, a32) < 1.0  # the threshold did something, not everything


def test_wavelet_denoise_full_knee_volume_sampled_blocks(T):
    """The whole knee volume (320 slices of 256 x 160, K = 4) at three levels; the pyramid
    acts on aligned 8 x 8 x 8 cubes independently, so the oracle checks sampled cubes from
    their own inputs alone."""
    S, M, K, ny, nz, lev = 320, 1, 4, 256, 160, 3
    gen = torch.Generator(device="cuda")
    gen.manual_seed(77)
    x = torch.randn((S, M, K, ny, nz), dtype=torch.complex64, device="cuda", generator=gen)
    a = x.clone()
    rng = np.random.default_rng(5)
    _, phi, mask, maps = random_problem(5, 1, ny, nz, 1, 8, K, M)
    maps = np.repeat(maps, S, axis=0)
    tau = 0.3
    with make_plan(T, phi, mask, maps) as p:
        p.wavelet_denoise(x, tau, lev)
        p.sync()
    for _ in range(6):
        i, j, k = (int(rng.integers(0, n // 8)) * 8 for n in (S, ny, nz))
        blk_in = a[i:i + 8, :, :, j:j + 8, k:k + 8].cpu().numpy().astype(np.complex128)
        blk_out = x[i:i + 8, :, :, j:j + 8, k:k + 8].cpu().numpy().astype(np.complex128)
        ref = O.wavelet_denoise(blk_in, tau, lev)
        assert nrmse(blk_out, ref) < WAV_TOL


def test_wavelet_denoise_rejects_bad_arguments(T):
    rng, phi, mask, maps = random_problem(950, 6, 16, 24, 2, 8, 2, 1)
    with make_plan(T, phi, mask, maps) as p:
        x = c64(crandn(rng, 6, 1, 2, 16, 24))
        with pytest.raises(T.T2shError) as ei:
            p.wavelet_denoise(x, 0.1, 2)  # 6 slices are not a multiple of 4
        assert ei.value.status == T.EINVAL
        with pytest.raises(T.T2shError) as ei:
            p.wavelet_denoise(x, -1.0, 1)
        assert ei.value.status == T.EINVAL
        p.wavelet_denoise(x, 0.1, 1)  # 6, 16, 24 are even: one level works
        p.sync()
        lib = T.lib()
        import ctypes
        st = lib.t2sh_wavelet_denoise(p._h, ctypes.c_void_p(x.data_ptr() + 8), ctypes.c_float(0.1), 1)
        assert st == T.EINVAL and "aligned" in T.last_error()  # 8 bytes off a 16-byte boundary
    d = T.make_dims(16, 24, 2, 8, 2, nslices=6, flags=T.HOST_IO)
    with T.Plan(d, phi.astype(np.float32), mask, maps.astype(np.complex64)) as p:
        with pytest.raises(T.T2shError) as ei:
            p.wavelet_denoise(torch.zeros((6, 1, 2, 16, 24), dtype=torch.complex64, device="cuda"), 0.1, 1)
        assert ei.value.status == T.EUNSUPPORTED
