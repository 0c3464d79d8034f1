"""The synthetic input recipe (stand-ins for the paper's knee scans): properties the tests,
the bench and the step bound rely on.  The generator holds no reconstruction arithmetic;
these checks pin what it promises."""
import numpy as np
import pytest

import t2sh_synth as synth


@pytest.mark.parametrize("T,K", [(80, 4), (32, 4), (12, 3)])
def test_t2_basis_orthonormal_signed_and_spanning_decays(T, K):
    phi = synth.t2_basis(T, K)
    assert phi.shape == (T, K)
    assert np.abs(phi.T @ phi - np.eye(K)).max() < 1e-12
    for k in range(K):
        assert phi[np.argmax(np.abs(phi[:, k])), k] > 0
    te = synth.echo_times_ms(T)
    for t2 in (25.0, 60.0, 150.0):   # decays inside the training range are captured
        s = np.exp(-te / t2)
        r = s - phi @ (phi.T @ s)
        assert np.linalg.norm(r) < 2e-2 * np.linalg.norm(s)


@pytest.mark.parametrize("M", [1, 2])
def test_coil_maps_normalised_for_the_step_bound(M):
    """max eigenvalue of S(p)^H S(p) is 1 at every pixel, so the Lipschitz bound of the
    data term is at most 1 and the plan's step is 1 with the maps alone."""
    rng = np.random.default_rng(3)
    maps = synth.coil_maps(8, 24, 20, rng, M=M)
    assert maps.shape == (8, M, 24, 20)
    sp = np.moveaxis(maps, (0, 1), (-2, -1))  # [y][z][C][M]
    lam = np.linalg.eigvalsh(np.conj(np.swapaxes(sp, -1, -2)) @ sp).max(-1)
    assert np.abs(lam - 1.0).max() < 1e-12


@pytest.mark.parametrize("frac,T,ny,nz", [(0.05, 80, 256, 160), (1.0 / 139.0, 80, 260, 240), (0.10, 32, 64, 48)])
def test_sampling_fraction_centre_and_density(frac, T, ny, nz):
    rng = np.random.default_rng(11)
    m = synth.vd_masks(T, ny, nz, frac, rng)
    assert m.dtype == np.uint8 and set(np.unique(m)) <= {0, 1}
    # the calibration square of echo 0 adds at most 36 samples to the target fraction
    assert abs(m[1:].mean() - frac) < 0.1 * frac
    c0y, c0z = ny // 2 - 3, nz // 2 - 3
    assert m[0, c0y:c0y + 6, c0z:c0z + 6].all()
    centre = m[:, ny // 2 - ny // 8:ny // 2 + ny // 8, nz // 2 - nz // 8:nz // 2 + nz // 8].mean()
    edge = np.concatenate([m[:, :ny // 8].ravel(), m[:, -(ny // 8):].ravel()]).mean()
    assert centre > 3 * edge


def test_scan_inputs_are_seeded():
    a = synth.scan_common(synth.KNEE_320x256x160)
    b = synth.scan_common(synth.KNEE_320x256x160)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    s1 = synth.slice_structure(synth.SINGLE_SLICE_64x48, 0)
    s2 = synth.slice_structure(synth.SINGLE_SLICE_64x48, 0)
    assert np.array_equal(s1.maps, s2.maps) and np.array_equal(s1.rho, s2.rho)
    s3 = synth.slice_structure(synth.SINGLE_SLICE_64x48, 1)
    assert not np.array_equal(s1.maps, s3.maps)


def test_complex_noise_power():
    w = synth.complex_noise((400000,), 0.3, np.random.default_rng(5))
    assert abs(np.mean(np.abs(w) ** 2) - 0.09) < 0.02 * 0.09
    assert abs(np.mean(w.real ** 2) - np.mean(w.imag ** 2)) < 0.02 * 0.045


def test_paper_shape_matches_table_one():
    p = synth.PAPER_288x260x240
    assert (p.nslices, p.ny, p.nz, p.ncoils, p.nechoes, p.nbasis, p.nmaps, p.block, p.iters) == \
        (288, 260, 240, 7, 80, 4, 2, 12, 250)
    assert p.lam == pytest.approx(0.0125) and p.frac == pytest.approx(1.0 / 139.0)
