"""Synthetic acquisitions for the tests and the CPU baseline (test infrastructure).

Structure (basis, phantom, maps, masks, noise) comes from the seeded generator
``t2sh_synth``; the acquisition itself (Eq. 1 per echo, or its projection Phi^T P y)
is computed with this oracle's float64 operators, so no parity input ever comes from
the CUDA path.  Same import rules as the rest of ``oracle/``.
"""
from __future__ import annotations

import numpy as np

import t2sh_synth as synth

from . import t2sh_oracle as O


def te_case(shape: synth.ScanShape, s: int = 0, sigma_frac: float = 0.01):
    """One slice with per-echo data y_t = P_t F S x_t + P_t w_t, x_t = rho exp(-t/T2)
    (not confined to the subspace), sigma = sigma_frac * max|noiseless sample|, then
    scaled by 1 / max |y| over acquired samples.
    Returns phi [T][K], mask [T][ny][nz], maps [C][M][ny][nz], y [C][T][ny][nz] (complex128)."""
    phi, mask, te = synth.scan_common(shape)
    st = synth.slice_structure(shape, s)
    xt = synth.decay_series(st.rho, st.t2, te)  # [T][ny][nz]
    x = np.zeros((shape.nmaps,) + xt.shape, np.complex128)
    x[0] = xt
    y0 = O.sense_forward(x, st.maps, mask)
    sig = sigma_frac * np.abs(y0).max()
    w = synth.complex_noise(y0.shape, sig, synth.rng_for(shape.seed, 3, s))
    y = y0 + mask[None] * w
    y = y / np.abs(y).max()
    return phi, mask, st.maps, y


def proj_scan(shape: synth.ScanShape, slices, sigma_frac: float = 0.01, volume_seed_word: int = 4):
    """Projected k-space ytil = Phi^T P (F S x + w) for the listed slices of a 3D
    phantom scan, in-subspace model x = Phi alpha_true with alpha_true = Phi^T x_t.
    The projected noise Phi^T P w, w ~ CN(0, sigma^2 I_T), is drawn with its exact
    distribution CN(0, sigma^2 Psi(n)) as Psi(n)^(1/2) xi, xi ~ CN(0, I_K).
    sigma = sigma_frac * max |echo-0 noiseless sample| of the central slice; the data are
    scaled by 1 / max |ytil| over the listed slices and the central slice.
    Returns phi, mask, maps [S][C][M][ny][nz], ytil [S][C][K][ny][nz] (complex128)."""
    phi, mask, te = synth.scan_common(shape)
    vol = synth.EllipsoidVolume.draw(synth.rng_for(shape.seed, volume_seed_word, 0))
    psi = O.space_time_kernel(mask, phi)
    ev, V = np.linalg.eigh(psi)
    root = (V * np.sqrt(np.clip(ev, 0, None))[..., None, :]) @ np.swapaxes(V, -1, -2)  # Psi^(1/2)

    def clean(s):
        st = synth.slice_structure(shape, s, volume=vol)
        xt = synth.decay_series(st.rho, st.t2, te)
        alpha = np.einsum("tk,tyz->kyz", phi, xt)[None]  # [1][K][..]
        if shape.nmaps > 1:
            alpha = np.concatenate([alpha, np.zeros((shape.nmaps - 1,) + alpha.shape[1:])], 0)
        fsa = O.fft2c(O.sense(alpha, st.maps))  # [C][K][..]
        echo0 = mask[0][None] * np.einsum("k,ckyz->cyz", phi[0], fsa)
        return st.maps, O.apply_psi(fsa, psi), np.abs(echo0).max()

    centre = shape.nslices // 2
    _, c_clean, c_echo0 = clean(centre)
    sig = sigma_frac * c_echo0

    def noisy(s, cl):
        xi = synth.complex_noise(cl.shape, 1.0, synth.rng_for(shape.seed, 5, s))  # [C][K][..]
        return cl + sig * np.einsum("yzkl,clyz->ckyz", root, xi)

    maps_all, out = [], []
    for s in slices:
        m, cl, _ = clean(s)
        maps_all.append(m)
        out.append(noisy(s, cl))
    scale = 1.0 / max(np.abs(noisy(centre, c_clean)).max(), max(np.abs(o).max() for o in out))
    return phi, mask, np.stack(maps_all), np.stack(out) * scale
