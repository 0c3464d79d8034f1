"""FP64 CPU oracle of the T2 Shuffling subspace-constrained LLR PICS solve.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
CUDA library never calls into this file and this file never calls into the CUDA
library: the two share no code, headers, tables or helpers.

Every function works on ONE decoupled readout slice (the 2D (ky, kz) problem left
after the inverse FFT along the fully sampled readout, Sec. II.A and Sec. III.B) in
complex128 / float64, with plain numpy primitives (``numpy.fft``, ``numpy.linalg``)
as steps.  Notation follows the paper:

    alpha  [M][K][Ny][Nz]   basis-coefficient images (Eq. 3, M soft-SENSE sets)
    maps   [C][M][Ny][Nz]   coil sensitivities S_{c,m} (Eq. 1, soft-SENSE Sec. II.A)
    mask   [T][Ny][Nz]      one-zero sampling pattern P_t per echo, centred k-space
    phi    [T][K]           real temporal basis Phi (Eq. 3)
    y      [C][T][Ny][Nz]   zero-filled k-space per coil and echo (Eq. 1)
    ytil   [C][K][Ny][Nz]   projected k-space Phi^T P y (re-sort and project, Sec. III.A)

Readings of the paper taken where it is silent:
  * F is the centred, unitary 2D DFT: fftshift . DFT . ifftshift / sqrt(Ny Nz).
  * The LLR random shift of iteration ``it`` is drawn from SplitMix64 (below); block
    (i, j) covers rows (sy + i b + r) mod Ny and columns (sz + j b + c) mod Nz; the
    last block along an axis is partial when b does not divide the size.
  * With M > 1 map sets the LLR takes each set's K images as its own blocks.
  * FISTA (Beck-Teboulle) starts from x0 = z0 = 0, t0 = 1, no restart; step 1/L with
    L = max_n lambda_max(Psi(n)) * max_p lambda_max(S(p)^H S(p)); threshold mu*lambda.

Parity pins live in ``tests/test_oracle_pins.py``; the functions below have none of
their own checks beyond argument validation.
"""
from __future__ import annotations

import numpy as np

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


# ---------------------------------------------------------------------------------
# Random LLR shifts (Sec. IV.C: "circular-shifted randomly ... by a small amount less
# than the patch size").  The paper names no generator; this oracle uses SplitMix64
# (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
# written here from its published definition.
# ---------------------------------------------------------------------------------
def splitmix64(seed: int, n: int) -> list[int]:
    """First ``n`` outputs of SplitMix64 started from state ``seed``."""
    state = seed & _M64
    out = []
    for _ in range(n):
        state = (state + _GOLDEN) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out.append(z ^ (z >> 31))
    return out


def llr_shifts(seed: int, iters: int, b: int) -> np.ndarray:
    """Shift pair (sy, sz) of every iteration: output it+1 of SplitMix64(seed),
    low 32 bits mod b -> sy, high 32 bits mod b -> sz.  Returns int64 [iters][2]."""
    h = splitmix64(seed, iters)
    return np.array([[(v & 0xFFFFFFFF) % b, (v >> 32) % b] for v in h], dtype=np.int64).reshape(iters, 2)


# ---------------------------------------------------------------------------------
# Fourier transform F (Eq. 1): 2D DFT over the phase-encode plane, centred as the
# FFTmod step of Sec. IV.A implies, unitary as the readout transform of Sec. III.B.
# ---------------------------------------------------------------------------------
def fft2c(x: np.ndarray) -> np.ndarray:
    """Centred unitary 2D DFT over the last two axes."""
    ax = (-2, -1)
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(x, axes=ax), axes=ax, norm="ortho"), axes=ax)


def ifft2c(k: np.ndarray) -> np.ndarray:
    """Adjoint (= inverse) of :func:`fft2c`."""
    ax = (-2, -1)
    return np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(k, axes=ax), axes=ax, norm="ortho"), axes=ax)


# ---------------------------------------------------------------------------------
# Sensitivity operator S (Eq. 1 with the soft-SENSE stacking of Sec. II.A).
# ---------------------------------------------------------------------------------
def sense(x: np.ndarray, maps: np.ndarray) -> np.ndarray:
    """S x: x [M][...][Ny][Nz] -> coil images [C][...][Ny][Nz], sum_m S_{c,m} x_m."""
    C, M = maps.shape[:2]
    assert x.shape[0] == M
    extra = x.ndim - 3
    s = maps.reshape((C, M) + (1,) * extra + maps.shape[2:])
    return np.sum(s * x[None], axis=1)


def sense_adj(xc: np.ndarray, maps: np.ndarray) -> np.ndarray:
    """S^H: coil images [C][...][Ny][Nz] -> [M][...][Ny][Nz], sum_c conj(S_{c,m}) x_c."""
    C, M = maps.shape[:2]
    assert xc.shape[0] == C
    extra = xc.ndim - 3
    s = np.conj(maps).reshape((C, M) + (1,) * extra + maps.shape[2:])
    return np.sum(s * xc[:, None], axis=0)


# ---------------------------------------------------------------------------------
# Forward model of Eq. 5, A = P F S Phi, and its adjoint, written out literally
# (the echo loop is explicit: each echo image is passed through Eq. 1 on its own).
# ---------------------------------------------------------------------------------
def backproject(alpha: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Eq. 3: x(n) = Phi alpha(n).  alpha [M][K][..] -> x [M][T][..]."""
    return np.einsum("tk,mk...->mt...", phi, alpha)


def sense_forward(x: np.ndarray, maps: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Eq. 1 per echo: y_{c,t} = P_t F (sum_m S_{c,m} x_{m,t}).
    x [M][T][Ny][Nz] -> y [C][T][Ny][Nz] (zero-filled)."""
    return mask[None].astype(np.float64) * fft2c(sense(x, maps))


def forward(alpha: np.ndarray, maps: np.ndarray, mask: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """A alpha = P F S Phi alpha (Eq. 5).  alpha [M][K][Ny][Nz] -> y [C][T][Ny][Nz]."""
    return sense_forward(backproject(alpha, phi), maps, mask)


def adjoint(y: np.ndarray, maps: np.ndarray, mask: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """A^H y = Phi^T S^H F^H P y.  y [C][T][Ny][Nz] -> [M][K][Ny][Nz]."""
    xt = sense_adj(ifft2c(mask[None].astype(np.float64) * y), maps)  # [M][T][..]
    return np.einsum("tk,mt...->mk...", phi, xt)


def normal_explicit(alpha: np.ndarray, maps: np.ndarray, mask: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """A^H A alpha through all T echoes (the plain definition; slow)."""
    return adjoint(forward(alpha, maps, mask, phi), maps, mask, phi)


# ---------------------------------------------------------------------------------
# Space-time kernel (Sec. IV.B): Psi(n) = Phi^T P(n) Phi, and the normal operator
# S^H F^H Psi F S that the commutation F S Phi = Phi F S turns A^H A into.
# ---------------------------------------------------------------------------------
def space_time_kernel(mask: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Psi [Ny][Nz][K][K] with Psi(n)_{kl} = sum_t Phi_{tk} P_t(n) Phi_{tl}."""
    return np.einsum("tk,tyz,tl->yzkl", phi, mask.astype(np.float64), phi)


def project(y: np.ndarray, mask: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Re-sort and project (Sec. III.A): ytil_{c,k}(n) = sum_t Phi_{tk} P_t(n) y_{c,t}(n)."""
    return np.einsum("tk,tyz,ctyz->ckyz", phi, mask.astype(np.float64), y)


def adjoint_projected(ytil: np.ndarray, maps: np.ndarray) -> np.ndarray:
    """A^H y from projected data: S^H F^H ytil.  ytil [C][K][..] -> [M][K][..]."""
    return sense_adj(ifft2c(ytil), maps)


def apply_psi(kc: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """u_k(n) = sum_l Psi(n)_{kl} v_l(n) for k-space images kc [C][K][Ny][Nz]."""
    return np.einsum("yzkl,clyz->ckyz", psi, kc)


def normal(alpha: np.ndarray, maps: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """A^H A alpha = S^H F^H Psi F S alpha (Sec. IV.B)."""
    return sense_adj(ifft2c(apply_psi(fft2c(sense(alpha, maps)), psi)), maps)


def lipschitz(maps: np.ndarray, psi: np.ndarray) -> float:
    """Upper bound of ||A^H A||: max_n lambda_max Psi(n) * max_p lambda_max S(p)^H S(p)."""
    lam_psi = np.linalg.eigvalsh(psi).max()
    sp = np.moveaxis(maps, (0, 1), (-2, -1))  # [Ny][Nz][C][M]
    gram = np.conj(np.swapaxes(sp, -1, -2)) @ sp
    lam_s = np.linalg.eigvalsh(gram).max()
    return float(lam_psi * lam_s)


# ---------------------------------------------------------------------------------
# Locally low rank prox (Eq. 4, Sec. II.B and Sec. IV.C): singular-value soft threshold
# (Cai, Candes, Shen 2010) of non-overlapping b x b x K blocks of the randomly
# circular-shifted coefficient images.
# ---------------------------------------------------------------------------------
def svt(X: np.ndarray, tau: float) -> np.ndarray:
    """prox of tau ||.||_*: U max(Sigma - tau, 0) V^H.  X [..][B][K] (batched)."""
    U, s, Vh = np.linalg.svd(X, full_matrices=False)
    return (U * np.maximum(s - tau, 0.0)[..., None, :]) @ Vh


def _block_edges(n: int, b: int) -> list[tuple[int, int]]:
    return [(i, min(i + b, n)) for i in range(0, n, b)]


def llr_prox(alpha: np.ndarray, b: int, tau: float, sy: int, sz: int) -> np.ndarray:
    """LLR prox of alpha [M][K][Ny][Nz] for the shift (sy, sz).

    Following the description of the baseline (Sec. IV.C): circularly shift the
    coefficient images so that shifted row r is original row (r + sy) mod Ny, cut
    non-overlapping b x b blocks from the origin (the last one partial), reshape each
    into a (pixels x K) matrix per map set, soft-threshold its singular values, put
    it back and undo the shift."""
    M, K, Ny, Nz = alpha.shape
    shifted = np.roll(alpha, shift=(-sy, -sz), axis=(-2, -1))
    out = np.empty_like(shifted)
    for (y0, y1) in _block_edges(Ny, b):
        for (z0, z1) in _block_edges(Nz, b):
            blk = shifted[:, :, y0:y1, z0:z1]  # [M][K][by][bz]
            X = blk.reshape(M, K, -1).transpose(0, 2, 1)  # [M][pixels][K]
            Xt = svt(X, tau)
            out[:, :, y0:y1, z0:z1] = Xt.transpose(0, 2, 1).reshape(blk.shape)
    return np.roll(out, shift=(sy, sz), axis=(-2, -1))


def llr_norm(alpha: np.ndarray, b: int, sy: int, sz: int) -> float:
    """sum_n ||R_n alpha||_* for the blocks of shift (sy, sz) (Eq. 4 without lambda)."""
    M, K, Ny, Nz = alpha.shape
    shifted = np.roll(alpha, shift=(-sy, -sz), axis=(-2, -1))
    tot = 0.0
    for (y0, y1) in _block_edges(Ny, b):
        for (z0, z1) in _block_edges(Nz, b):
            X = shifted[:, :, y0:y1, z0:z1].reshape(M, K, -1).transpose(0, 2, 1)
            tot += float(np.linalg.svd(X, compute_uv=False).sum())
    return tot


# ---------------------------------------------------------------------------------
# FISTA (Beck and Teboulle 2009) on Eq. 5, as Sec. II.A and Sec. III.B describe it:
# gradient step on the data term, then the prox of the regulariser.
# ---------------------------------------------------------------------------------
def adjoint_data(kspace: np.ndarray, kform: str, maps: np.ndarray, mask: np.ndarray,
                 phi: np.ndarray) -> np.ndarray:
    """A^H y from T-form (``kform='te'``, [C][T][..]) or projected (``'proj'``, [C][K][..]) data."""
    if kform == "te":
        return adjoint(kspace, maps, mask, phi)
    if kform == "proj":
        return adjoint_projected(kspace, maps)
    raise ValueError(kform)


def data_term(kspace: np.ndarray, kform: str, maps: np.ndarray, mask: np.ndarray, phi: np.ndarray,
              alpha: np.ndarray) -> tuple[float, float]:
    """Data term of Eq. 5 at alpha, f = 1/2 ||P F S Phi alpha - y||^2 over the acquired
    samples, split as f = h + c with h = 1/2 <alpha, A^H A alpha> - Re <alpha, A^H y>
    (the part that depends on alpha) and c = 1/2 ||P y||^2.

    T-form data: f from its definition (the residual of the forward model), c from y,
    h = f - c.  Projected data do not determine c (NaN); h is then formed from A^H A alpha
    and A^H y (Sec. IV.B's normal operator and the projected adjoint)."""
    if kform == "te":
        y = mask[None].astype(float) * kspace
        f = 0.5 * float(np.sum(np.abs(forward(alpha, maps, mask, phi) - y) ** 2))
        c = 0.5 * float(np.sum(np.abs(y) ** 2))
        return f - c, c
    if kform == "proj":
        w = normal(alpha, maps, space_time_kernel(mask, phi))
        h = 0.5 * float(np.real(np.vdot(alpha, w))) - float(np.real(np.vdot(alpha, adjoint_projected(kspace, maps))))
        return h, float("nan")
    raise ValueError(kform)


def fista(kspace: np.ndarray, kform: str, maps: np.ndarray, mask: np.ndarray, phi: np.ndarray,
          lam: float, b: int, iters: int, seed: int, step: float | None = None,
          shifts: bool = True, x0: np.ndarray | None = None, return_trace: bool = False):
    """Solve Eq. 5 by ``iters`` FISTA iterations; returns alpha [M][K][Ny][Nz].

    Iteration k: g = z_k - mu (A^H A z_k - A^H y); x_{k+1} = LLR prox of g with
    threshold mu*lambda and the shift of iteration k; t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2;
    z_{k+1} = x_{k+1} + ((t_k - 1)/t_{k+1}) (x_{k+1} - x_k)."""
    C, M = maps.shape[:2]
    K = phi.shape[1]
    Ny, Nz = mask.shape[1:]
    psi = space_time_kernel(mask, phi)
    mu = (1.0 / lipschitz(maps, psi)) if step is None else float(step)
    aty = adjoint_data(kspace, kform, maps, mask, phi)
    x = np.zeros((M, K, Ny, Nz), np.complex128) if x0 is None else x0.astype(np.complex128)
    z = x.copy()
    t = 1.0
    sh = llr_shifts(seed, iters, b) if shifts else np.zeros((iters, 2), np.int64)
    trace = []
    for it in range(iters):
        g = z - mu * (normal(z, maps, psi) - aty)
        x_new = llr_prox(g, b, mu * lam, int(sh[it, 0]), int(sh[it, 1]))
        t_new = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = x_new + ((t - 1.0) / t_new) * (x_new - x)
        x, t = x_new, t_new
        if return_trace:
            trace.append(x.copy())
    if return_trace:
        return x, mu, trace
    return x


def cg(apply_op, rhs: np.ndarray, x0: np.ndarray, iters: int) -> np.ndarray:
    """Conjugate gradients (Hestenes and Stiefel) for the Hermitian positive definite
    system apply_op(x) = rhs, started at x0, exactly ``iters`` iterations:
      r = rhs - A x0, p = r;  a = <r, r> / <p, A p>;  x += a p;  r -= a A p;
      b = <r_new, r_new> / <r, r>;  p = r + b p.
    A zero denominator makes its quotient zero, so a solved system stays put."""
    x = x0.astype(np.complex128).copy()
    r = rhs - apply_op(x)
    p = r.copy()
    rr = float(np.vdot(r, r).real)
    for _ in range(iters):
        q = apply_op(p)
        pq = float(np.vdot(p, q).real)
        a = rr / pq if pq != 0.0 else 0.0
        x = x + a * p
        r = r - a * q
        rr_new = float(np.vdot(r, r).real)
        bb = rr_new / rr if rr != 0.0 else 0.0
        p = r + bb * p
        rr = rr_new
    return x


def admm(kspace: np.ndarray, kform: str, maps: np.ndarray, mask: np.ndarray, phi: np.ndarray,
         lam: float, b: int, iters: int, seed: int, rho: float, cg_iters: int,
         shifts: bool = True, return_all: bool = False):
    """Solve Eq. 5 by ``iters`` iterations of ADMM in scaled form with the splitting
    alpha = v (the LLR term on v), starting from alpha = v = u = 0:
      alpha_{k+1} = argmin 1/2 ||A alpha - y||^2 + rho/2 ||alpha - v_k + u_k||^2, i.e.
                    (A^H A + rho I) alpha = A^H y + rho (v_k - u_k), by ``cg_iters``
                    conjugate-gradient iterations started at alpha_k;
      v_{k+1}     = LLR prox of alpha_{k+1} + u_k with threshold lambda / rho and the
                    shift of iteration k (the same shift sequence as FISTA);
      u_{k+1}     = u_k + alpha_{k+1} - v_{k+1}.
    Returns v [M][K][Ny][Nz] (and alpha, u with return_all)."""
    C, M = maps.shape[:2]
    K = phi.shape[1]
    Ny, Nz = mask.shape[1:]
    psi = space_time_kernel(mask, phi)
    aty = adjoint_data(kspace, kform, maps, mask, phi)
    alpha = np.zeros((M, K, Ny, Nz), np.complex128)
    v = np.zeros_like(alpha)
    u = np.zeros_like(alpha)
    sh = llr_shifts(seed, iters, b) if shifts else np.zeros((iters, 2), np.int64)

    def op(x):
        return normal(x, maps, psi) + rho * x

    for it in range(iters):
        alpha = cg(op, aty + rho * (v - u), alpha, cg_iters)
        w = alpha + u
        v = llr_prox(w, b, lam / rho, int(sh[it, 0]), int(sh[it, 1]))
        u = w - v
    if return_all:
        return v, alpha, u
    return v


def synthesize_te(alpha: np.ndarray, maps: np.ndarray, phi: np.ndarray, te_index) -> np.ndarray:
    """Virtual-coil images at the listed echoes (Sec. III.C, Process TE): back-projection
    with the basis, x_m(t) = sum_k Phi[t, k] alpha[m, k], then the coil model
    x_c(t) = sum_m S_{c,m} x_m(t).  Returns [nte][C][Ny][Nz]."""
    xt = np.einsum("tk,mkyz->tmyz", phi[np.asarray(te_index)], alpha)
    return np.einsum("cmyz,tmyz->tcyz", maps, xt)


def homodyne_z(x: np.ndarray, pf: float) -> np.ndarray:
    """Homodyne detection (Noll 1991) along z, the slice direction, for partial Fourier
    fraction pf in (1/2, 1].  With the centred, unitary DFT along z (frequency d relative
    to DC at Nz/2), the acquired lines are d in [-w, Nz/2) with w = ceil(pf Nz) - Nz/2;
    the band |d| <= w is sampled on both sides.  Weighting H(d) = 0 (d < -w), 1 (|d| <= w),
    2 (d > w); phase from the band alone, phi = arg IFFT(k 1_band);
    result Re(IFFT(H k) e^(-i phi)) (real, any leading axes)."""
    Nz = x.shape[-1]
    c = Nz // 2
    w = int(np.ceil(pf * Nz)) - c
    d = np.arange(Nz) - c
    k = np.fft.fftshift(np.fft.fft(np.fft.ifftshift(x, axes=-1), axis=-1, norm="ortho"), axes=-1)
    H = np.where(d < -w, 0.0, np.where(d <= w, 1.0, 2.0))
    band = (np.abs(d) <= w).astype(float)

    def ifftc(kk):
        return np.fft.fftshift(np.fft.ifft(np.fft.ifftshift(kk, axes=-1), axis=-1, norm="ortho"), axes=-1)

    h = ifftc(H * k)
    lo = ifftc(band * k)
    mag = np.abs(lo)
    ph = np.where(mag > 0, np.conj(lo) / np.where(mag > 0, mag, 1.0), 1.0)
    return (h * ph).real


def postprocess(alpha: np.ndarray, maps: np.ndarray, phi: np.ndarray, te_index, pf: float) -> np.ndarray:
    """TE images of one slice (Sec. III.C and the Reconstruction paragraph of Sec. V): coil
    images at the listed echoes, homodyne along z per virtual coil, root sum of squares
    over coils.  Returns [nte][Ny][Nz] (real)."""
    xc = synthesize_te(alpha, maps, phi, te_index)
    hd = homodyne_z(xc, pf)
    return np.sqrt(np.sum(hd * hd, axis=1))


# ----------------------------------------------------------------------------------
# Wavelet denoising (Sec. II.C after Eq. 5, and Process TE of Sec. III.C): after the
# solve, the slices are re-joined into the volume and every basis-coefficient image gets
# one wavelet soft-threshold.  The paper names neither the wavelet nor the threshold;
# readings: the orthonormal Haar wavelet, a `levels`-level 3D pyramid (each level
# transforms the previous level's approximation block along x, y and z), complex soft
# thresholding of every detail coefficient with the threshold tau, the coarsest
# approximation kept.  Volume axes: x = readout (slice index), y, z.
# ----------------------------------------------------------------------------------
def _haar_axis(blk: np.ndarray, ax: int) -> np.ndarray:
    """One level of the orthonormal Haar analysis along axis ax: (a + b)/sqrt(2) of the
    pairs (2i, 2i + 1) in the first half, (a - b)/sqrt(2) in the second."""
    n = blk.shape[ax]
    a = np.take(blk, np.arange(0, n, 2), axis=ax)
    b = np.take(blk, np.arange(1, n, 2), axis=ax)
    return np.concatenate([(a + b) / np.sqrt(2.0), (a - b) / np.sqrt(2.0)], axis=ax)


def _ihaar_axis(blk: np.ndarray, ax: int) -> np.ndarray:
    n = blk.shape[ax]
    lo = np.take(blk, np.arange(0, n // 2), axis=ax)
    hi = np.take(blk, np.arange(n // 2, n), axis=ax)
    out = np.empty_like(blk)
    idx_e = [slice(None)] * blk.ndim
    idx_o = [slice(None)] * blk.ndim
    idx_e[ax] = slice(0, n, 2)
    idx_o[ax] = slice(1, n, 2)
    out[tuple(idx_e)] = (lo + hi) / np.sqrt(2.0)
    out[tuple(idx_o)] = (lo - hi) / np.sqrt(2.0)
    return out


def haar3(v: np.ndarray, levels: int) -> np.ndarray:
    """Forward 3D Haar pyramid of v [Nx][Ny][Nz] (every size a multiple of 2^levels), in
    the Mallat layout: level l replaces the block [:Nx/2^(l-1), :Ny/2^(l-1), :Nz/2^(l-1)]
    by its one-level transform (low halves first along every axis)."""
    c = np.asarray(v, np.complex128).copy()
    n = list(c.shape)
    for _ in range(levels):
        blk = c[:n[0], :n[1], :n[2]]
        for ax in range(3):
            blk = _haar_axis(blk, ax)
        c[:n[0], :n[1], :n[2]] = blk
        n = [m // 2 for m in n]
    return c


def ihaar3(c: np.ndarray, levels: int) -> np.ndarray:
    """Inverse of haar3."""
    v = np.asarray(c, np.complex128).copy()
    shape = v.shape
    for lev in range(levels - 1, -1, -1):
        n = [m >> lev for m in shape]
        blk = v[:n[0], :n[1], :n[2]]
        for ax in range(3):
            blk = _ihaar_axis(blk, ax)
        v[:n[0], :n[1], :n[2]] = blk
    return v


def soft_threshold(c: np.ndarray, tau: float) -> np.ndarray:
    """Complex soft threshold: c max(1 - tau/|c|, 0) (0 where c = 0)."""
    mag = np.abs(c)
    return c * np.where(mag > tau, 1.0 - tau / np.where(mag > 0, mag, 1.0), 0.0)


def wavelet_denoise(alpha: np.ndarray, tau: float, levels: int) -> np.ndarray:
    """Wavelet soft-threshold of the re-joined coefficient volume alpha [Nx][M][K][Ny][Nz]
    (Nx readout slices): for every (m, k) image, haar3 -> soft-threshold every coefficient
    outside the coarsest approximation block -> ihaar3."""
    alpha = np.asarray(alpha, np.complex128)
    Nx, M, K, Ny, Nz = alpha.shape
    f = 1 << levels
    if Nx % f or Ny % f or Nz % f:
        raise ValueError("every volume size must be a multiple of 2^levels")
    out = np.empty_like(alpha)
    for m in range(M):
        for k in range(K):
            c = haar3(alpha[:, m, k], levels)
            keep = c[:Nx // f, :Ny // f, :Nz // f].copy()
            c = soft_threshold(c, tau)
            c[:Nx // f, :Ny // f, :Nz // f] = keep
            out[:, m, k] = ihaar3(c, levels)
    return out


# ----------------------------------------------------------------------------------
# Pre-processing (Sec. III.A): the acquisition is a sparse array of fully sampled
# readout lines, line j holding the channels [Ctot][Nx] of phase encode (ky_j, kz_j) at
# echo t_j.  Index conventions: DC of every axis at index N/2.
# ----------------------------------------------------------------------------------
def calibration_average(lines: np.ndarray, ky, kz, ny: int, nz: int, win: int) -> np.ndarray:
    """Re-sort and average: the central win x win x win k-space window of every channel,
    each (ky, kz) averaged over the lines (echoes) that sampled it, unsampled points zero.
    lines [n][Ctot][Nx]; returns [Ctot][win][win][win] (axes kx, ky, kz)."""
    n, ctot, nx = lines.shape
    cal = np.zeros((ctot, win, win, win), np.complex128)
    cnt = np.zeros((win, win))
    x0, y0, z0 = nx // 2 - win // 2, ny // 2 - win // 2, nz // 2 - win // 2
    for j in range(n):
        a, b = int(ky[j]) - y0, int(kz[j]) - z0
        if 0 <= a < win and 0 <= b < win:
            cal[:, :, a, b] += lines[j, :, x0:x0 + win]
            cnt[a, b] += 1
    return cal / np.where(cnt > 0, cnt, 1.0)[None, None]


def compression_matrix(cal: np.ndarray, ncomp: int) -> np.ndarray:
    """SVD coil compression (Zhang et al. 2013): with the calibration points as rows of
    X [points][Ctot], the virtual channels are X W[:, :ncomp], W the right singular
    vectors (eigenvectors of X^H X) by decreasing singular value.  Each column is fixed
    to a canonical phase: its entry of largest magnitude (first such index) is real
    positive.  Returns W [Ctot][ncomp]."""
    ctot = cal.shape[0]
    X = cal.reshape(ctot, -1).T
    G = X.conj().T @ X
    ev, V = np.linalg.eigh(G)
    V = V[:, np.argsort(-ev)[:ncomp]]
    for c in range(ncomp):
        i = int(np.argmax(np.abs(V[:, c])))
        V[:, c] *= np.conj(V[i, c]) / np.abs(V[i, c])
    return V


def preprocess(lines: np.ndarray, t_idx, ky, kz, W: np.ndarray, phi: np.ndarray, ny: int, nz: int):
    """Coil-compress every line (y_v = y W), decouple the readout slices by the centred
    unitary 1D inverse DFT along x, and re-sort and project onto the basis:
    ytil[x][c][k][ky][kz] = sum over lines j at (ky, kz) of Phi[t_j][k] yhat_j[c][x].
    Also the sampling masks mask[t][ky][kz].  Returns (ytil [Nx][C][K][Ny][Nz], mask)."""
    n, ctot, nx = lines.shape
    T, K = phi.shape
    C = W.shape[1]
    yv = np.einsum("jcx,cd->jdx", lines, W)
    yh = np.fft.fftshift(np.fft.ifft(np.fft.ifftshift(yv, axes=-1), axis=-1, norm="ortho"), axes=-1)
    ytil = np.zeros((nx, C, K, ny, nz), np.complex128)
    mask = np.zeros((T, ny, nz), np.uint8)
    for j in range(n):
        ytil[:, :, :, ky[j], kz[j]] += np.einsum("k,cx->xck", phi[t_idx[j]], yh[j])
        mask[t_idx[j], ky[j], kz[j]] = 1
    return ytil, mask


def objective(alpha: np.ndarray, y: np.ndarray, maps: np.ndarray, mask: np.ndarray,
              phi: np.ndarray, lam: float, b: int, sy: int = 0, sz: int = 0) -> float:
    """Eq. 5 cost for T-form data y with the block grid of shift (sy, sz)."""
    r = y - forward(alpha, maps, mask, phi)
    return 0.5 * float(np.vdot(r, r).real) + lam * llr_norm(alpha, b, sy, sz)


def nrmse(x: np.ndarray, ref: np.ndarray) -> float:
    """||x - ref||_2 / ||ref||_2 over all values."""
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))
