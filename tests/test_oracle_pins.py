"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each compares the oracle with an
independent route (a definition built as a dense matrix, a closed form, a published
test vector, an optimality condition, a second solver written here).
"""
import os

import numpy as np
import pytest

import oracle as O
import t2sh_synth as synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------------
# helpers built from definitions, independent of the oracle's numpy.fft route
# ----------------------------------------------------------------------------------
def centred_dft_matrix(n):
    """D[k, j] = exp(-2 pi i (k - n/2)(j - n/2) / n) / sqrt(n): the centred unitary DFT
    written from its definition (image and k-space origins at index n/2)."""
    k = np.arange(n)[:, None] - n // 2
    j = np.arange(n)[None, :] - n // 2
    return np.exp(-2j * np.pi * k * j / n) / np.sqrt(n)


def dense_A(maps, mask, phi):
    """Dense matrix of A = P F S Phi (Eq. 5) on vec(alpha[M][K][Ny][Nz]) ->
    vec(y[C][T][Ny][Nz]), assembled from Kronecker products of the definitions."""
    C, M, Ny, Nz = maps.shape
    T, K = phi.shape
    N = Ny * Nz
    F = np.kron(centred_dft_matrix(Ny), centred_dft_matrix(Nz))  # acts on vec(img[Ny][Nz])
    A = np.zeros((C * T * N, M * K * N), np.complex128)
    for c in range(C):
        for t in range(T):
            P = np.diag(mask[t].ravel().astype(float))
            for m in range(M):
                S = np.diag(maps[c, m].ravel())
                blk = P @ F @ S
                for k in range(K):
                    r0 = (c * T + t) * N
                    c0 = (m * K + k) * N
                    A[r0:r0 + N, c0:c0 + N] += phi[t, k] * blk
    return A


def tiny_problem(seed, Ny=8, Nz=8, C=2, T=6, K=2, M=1, frac=0.5):
    rng = np.random.default_rng(seed)
    phi = synth.t2_basis(T, K)
    maps = synth.coil_maps(C, Ny, Nz, rng, M=M)
    mask = (rng.random((T, Ny, Nz)) < frac).astype(np.uint8)
    return phi, maps, mask, rng


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ----------------------------------------------------------------------------------
# shift generator
# ----------------------------------------------------------------------------------
def test_splitmix64_published_vectors():
    n_checked = 0
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(v) for v in line.split()]
            seed, n, ref = w[0], w[1], w[2:]
            assert O.splitmix64(seed, n) == ref
            n_checked += 1
    assert n_checked >= 2


def test_llr_shifts_range_and_split():
    sh = O.llr_shifts(1809, 4000, 8)
    assert sh.shape == (4000, 2) and sh.dtype == np.int64
    assert sh.min() == 0 and sh.max() == 7
    # both axes take every value, and they are not the same sequence
    assert set(sh[:, 0]) == set(range(8)) and set(sh[:, 1]) == set(range(8))
    assert np.mean(sh[:, 0] == sh[:, 1]) < 0.3
    h = O.splitmix64(1809, 3)
    assert sh[2, 0] == (h[2] & 0xFFFFFFFF) % 8 and sh[2, 1] == (h[2] >> 32) % 8


# ----------------------------------------------------------------------------------
# F: centred unitary DFT
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("ny,nz", [(8, 12), (12, 8), (48, 64), (64, 48), (160, 8), (6, 10)])
def test_fft2c_matches_definition(ny, nz):
    rng = np.random.default_rng(ny * 1000 + nz)
    x = crandn(rng, 3, ny, nz)
    ref = np.einsum("ab,sbc,dc->sad", centred_dft_matrix(ny), x, centred_dft_matrix(nz))
    got = O.fft2c(x)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max() * 10
    # unitary and inverse
    assert np.allclose(np.linalg.norm(got), np.linalg.norm(x), rtol=1e-13)
    assert np.abs(O.ifft2c(got) - x).max() < 1e-12


def test_fft2c_centred_delta_and_constant():
    ny, nz = 16, 12
    d = np.zeros((ny, nz), complex)
    d[ny // 2, nz // 2] = 1.0
    assert np.allclose(O.fft2c(d), np.full((ny, nz), 1 / np.sqrt(ny * nz)), atol=1e-15)
    k = O.fft2c(np.ones((ny, nz), complex))
    ref = np.zeros((ny, nz))
    ref[ny // 2, nz // 2] = np.sqrt(ny * nz)
    assert np.allclose(k, ref, atol=1e-12)


# ----------------------------------------------------------------------------------
# forward model, adjoint, space-time kernel
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("M", [1, 2])
def test_forward_and_normal_match_dense_matrix(M):
    phi, maps, mask, rng = tiny_problem(11 + M, M=M)
    A = dense_A(maps, mask, phi)
    alpha = crandn(rng, M, 2, 8, 8)
    y = O.forward(alpha, maps, mask, phi)
    assert np.abs(y.ravel() - A @ alpha.ravel()).max() < 1e-12
    yy = crandn(rng, 2, 6, 8, 8) * mask[None]
    assert np.abs(O.adjoint(yy, maps, mask, phi).ravel() - A.conj().T @ yy.ravel()).max() < 1e-12
    psi = O.space_time_kernel(mask, phi)
    nrm = O.normal(alpha, maps, psi)
    assert np.abs(nrm.ravel() - A.conj().T @ (A @ alpha.ravel())).max() < 1e-12


@pytest.mark.parametrize("M", [1, 2])
def test_data_term_matches_dense_least_squares(M):
    """The data term of Eq. 5 against 1/2 ||A alpha - P y||^2 with the Kronecker-built A,
    the split f = h + c, projected data (same h, c undetermined), f(alpha_true) = 0 on
    noiseless data and h(0) = 0."""
    phi, maps, mask, rng = tiny_problem(31 + M, M=M)
    A = dense_A(maps, mask, phi)
    alpha = crandn(rng, M, 2, 8, 8)
    y = crandn(rng, 2, 6, 8, 8)
    py = y * mask[None]
    f_dense = 0.5 * np.sum(np.abs(A @ alpha.ravel() - py.ravel()) ** 2)
    h, c = O.data_term(y, "te", maps, mask, phi, alpha)
    assert abs(h + c - f_dense) < 1e-10 * f_dense
    assert abs(c - 0.5 * np.sum(np.abs(py) ** 2)) < 1e-10 * c
    # projected data: the same alpha-dependent part, from the expanded form
    hp, cp = O.data_term(O.project(y, mask, phi), "proj", maps, mask, phi, alpha)
    assert abs(hp - h) < 1e-10 * abs(h) and np.isnan(cp)
    # noiseless data: the data term vanishes at the true coefficients
    y0 = A @ alpha.ravel()
    h0, c0 = O.data_term(y0.reshape(2, 6, 8, 8), "te", maps, mask, phi, alpha)
    assert abs(h0 + c0) < 1e-10 * c0
    assert O.data_term(y, "te", maps, mask, phi, np.zeros_like(alpha))[0] == 0.0


def test_adjoint_identity_knee_like():
    rng = np.random.default_rng(5)
    T, K, C, M, ny, nz = 20, 4, 4, 2, 32, 24
    phi = synth.t2_basis(T, K)
    maps = synth.coil_maps(C, ny, nz, rng, M=M)
    mask = synth.vd_masks(T, ny, nz, 0.2, rng)
    x = crandn(rng, M, K, ny, nz)
    y = crandn(rng, C, T, ny, nz)
    lhs = np.vdot(y, O.forward(x, maps, mask, phi))
    rhs = np.vdot(O.adjoint(y, maps, mask, phi), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_psi_is_identity_under_full_sampling():
    phi = synth.t2_basis(40, 4)
    assert np.allclose(phi.T @ phi, np.eye(4), atol=1e-13)
    psi = O.space_time_kernel(np.ones((40, 6, 4), np.uint8), phi)
    assert np.abs(psi - np.eye(4)[None, None]).max() < 1e-13


def test_psi_real_symmetric_bounded():
    rng = np.random.default_rng(3)
    phi = synth.t2_basis(32, 4)
    mask = synth.vd_masks(32, 16, 12, 0.1, rng)
    psi = O.space_time_kernel(mask, phi)
    assert psi.dtype == np.float64
    assert np.abs(psi - np.swapaxes(psi, -1, -2)).max() == 0.0
    ev = np.linalg.eigvalsh(psi)
    assert ev.min() > -1e-13 and ev.max() < 1 + 1e-13
    # a point no echo samples has Psi = 0; a point only echo t samples has phi_t phi_t^T
    m = np.zeros((32, 2, 2), np.uint8)
    m[5, 0, 1] = 1
    p = O.space_time_kernel(m, phi)
    assert np.all(p[1, :] == 0) and np.all(p[0, 0] == 0)
    assert np.allclose(p[0, 1], np.outer(phi[5], phi[5]), atol=0)


@pytest.mark.parametrize("M", [1, 2])
def test_commutation_psi_path_equals_echo_path(M):
    """Sec. IV.B: S^H F^H Psi F S == A^H A computed through every echo."""
    rng = np.random.default_rng(21 + M)
    T, K, C, ny, nz = 24, 4, 3, 16, 12
    phi = synth.t2_basis(T, K)
    maps = synth.coil_maps(C, ny, nz, rng, M=M)
    mask = synth.vd_masks(T, ny, nz, 0.15, rng)
    a = crandn(rng, M, K, ny, nz)
    psi = O.space_time_kernel(mask, phi)
    ref = O.normal_explicit(a, maps, mask, phi)
    assert np.abs(O.normal(a, maps, psi) - ref).max() <= 1e-12 * np.abs(ref).max()
    # the same commutation for the data side: A^H y == S^H F^H (Phi^T P y)
    y = crandn(rng, C, T, ny, nz)
    r1 = O.adjoint(y, maps, mask, phi)
    r2 = O.adjoint_projected(O.project(y, mask, phi), maps)
    assert np.abs(r1 - r2).max() <= 1e-12 * np.abs(r1).max()


def test_lipschitz_bounds_normal_operator():
    for M in (1, 2):
        phi, maps, mask, rng = tiny_problem(40 + M, M=M)
        A = dense_A(maps, mask, phi)
        lmax = np.linalg.eigvalsh(A.conj().T @ A).max()
        L = O.lipschitz(maps, O.space_time_kernel(mask, phi))
        assert lmax <= L * (1 + 1e-12)
    # full sampling, maps normalised: L = ||A^H A|| = 1
    phi, maps, _, _ = tiny_problem(50)
    full = np.ones((6, 8, 8), np.uint8)
    A = dense_A(maps, full, phi)
    L = O.lipschitz(maps, O.space_time_kernel(full, phi))
    assert abs(L - 1.0) < 1e-12
    assert abs(np.linalg.eigvalsh(A.conj().T @ A).max() - 1.0) < 1e-12


# ----------------------------------------------------------------------------------
# singular value soft threshold and the LLR block grid
# ----------------------------------------------------------------------------------
def test_svt_closed_forms():
    rng = np.random.default_rng(7)
    X = crandn(rng, 64, 4)
    s = np.linalg.svd(X, compute_uv=False)
    assert np.abs(O.svt(X, 0.0) - X).max() < 1e-12
    assert np.abs(O.svt(X, s[0] * 1.0001)).max() == 0.0
    # rank one: sigma u v^H -> (sigma - tau)+ u v^H
    u = crandn(rng, 64); u /= np.linalg.norm(u)
    v = crandn(rng, 4); v /= np.linalg.norm(v)
    R1 = 3.0 * np.outer(u, v.conj())
    assert np.abs(O.svt(R1, 1.0) - 2.0 * np.outer(u, v.conj())).max() < 1e-12
    # orthogonal columns with norms d: the thresholds act column by column
    Q, _ = np.linalg.qr(crandn(rng, 64, 4))
    d = np.array([5.0, 2.0, 0.7, 0.1])
    out = O.svt(Q * d, 0.5)
    assert np.abs(out - Q * np.maximum(d - 0.5, 0)).max() < 1e-12
    # degenerate singular values: result independent of the basis chosen inside
    Xd = Q * np.array([2.0, 2.0, 2.0, 1.0])
    assert np.abs(O.svt(Xd, 0.5) - Q * np.array([1.5, 1.5, 1.5, 0.5])).max() < 1e-12


def test_svt_is_the_nuclear_norm_prox():
    """Optimality: the prox minimises 1/2||Z - X||^2 + tau ||Z||_*; random
    perturbations never lower that cost."""
    rng = np.random.default_rng(8)
    X = crandn(rng, 16, 4)
    tau = 1.3
    Z = O.svt(X, tau)

    def cost(W):
        return 0.5 * np.linalg.norm(W - X) ** 2 + tau * np.linalg.svd(W, compute_uv=False).sum()

    c0 = cost(Z)
    for _ in range(200):
        d = crandn(rng, 16, 4) * 10 ** rng.uniform(-4, -1)
        assert cost(Z + d) >= c0 - 1e-12


def _block_pixels(Ny, Nz, b, sy, sz, i, j):
    """Pixels of block (i, j) for shift (sy, sz), straight from the grid definition."""
    rows = [(sy + i * b + r) % Ny for r in range(b) if i * b + r < Ny]
    cols = [(sz + j * b + c) % Nz for c in range(b) if j * b + c < Nz]
    return rows, cols


@pytest.mark.parametrize("Ny,Nz,b,sy,sz", [(16, 16, 8, 3, 5), (20, 12, 8, 7, 1), (12, 20, 6, 0, 5), (13, 9, 4, 2, 3)])
def test_llr_prox_acts_on_the_shifted_blocks(Ny, Nz, b, sy, sz):
    rng = np.random.default_rng(Ny + Nz + b)
    K, M = 4, 1
    nby, nbz = -(-Ny // b), -(-Nz // b)
    for (i, j) in [(0, 0), (nby - 1, nbz - 1), (nby // 2, 0)]:
        rows, cols = _block_pixels(Ny, Nz, b, sy, sz, i, j)
        alpha = np.zeros((M, K, Ny, Nz), complex)
        u = crandn(rng, len(rows), len(cols))
        u /= np.linalg.norm(u)
        v = crandn(rng, K)
        v /= np.linalg.norm(v)
        for a, r in enumerate(rows):
            for c_, cc in enumerate(cols):
                alpha[0, :, r, cc] = 4.0 * u[a, c_] * v  # rank-1 block, sigma = 4
        out = O.llr_prox(alpha, b, 1.5, sy, sz)
        assert np.abs(out - alpha * (2.5 / 4.0)).max() < 1e-12
    # tau = 0 is the identity; a large tau clears everything
    a = crandn(rng, M, K, Ny, Nz)
    assert np.abs(O.llr_prox(a, b, 0.0, sy, sz) - a).max() < 1e-12
    assert np.abs(O.llr_prox(a, b, 1e6, sy, sz)).max() == 0.0


def test_llr_prox_is_block_separable_and_per_map():
    rng = np.random.default_rng(99)
    M, K, Ny, Nz, b, sy, sz = 2, 4, 16, 16, 8, 6, 2
    a = crandn(rng, M, K, Ny, Nz)
    out = O.llr_prox(a, b, 2.0, sy, sz)
    rows, cols = _block_pixels(Ny, Nz, b, sy, sz, 1, 0)
    a2 = a.copy()
    # change a pixel outside block (1, 0) and map set 1 inside it
    orow = [r for r in range(Ny) if r not in rows][0]
    a2[0, :, orow, cols[0]] += 5.0
    a2[1, :, rows[0], cols[0]] += 5.0
    out2 = O.llr_prox(a2, b, 2.0, sy, sz)
    idx = np.ix_(rows, cols)
    assert np.abs(out2[0][:, idx[0], idx[1]] - out[0][:, idx[0], idx[1]]).max() < 1e-12
    # each map set's block is the SVT of its own (pixels x K) matrix
    X = a[1][:, idx[0], idx[1]].reshape(K, -1).T
    ref = O.svt(X, 2.0).T.reshape(K, len(rows), len(cols))
    assert np.abs(out[1][:, idx[0], idx[1]] - ref).max() < 1e-12


# ----------------------------------------------------------------------------------
# FISTA
# ----------------------------------------------------------------------------------
def test_exact_recovery_full_sampling():
    """Noiseless, fully sampled, lambda = 0, sum_c |S_c|^2 = 1: x_1 = alpha_true (mu = 1)."""
    rng = np.random.default_rng(1)
    T, K, C, ny, nz = 16, 4, 4, 16, 12
    phi = synth.t2_basis(T, K)
    maps = synth.coil_maps(C, ny, nz, rng)
    full = np.ones((T, ny, nz), np.uint8)
    a_true = crandn(rng, 1, K, ny, nz)
    y = O.forward(a_true, maps, full, phi)
    x, mu, trace = O.fista(y, "te", maps, full, phi, lam=0.0, b=4, iters=5, seed=3, return_trace=True)
    assert abs(mu - 1.0) < 1e-12
    for xi in trace:
        assert np.abs(xi - a_true).max() < 1e-12
    # a phantom outside the subspace gives its projection Phi^T x
    xt = crandn(rng, 1, T, ny, nz)
    y2 = O.sense_forward(xt, maps, full)
    x2 = O.fista(y2, "te", maps, full, phi, lam=0.0, b=4, iters=2, seed=3)
    assert np.abs(x2 - np.einsum("tk,mtyz->mkyz", phi, xt)).max() < 1e-12


def test_fista_lambda0_converges_to_least_squares():
    phi, maps, mask, rng = tiny_problem(77, frac=0.7)
    A = dense_A(maps, mask, phi)
    assert np.linalg.matrix_rank(A) == A.shape[1]
    a_true = crandn(rng, 1, 2, 8, 8)
    y = (A @ a_true.ravel()).reshape(2, 6, 8, 8) + 0.05 * crandn(rng, 2, 6, 8, 8) * mask[None]
    ls = np.linalg.lstsq(A, y.ravel(), rcond=None)[0]
    x = O.fista(y, "te", maps, mask, phi, lam=0.0, b=4, iters=3000, seed=0)
    assert np.abs(x.ravel() - ls).max() < 1e-8


def test_fista_no_shift_reaches_the_convex_minimiser():
    """Shifts off: Eq. 5 is convex with one fixed block grid.  A proximal-gradient
    (ISTA) run written here on the dense matrix, with an SVT built from numpy's SVD per
    block, reaches the same minimiser and cost."""
    phi, maps, mask, rng = tiny_problem(78, frac=0.7)
    A = dense_A(maps, mask, phi)
    a_true = crandn(rng, 1, 2, 8, 8)
    y = (A @ a_true.ravel()).reshape(2, 6, 8, 8) + 0.1 * crandn(rng, 2, 6, 8, 8) * mask[None]
    lam, b = 0.3, 4
    x = O.fista(y, "te", maps, mask, phi, lam=lam, b=b, iters=2000, seed=0, shifts=False)

    L = np.linalg.eigvalsh(A.conj().T @ A).max()
    AhA = A.conj().T @ A
    Ahy = A.conj().T @ y.ravel()
    w = np.zeros(A.shape[1], complex)
    for _ in range(6000):
        g = (w - (AhA @ w - Ahy) / L).reshape(2, 8, 8)
        for y0 in range(0, 8, b):
            for z0 in range(0, 8, b):
                X = g[:, y0:y0 + b, z0:z0 + b].reshape(2, -1).T
                U, s, Vh = np.linalg.svd(X, full_matrices=False)
                g[:, y0:y0 + b, z0:z0 + b] = ((U * np.maximum(s - lam / L, 0)) @ Vh).T.reshape(2, b, b)
        w = g.ravel()
    f_ista = O.objective(w.reshape(1, 2, 8, 8), y, maps, mask, phi, lam, b)
    f_fista = O.objective(x, y, maps, mask, phi, lam, b)
    assert abs(f_fista - f_ista) <= 1e-9 * abs(f_ista)
    assert np.abs(x.ravel() - w).max() < 1e-6
    # fixed point of the prox-gradient map
    mu = 1.0 / O.lipschitz(maps, O.space_time_kernel(mask, phi))
    g = x - mu * (O.normal(x, maps, O.space_time_kernel(mask, phi)) - O.adjoint(y, maps, mask, phi))
    assert np.abs(O.llr_prox(g, b, mu * lam, 0, 0) - x).max() < 1e-8


def test_fista_momentum_sequence():
    """t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 with t_0 = 1: check the second iterate on a
    problem where the gradient step is the identity map onto a_true (full sampling,
    lambda = 0), so z_1 = x_1 and x_2 = x_1: momentum only scales a zero difference."""
    rng = np.random.default_rng(2)
    phi = synth.t2_basis(8, 2)
    maps = synth.coil_maps(2, 8, 8, rng)
    mask = np.ones((8, 8, 8), np.uint8)
    mask[:, ::2, 1::3] = 0  # partial sampling: gradient step is not exact any more
    a_true = crandn(rng, 1, 2, 8, 8)
    y = O.forward(a_true, maps, mask, phi)
    x, mu, tr = O.fista(y, "te", maps, mask, phi, lam=0.0, b=4, iters=3, seed=0, step=1.0, return_trace=True)
    psi = O.space_time_kernel(mask, phi)
    aty = O.adjoint(y, maps, mask, phi)
    x1 = aty  # from x0 = z0 = 0
    t1 = (1 + np.sqrt(5)) / 2
    z1 = x1 + ((1 - 1) / t1) * x1
    x2 = z1 - (O.normal(z1, maps, psi) - aty)
    t2 = (1 + np.sqrt(1 + 4 * t1 * t1)) / 2
    z2 = x2 + ((t1 - 1) / t2) * (x2 - x1)
    x3 = z2 - (O.normal(z2, maps, psi) - aty)
    assert np.abs(tr[0] - x1).max() < 1e-13
    assert np.abs(tr[1] - x2).max() < 1e-13
    assert np.abs(tr[2] - x3).max() < 1e-13


def test_fista_rate_bound_beck_teboulle():
    """Beck & Teboulle (2009, Thm 4.4): F(x_k) - F* <= 2 L ||x_0 - x*||^2 / (k + 1)^2.
    Checked at lambda = 0 (F* from least squares) on an ill-conditioned tiny problem."""
    phi, maps, mask, rng = tiny_problem(80, frac=0.45)
    A = dense_A(maps, mask, phi)
    y = crandn(rng, 2, 6, 8, 8) * mask[None]
    ls = np.linalg.lstsq(A, y.ravel(), rcond=None)[0]
    fstar = 0.5 * np.linalg.norm(A @ ls - y.ravel()) ** 2
    L = O.lipschitz(maps, O.space_time_kernel(mask, phi))
    _, mu, tr = O.fista(y, "te", maps, mask, phi, lam=0.0, b=4, iters=200, seed=0, return_trace=True)
    R2 = np.linalg.norm(ls) ** 2
    for k in (1, 5, 20, 50, 100, 200):
        fk = 0.5 * np.linalg.norm(A @ tr[k - 1].ravel() - y.ravel()) ** 2
        assert fk - fstar <= 2 * L * R2 / (k + 1) ** 2 + 1e-12


# ----------------------------------------------------------------------------------
# ADMM with conjugate-gradient inner solves
# ----------------------------------------------------------------------------------
def test_cg_solves_a_dense_hpd_system_in_n_steps():
    """n CG iterations solve an n x n Hermitian positive definite system (exact
    arithmetic; float64 to 1e-9), against numpy's dense solver."""
    rng = np.random.default_rng(5)
    n = 12
    B = crandn(rng, n, n)
    H = B.conj().T @ B + 0.5 * np.eye(n)
    rhs = crandn(rng, n)
    x = O.cg(lambda v: H @ v, rhs, np.zeros(n, complex), n)
    assert np.abs(x - np.linalg.solve(H, rhs)).max() < 1e-9 * np.abs(np.linalg.solve(H, rhs)).max()
    # a solved system stays put (zero residual: zero step, zero direction)
    x2 = O.cg(lambda v: H @ v, rhs, np.linalg.solve(H, rhs), 3)
    assert np.abs(x2 - np.linalg.solve(H, rhs)).max() < 1e-12


def test_cg_on_the_regularised_normal_equations_matches_dense_solve():
    """The ADMM alpha-update (A^H A + rho I) alpha = rhs through the oracle's normal
    operator equals the dense solve with the Kronecker-built A."""
    phi, maps, mask, rng = tiny_problem(79, frac=0.4)
    A = dense_A(maps, mask, phi)
    psi = O.space_time_kernel(mask, phi)
    rho = 0.3
    rhs = crandn(rng, 1, 2, 8, 8)
    H = A.conj().T @ A + rho * np.eye(A.shape[1])
    ref = np.linalg.solve(H, rhs.ravel())
    x = O.cg(lambda v: O.normal(v, maps, psi) + rho * v, rhs, np.zeros_like(rhs), 200)
    assert np.abs(x.ravel() - ref).max() < 1e-9 * np.abs(ref).max()


def test_admm_lambda0_recovers_noiseless_full_sampling():
    """lambda = 0: the prox is the identity, u stays 0 and the alpha-update is a proximal
    point step towards the least-squares solution, here the noiseless phantom."""
    rng = np.random.default_rng(2)
    T, K, C, ny, nz = 12, 3, 3, 12, 8
    phi = synth.t2_basis(T, K)
    maps = synth.coil_maps(C, ny, nz, rng)
    full = np.ones((T, ny, nz), np.uint8)
    a_true = crandn(rng, 1, K, ny, nz)
    y = O.forward(a_true, maps, full, phi)
    v, alpha, u = O.admm(y, "te", maps, full, phi, lam=0.0, b=4, iters=40, seed=1, rho=0.5, cg_iters=3,
                         return_all=True)
    assert np.abs(u).max() < 1e-12
    assert np.abs(v - a_true).max() < 1e-9 * np.abs(a_true).max()


def test_admm_and_fista_reach_the_same_convex_minimiser():
    """Shifts off: ADMM (exact enough inner solves) and FISTA minimise the same convex
    Eq. 5 cost; both reach one minimiser and cost, and the ADMM fixed point satisfies
    v = prox(v - (A^H A v - A^H y) / rho) with threshold lambda / rho, the optimality
    condition of the cost (u = (A^H y - A^H A v) / rho at the fixed point)."""
    phi, maps, mask, rng = tiny_problem(80, frac=0.7)
    A = dense_A(maps, mask, phi)
    a_true = crandn(rng, 1, 2, 8, 8)
    y = (A @ a_true.ravel()).reshape(2, 6, 8, 8) + 0.1 * crandn(rng, 2, 6, 8, 8) * mask[None]
    lam, b, rho = 0.3, 4, 0.5
    x_f = O.fista(y, "te", maps, mask, phi, lam=lam, b=b, iters=3000, seed=0, shifts=False)
    v, alpha, u = O.admm(y, "te", maps, mask, phi, lam=lam, b=b, iters=600, seed=0, rho=rho, cg_iters=12,
                         shifts=False, return_all=True)
    f_f = O.objective(x_f, y, maps, mask, phi, lam, b)
    f_a = O.objective(v, y, maps, mask, phi, lam, b)
    assert abs(f_a - f_f) <= 1e-8 * abs(f_f)
    assert np.abs(v - x_f).max() < 1e-6
    assert np.abs(alpha - v).max() < 1e-8  # primal residual
    psi = O.space_time_kernel(mask, phi)
    aty = O.adjoint(y, maps, mask, phi)
    assert np.abs(u - (aty - O.normal(v, maps, psi)) / rho).max() < 1e-7
    g = v - (O.normal(v, maps, psi) - aty) / rho
    assert np.abs(O.llr_prox(g, b, lam / rho, 0, 0) - v).max() < 1e-7


# ----------------------------------------------------------------------------------
# post-processing: TE synthesis, homodyne along z, root sum of squares
# ----------------------------------------------------------------------------------
def _real_positive_lines(rng, shape, nz, amp=0.3):
    """Real lines 1 + amp * (random real band-limited signal without the Nyquist line):
    positive enough that their low-pass stays positive."""
    spec = crandn(rng, *shape, nz)
    spec[..., nz // 2] = 0.0  # Nyquist line
    x = np.fft.ifft(spec, axis=-1).real
    x = x / np.abs(x).max()
    return 1.0 + amp * x


@pytest.mark.parametrize("nz,pf", [(48, 0.65), (40, 0.75), (64, 0.5625), (30, 0.7)])
def test_homodyne_recovers_a_real_image_exactly(nz, pf):
    """Real image without Nyquist content: the unpaired side weighted by 2 stands in for its
    conjugate partners, so Re(IFFT(H k)) = x; its low-pass is positive, so the phase is 0."""
    rng = np.random.default_rng(int(nz * 100 * pf))
    x = _real_positive_lines(rng, (5,), nz)
    # the Nyquist line of the centred transform is the index-0 line of the plain one
    # after the half-length shift: check it is (numerically) empty
    assert np.abs(np.fft.fft(np.fft.ifftshift(x, axes=-1), axis=-1)[..., nz // 2]).max() < 1e-9
    out = O.homodyne_z(x.astype(complex), pf)
    assert np.abs(out - x).max() < 1e-12
    # a global phase is removed by the phase estimate
    out2 = O.homodyne_z(x * np.exp(1j * 0.7), pf)
    assert np.abs(out2 - x).max() < 1e-12


def test_homodyne_full_fraction_is_the_magnitude():
    rng = np.random.default_rng(9)
    x = crandn(rng, 3, 8, 20)
    assert np.abs(O.homodyne_z(x, 1.0) - np.abs(x)).max() < 1e-12


def test_postprocess_full_fraction_is_rss_of_the_te_image():
    """pf = 1 and sum_c |S_c|^2 = 1 per map set (M = 1): the RSS of the coil images is the
    magnitude of the back-projected TE image."""
    rng = np.random.default_rng(10)
    T, K, C, ny, nz = 16, 4, 5, 12, 10
    phi = synth.t2_basis(T, K)
    maps = synth.coil_maps(C, ny, nz, rng)
    alpha = crandn(rng, 1, K, ny, nz)
    te = [2, 7, 15]
    img = O.postprocess(alpha, maps, phi, te, 1.0)
    xt = np.einsum("tk,kyz->tyz", phi[te], alpha[0])
    assert np.abs(img - np.abs(xt)).max() < 1e-12


def test_backprojection_reproduces_an_in_subspace_decay():
    """x_t in the span of Phi (here Phi c): Phi Phi^T x_t = x_t, so the TE synthesis of
    alpha = Phi^T x_t returns the decay itself (single coil, unit map)."""
    rng = np.random.default_rng(11)
    T, K, ny, nz = 20, 4, 6, 8
    phi = synth.t2_basis(T, K)
    cvec = crandn(rng, K, ny, nz)
    xt = np.einsum("tk,kyz->tyz", phi, cvec)
    alpha = np.einsum("tk,tyz->kyz", phi, xt)[None]
    maps = np.ones((1, 1, ny, nz), complex)
    got = O.synthesize_te(alpha, maps, phi, list(range(T)))[:, 0]
    assert np.abs(got - xt).max() < 1e-12


# ----------------------------------------------------------------------------------
# pre-processing: calibration average, coil compression, readout decoupling, projection
# ----------------------------------------------------------------------------------
def _sparse_from_full(rng, yfull, mask):
    """Sparse readout lines of a full k-space yfull [Ctot][T][Nx][Ny][Nz] at the sampled
    (t, ky, kz) of mask, in a shuffled order."""
    t, a, b = np.nonzero(mask)
    order = rng.permutation(len(t))
    t, a, b = t[order], a[order], b[order]
    lines = np.stack([yfull[:, t[j], :, a[j], b[j]] for j in range(len(t))])
    return lines, t, a, b


def test_preprocess_equals_dense_projection_of_decoupled_kspace():
    """Projection from the sparse lines equals Phi^T P applied to the readout-decoupled
    dense k-space; the readout transform is checked against the centred DFT matrix."""
    rng = np.random.default_rng(20)
    Ctot, C, T, K, nx, ny, nz = 5, 3, 10, 3, 12, 10, 8
    phi = synth.t2_basis(T, K)
    mask = (rng.random((T, ny, nz)) < 0.3).astype(np.uint8)
    yfull = crandn(rng, Ctot, T, nx, ny, nz) * mask[None, :, None]
    lines, t, a, b = _sparse_from_full(rng, yfull, mask)
    W = np.linalg.qr(crandn(rng, Ctot, C))[0]
    ytil, m2 = O.preprocess(lines, t, a, b, W, phi, ny, nz)
    assert np.array_equal(m2, mask)
    Dx = centred_dft_matrix(nx)
    yv = np.einsum("ctxyz,cd->dtxyz", yfull, W)
    xdec = np.einsum("xk,dtkyz->dtxyz", Dx.conj().T, yv)          # centred unitary IDFT along x
    ref = np.einsum("tk,dtxyz->xdkyz", phi, xdec * mask[None, :, None])
    assert np.abs(ytil - ref).max() < 1e-12


def test_compression_is_lossless_for_data_in_a_coil_subspace():
    """Calibration data spanning a C-dimensional channel subspace: the compression matrix
    is orthonormal, spans that subspace, orders by energy and keeps all of the data."""
    rng = np.random.default_rng(21)
    Ctot, C, w = 8, 3, 6
    B = crandn(rng, C, Ctot)
    Z = crandn(rng, w ** 3, C) * np.array([3.0, 2.0, 1.0])
    cal = (Z @ B).T.reshape(Ctot, w, w, w)
    W = O.compression_matrix(cal, C)
    assert np.abs(W.conj().T @ W - np.eye(C)).max() < 1e-12
    X = cal.reshape(Ctot, -1).T
    assert np.linalg.norm(X - X @ W @ W.conj().T) < 1e-10 * np.linalg.norm(X)
    energy = np.linalg.norm(X @ W, axis=0)
    assert np.all(np.diff(energy) < 0)
    i = np.argmax(np.abs(W), axis=0)
    assert np.all(np.abs(W[i, range(C)].imag) < 1e-15) and np.all(W[i, range(C)].real > 0)


def test_calibration_average_over_echoes():
    """Two echoes sampling the same central (ky, kz) are averaged; a line outside the
    window is ignored; an unsampled window point stays zero."""
    Ctot, nx, ny, nz, w = 2, 8, 8, 8, 4
    lines = np.zeros((3, Ctot, nx), complex)
    lines[0] = 1.0
    lines[1] = 3.0
    lines[2] = 100.0
    ky = [4, 4, 0]
    kz = [5, 5, 0]
    cal = O.calibration_average(lines, ky, kz, ny, nz, w)
    assert cal.shape == (Ctot, w, w, w)
    assert np.all(cal[:, :, 2, 3] == 2.0)        # (ky, kz) = (4, 5) -> window (2, 3)
    assert np.count_nonzero(cal) == Ctot * w      # only that point, all w kx samples


# ----------------------------------------------------------------------------------
# direct pins of the helpers the composite functions use
# ----------------------------------------------------------------------------------
def test_llr_norm_brute_force_blocks():
    """sum_n ||R_n alpha||_* with blocks cut by explicit index sets: rows (sy + i b + r) mod Ny,
    columns likewise, the last block partial, one matrix per map set; nuclear norms by
    numpy's matrix norm."""
    rng = np.random.default_rng(41)
    M, K, Ny, Nz, b, sy, sz = 2, 3, 6, 5, 4, 3, 2
    a = crandn(rng, M, K, Ny, Nz)
    total = 0.0
    for m in range(M):
        for i0 in range(0, Ny, b):
            rows = [(sy + i0 + r) % Ny for r in range(min(b, Ny - i0))]
            for j0 in range(0, Nz, b):
                cols = [(sz + j0 + c) % Nz for c in range(min(b, Nz - j0))]
                X = np.array([[a[m, k, y, z] for k in range(K)] for y in rows for z in cols])
                total += np.linalg.norm(X, "nuc")
    assert abs(O.llr_norm(a, b, sy, sz) - total) < 1e-12 * total


def test_adjoint_data_forms_agree_and_reject_unknown():
    phi, maps, mask, rng = tiny_problem(43)
    y = crandn(rng, 2, 6, 8, 8)
    te = O.adjoint_data(y, "te", maps, mask, phi)
    pr = O.adjoint_data(O.project(y, mask, phi), "proj", maps, mask, phi)
    assert np.abs(te - pr).max() < 1e-12 * np.abs(te).max()
    with pytest.raises(ValueError):
        O.adjoint_data(y, "raw", maps, mask, phi)


def test_sense_pair_is_adjoint_and_backprojection_round_trips():
    phi, maps, mask, rng = tiny_problem(44, M=2)
    x = crandn(rng, 2, 3, 8, 8)
    yc = crandn(rng, 2, 3, 8, 8)
    lhs = np.vdot(yc, O.sense(x, maps))
    rhs = np.vdot(O.sense_adj(yc, maps), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    alpha = crandn(rng, 2, 2, 8, 8)
    xt = O.backproject(alpha, phi)                     # [M][T][..]
    back = np.einsum("tk,mt...->mk...", phi, xt)       # Phi^T x with orthonormal columns
    assert np.abs(back - alpha).max() < 1e-12 * np.abs(alpha).max()


# ----------------------------------------------------------------------------------
# wavelet soft-threshold of the coefficient volume (Sec. II.C, Sec. III.C)
# ----------------------------------------------------------------------------------
def haar_matrix(n):
    """One level of the orthonormal Haar analysis on n points, written from its
    definition: row i < n/2 is (e_2i + e_2i+1)/sqrt(2), row n/2 + i is (e_2i - e_2i+1)/sqrt(2)."""
    H = np.zeros((n, n))
    for i in range(n // 2):
        H[i, 2 * i] = H[i, 2 * i + 1] = 1 / np.sqrt(2)
        H[n // 2 + i, 2 * i] = 1 / np.sqrt(2)
        H[n // 2 + i, 2 * i + 1] = -1 / np.sqrt(2)
    return H


def dense_pyramid(shape, levels):
    """Dense matrix of the 3D Haar pyramid on vec(v) (C order): level l is the Kronecker
    product of the three 1D Haar matrices of the current approximation block, embedded in
    the identity on every other coefficient."""
    N = int(np.prod(shape))
    W = np.eye(N)
    idx = np.arange(N).reshape(shape)
    n = list(shape)
    for _ in range(levels):
        sub = idx[:n[0], :n[1], :n[2]].ravel()
        L = np.eye(N)
        L[np.ix_(sub, sub)] = np.kron(np.kron(haar_matrix(n[0]), haar_matrix(n[1])), haar_matrix(n[2]))
        W = L @ W
        n = [m // 2 for m in n]
    return W


@pytest.mark.parametrize("shape,levels", [((4, 2, 4), 1), ((4, 4, 8), 2), ((8, 4, 8), 2), ((8, 8, 8), 3)])
def test_haar3_is_the_dense_pyramid(shape, levels):
    rng = np.random.default_rng(11)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    W = dense_pyramid(shape, levels)
    assert np.allclose(W @ W.T, np.eye(W.shape[0]), atol=1e-13)  # orthonormal
    c = O.haar3(v, levels)
    assert np.abs(c.ravel() - W @ v.ravel()).max() < 1e-13
    assert np.abs(O.ihaar3(c, levels) - v).max() < 1e-13


def test_wavelet_denoise_threshold_zero_is_identity():
    rng = np.random.default_rng(12)
    a = rng.standard_normal((8, 2, 3, 4, 8)) + 1j * rng.standard_normal((8, 2, 3, 4, 8))
    for lev in (1, 2):
        assert np.abs(O.wavelet_denoise(a, 0.0, lev) - a).max() < 1e-13


def test_wavelet_denoise_large_threshold_is_the_block_mean():
    """With tau above every detail magnitude only the coarsest Haar approximation is left:
    the projection on volumes constant over aligned 2^L cubes, i.e. the cube means."""
    rng = np.random.default_rng(13)
    a = rng.standard_normal((8, 1, 2, 8, 16)) + 1j * rng.standard_normal((8, 1, 2, 8, 16))
    for lev in (1, 2, 3):
        f = 1 << lev
        got = O.wavelet_denoise(a, 1e6, lev)
        Nx, M, K, Ny, Nz = a.shape
        cube = a.reshape(Nx // f, f, M, K, Ny // f, f, Nz // f, f).mean(axis=(1, 5, 7))
        want = np.repeat(np.repeat(np.repeat(cube, f, axis=0), f, axis=3), f, axis=4)
        assert np.abs(got - want).max() < 1e-12


def test_wavelet_denoise_shrinks_one_detail_atom():
    """A volume that is one detail basis function times c comes back as
    max(|c| - tau, 0) e^(i arg c) times the same function; a constant volume is kept."""
    shape, lev = (4, 4, 8), 2
    W = dense_pyramid(shape, lev)
    for i, c in [(5, 3.0 - 4.0j), (100, 0.5j), (127, -2.0)]:  # detail indices (the approximation is 0, 1)
        atom = (W.T[:, i]).reshape(shape)
        for tau in (0.1, 1.0, 10.0):
            got = O.wavelet_denoise((c * atom)[:, None, None], tau, lev)[:, 0, 0]
            shrink = max(abs(c) - tau, 0.0) / abs(c)
            assert np.abs(got - shrink * c * atom).max() < 1e-13
    const = np.full((4, 1, 1, 4, 8), 2.5 - 1j)
    assert np.abs(O.wavelet_denoise(const, 100.0, lev) - const).max() < 1e-13


def test_soft_threshold_closed_form():
    c = np.array([3 + 4j, -0.3, 0.0, 1j * 2.0])
    got = O.soft_threshold(c, 1.0)
    assert np.allclose(np.abs(got), np.maximum(np.abs(c) - 1.0, 0.0), atol=1e-15)
    nz = np.abs(got) > 0
    assert np.allclose(got[nz] / np.abs(got[nz]), c[nz] / np.abs(c[nz]))
