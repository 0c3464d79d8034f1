"""t2sh_objective: the data term of Eq. 5 at x, per slice, against the oracle's definition
(T-form and projected k-space, one and two map sets, a ragged shape), host buffers, and
its use between resumable solve steps (the solver state is not touched)."""
import numpy as np
import pytest

import oracle as O

from t2sh_cases import crandn
from test_gpu_parity import T, c64, host, make_plan, random_problem  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def close(a, b, scale, tol=2e-5):
    return abs(a - b) <= tol * scale


@pytest.mark.parametrize("S,ny,nz,C,Tn,K,M", [(2, 64, 48, 4, 12, 4, 1), (2, 96, 36, 3, 10, 3, 2)])
def test_objective_matches_oracle_both_forms(T, S, ny, nz, C, Tn, K, M):
    rng, phi, mask, maps = random_problem(700 + ny, S, ny, nz, C, Tn, K, M)
    y = crandn(rng, S, C, Tn, ny, nz) * 0.1
    x = crandn(rng, S, M, K, ny, nz) * 0.3
    xs = x.astype(np.complex64).astype(np.complex128)
    ys = y.astype(np.complex64).astype(np.complex128)
    ytil = np.stack([O.project(ys[s], mask, phi) for s in range(S)])
    with make_plan(T, phi, mask, maps) as p:
        h_te, c_te = p.objective(c64(y), T.KSPACE_TE, c64(x))
        h_pr, c_pr = p.objective(c64(ytil), T.KSPACE_PROJ, c64(x))
        p.sync()
    for s in range(S):
        h, c = O.data_term(ys[s], "te", maps[s], mask, phi, xs[s])
        hp, _ = O.data_term(ytil[s].astype(np.complex64).astype(np.complex128), "proj", maps[s], mask, phi, xs[s])
        # scale: the two inner products that h subtracts
        w = O.normal(xs[s], maps[s], O.space_time_kernel(mask, phi))
        scale = 0.5 * abs(np.vdot(xs[s], w)) + abs(h) + c
        assert close(h_te[s], h, scale), (s, h_te[s], h)
        assert close(c_te[s], c, c), (s, c_te[s], c)
        assert close(h_pr[s], hp, scale), (s, h_pr[s], hp)
        assert np.isnan(c_pr[s])


def test_objective_host_buffers_and_between_iterations(T):
    """A host-buffer plan gives the same values; calling it between solve steps leaves the
    solve bitwise unchanged; the solve lowers the data term below its value at 0."""
    S, ny, nz, C, Tn, K = 2, 64, 48, 4, 12, 4
    rng, phi, mask, maps = random_problem(733, S, ny, nz, C, Tn, K, 1)
    y = (crandn(rng, S, C, Tn, ny, nz) * mask[None, None] * 0.1).astype(np.complex64)
    x = (crandn(rng, S, 1, K, ny, nz) * 0.3).astype(np.complex64)
    kw = dict(block=8, lam=0.01, iters=12, seed=5)
    with make_plan(T, phi, mask, maps, **kw) as p:
        ref = host(p.solve(c64(y), T.KSPACE_TE))
        h_d, c_d = p.objective(c64(y), T.KSPACE_TE, c64(x))
        p.solve_begin(c64(y), T.KSPACE_TE)
        p.solve_iterate(5)
        p.objective(c64(y), T.KSPACE_TE, c64(x))
        p.solve_iterate(7)
        got = host(p.solve_end())
        h_sol, c_sol = p.objective(c64(y), T.KSPACE_TE, c64(ref))
        p.sync()
    assert np.array_equal(got, ref)
    assert np.all(h_sol < 0.0)  # f(x_solve) < f(0) = c
    d = T.make_dims(ny, nz, C, Tn, K, nslices=S, flags=T.HOST_IO, **kw)
    with T.Plan(d, phi.astype(np.float32), mask.astype(np.uint8), maps.astype(np.complex64)) as ph:
        h_h, c_h = ph.objective(y, T.KSPACE_TE, x)
    np.testing.assert_allclose(h_h, h_d, rtol=1e-9, atol=1e-9 * np.abs(c_d).max())
    np.testing.assert_allclose(c_h, c_d, rtol=1e-12)
