"""GPU parity of the TE-image post-processing (t2sh_postprocess: back-projection at chosen
echoes, virtual-coil images, homodyne along z, root sum of squares) against the oracle's
postprocess().  The band width is an integer decided from the float fraction, so the
oracle receives the same float32-rounded fraction as the library.

Tolerance: one forward and two inverse float32 DFTs along z, a K-term back-projection and
a C-term sum of squares: NRMSE <= 1e-5 over each slice's TE images."""
import numpy as np
import pytest

import oracle as O
import t2sh_synth as synth

from t2sh_cases import crandn, proj_scan
from test_gpu_parity import T, c64, dev, make_plan, nrmse, r32, random_problem  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

POST_TOL = 1e-5


@pytest.mark.parametrize("S,ny,nz,C,Tn,K,M,pf,te", [
    (2, 64, 48, 8, 32, 4, 1, 0.65, [3, 8, 15]),
    (1, 256, 160, 4, 80, 4, 1, 0.65, [3, 8, 15]),
    (1, 260, 240, 7, 80, 4, 2, 0.65, [3, 8, 15]),   # Table I slice matrix, two map sets
    (2, 40, 30, 3, 12, 3, 2, 0.75, [0, 11]),
    (1, 48, 36, 2, 10, 2, 1, 1.0, [0, 1, 2, 3, 4, 5, 6, 7]),  # full fraction: RSS of |TE image|
])
def test_postprocess_matches_oracle(T, S, ny, nz, C, Tn, K, M, pf, te):
    rng, phi, mask, maps = random_problem(600 + ny + M, S, ny, nz, C, Tn, K, M)
    alpha = crandn(rng, S, M, K, ny, nz)
    alpha32 = alpha.astype(np.complex64).astype(np.complex128)
    with make_plan(T, phi, mask, maps) as p:
        got = p.postprocess(c64(alpha), te, pf=pf).cpu().numpy().astype(np.float64)
        p.sync()
    pf32 = float(np.float32(pf))
    for s in range(S):
        ref = O.postprocess(alpha32[s], maps[s], phi, te, pf32)
        e = nrmse(got[s], ref)
        print(f"{ny}x{nz} M={M} pf={pf}: NRMSE {e:.2e}")
        assert e < POST_TOL


def test_postprocess_of_a_reconstruction(T):
    """TE images (PD / intermediate / T2-weighted: echoes 3, 9, 17 of the 5 ms synthetic
    echo train, 20 / 50 / 90 ms for the paper's 21 / 50 / 90 ms) of the solved knee slices."""
    sh = synth.KNEE_320x256x160
    sl = [0, 160]
    phi, mask, maps, ytil = proj_scan(sh, sl)
    phi, maps = r32(phi, maps)
    te = [3, 9, 17]
    with make_plan(T, phi, mask, maps, block=sh.block, lam=sh.lam, iters=20, seed=sh.seed) as p:
        alpha = p.solve(c64(ytil), T.KSPACE_PROJ)
        img = p.postprocess(alpha, te, pf=0.65).cpu().numpy().astype(np.float64)
        a = alpha.cpu().numpy().astype(np.complex128)
    for i in range(len(sl)):
        ref = O.postprocess(a[i], maps[i], phi, te, float(np.float32(0.65)))
        assert nrmse(img[i], ref) < POST_TOL
        assert np.all(img[i] >= 0)


def test_postprocess_rejects_bad_arguments(T):
    rng, phi, mask, maps = random_problem(5, 1, 32, 32, 2, 8, 4, 1)
    with make_plan(T, phi, mask, maps) as p:
        a = c64(crandn(rng, 1, 1, 4, 32, 32))
        for te, pf in [([8], 0.65), ([-1], 0.65), ([0], 0.5), ([0], 1.01), (list(range(8)) + [0], 0.7)]:
            with pytest.raises(T.T2shError):
                p.postprocess(a, te, pf=pf)
