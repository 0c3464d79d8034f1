"""Serving loop: scans that arrive while others are on the GPU are admitted as memory
frees up, run concurrently, and give the same result as when solved alone."""
import numpy as np
import pytest

import t2sh_synth as synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_04195_gb300 import build as B
    B.build()
    from paper_1809_04195_gb300 import t2sh
    return t2sh


SHAPES = [(4, 64, 48, 4, 16, 4), (3, 96, 64, 3, 12, 4), (2, 48, 48, 6, 10, 3)]  # S, ny, nz, C, T, K


def make_request(T, serve, scan_id, scanner, arrival, shape_index):
    S, ny, nz, C, Tn, K = SHAPES[shape_index]
    rng = np.random.default_rng(1000 + scan_id)
    phi = torch.from_numpy(synth.t2_basis(Tn, K).astype(np.float32)).cuda()
    mask = torch.from_numpy(synth.vd_masks(Tn, ny, nz, 0.25, rng)).cuda()
    maps = torch.from_numpy(np.stack([synth.coil_maps(C, ny, nz, rng) for _ in range(S)]).astype(np.complex64)).cuda()
    k = (rng.standard_normal((S, C, K, ny, nz)) + 1j * rng.standard_normal((S, C, K, ny, nz))) * 0.05
    kspace = torch.from_numpy(k.astype(np.complex64)).cuda()
    dims = T.make_dims(ny, nz, C, Tn, K, nslices=S, block=8, lam=0.01, iters=20 + 5 * shape_index, seed=scan_id)
    return serve.ScanRequest(scan_id, scanner, arrival, shape_index, dims, phi, mask, maps, kspace, T.KSPACE_PROJ)


@pytest.mark.gpu
def test_continuous_batching_matches_solo_solves(T):
    from paper_1809_04195_gb300 import serve
    arrivals = serve.poisson_arrivals(6, 3, mean_gap_s=0.01, seed=4)
    reqs = [make_request(T, serve, i, s, t, i % 3) for i, (t, s) in enumerate(arrivals)]
    budget = 2 * max(serve.footprint_bytes(T, r.dims, r.kform) for r in reqs) + 1  # about two scans at once
    srv = serve.Server(T, budget, iters_per_tick=7)
    for r in reqs:
        srv.submit(r)
    rep = srv.run()
    assert rep["scans"] == 6 and rep["max_concurrent_scans"] >= 2
    assert rep["latency_p99_s"] >= rep["latency_p50_s"] > 0
    for r in srv.done:
        assert r.done_s >= r.admitted_s >= r.arrival_s
        with T.Plan(r.dims, r.phi, r.mask, r.maps) as p:
            alone = p.solve(r.kspace, r.kform)
        assert torch.equal(alone, r.result), r.scan_id


@pytest.mark.gpu
def test_admission_refuses_a_scan_larger_than_the_budget(T):
    from paper_1809_04195_gb300 import serve
    r = make_request(T, serve, 0, 0, 0.0, 0)
    srv = serve.Server(T, 1024)
    with pytest.raises(ValueError):
        srv.submit(r)


def test_poisson_arrivals_are_ordered_and_seeded():
    from paper_1809_04195_gb300 import serve
    a = serve.poisson_arrivals(200, 4, 300.0, seed=1)
    b = serve.poisson_arrivals(200, 4, 300.0, seed=1)
    assert a == b and [t for t, _ in a] == sorted(t for t, _ in a)
    assert {s for _, s in a} == {0, 1, 2, 3}
    gaps = np.diff([t for t, _ in a])
    assert 40 < gaps.mean() < 110  # 4 scanners x 1 per 300 s -> mean merged gap 75 s
