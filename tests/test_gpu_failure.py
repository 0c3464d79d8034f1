"""Failure handling without a GPU fault: an allocation failure is reported as T2SH_ENOMEM
and leaves the context usable; a bounded device wait that runs out (a barrier nothing
completes) is reported as T2SH_ETIMEOUT by the next t2sh_sync and leaves the plan usable."""
import ctypes

import numpy as np
import pytest

import oracle as O

from t2sh_cases import crandn
from test_gpu_parity import T, c64, dev, host, make_plan, nrmse, random_problem  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def small_solve_matches_oracle(T, seed):
    rng, phi, mask, maps = random_problem(seed, 1, 32, 24, 2, 8, 4, 1)
    y = crandn(rng, 1, 2, 8, 32, 24) * mask[None, None] * 0.1
    with make_plan(T, phi, mask, maps, block=8, lam=0.02, iters=6, seed=1) as p:
        got = host(p.solve(c64(y), T.KSPACE_TE))
        p.sync()
    ref = O.fista(y[0].astype(np.complex64).astype(np.complex128), "te", maps[0], mask, phi, 0.02, 8, 6, 1)
    assert nrmse(got[0], ref) < 1e-4


def test_allocation_failure_is_reported_and_the_context_survives(T):
    """A plan whose maps alone would need ~8.8 PB: the first device allocation fails, the
    call returns T2SH_ENOMEM before any input is read (the pointers given are small device
    buffers), and the device keeps working."""
    d = T.make_dims(512, 512, 64, 8, 4, nslices=65535, block=8, iters=2)
    small = torch.zeros(1024, dtype=torch.complex64, device="cuda")
    h = ctypes.c_void_p(0)
    st = torch.cuda.current_stream()
    status = T.lib().t2sh_plan(ctypes.byref(d), ctypes.c_void_p(small.data_ptr()), ctypes.c_void_p(small.data_ptr()),
                               ctypes.c_void_p(small.data_ptr()), ctypes.c_void_p(st.cuda_stream), ctypes.byref(h))
    assert status == T.ENOMEM
    assert not h.value
    assert len(T.last_error()) > 0
    torch.cuda.synchronize()
    small_solve_matches_oracle(T, 51)


def test_bounded_wait_timeout_is_reported_and_the_plan_stays_usable(T):
    rng, phi, mask, maps = random_problem(52, 1, 32, 24, 2, 8, 4, 1)
    y = crandn(rng, 1, 2, 8, 32, 24) * mask[None, None] * 0.1
    with make_plan(T, phi, mask, maps, block=8, lam=0.02, iters=6, seed=1) as p:
        p.wait_selftest(2_000_000)  # 2 ms
        with pytest.raises(T.T2shError) as e:
            p.sync()
        assert e.value.status == T.ETIMEOUT
        p.sync()  # the flag was cleared
        got = host(p.solve(c64(y), T.KSPACE_TE))
        p.sync()
    ref = O.fista(y[0].astype(np.complex64).astype(np.complex128), "te", maps[0], mask, phi, 0.02, 8, 6, 1)
    assert nrmse(got[0], ref) < 1e-4
    with pytest.raises(T.T2shError):
        p2 = make_plan(T, phi, mask, maps)
        try:
            p2.wait_selftest(0)
        finally:
            p2.close()


def test_plan_memory_is_reused_bitwise_and_released(T):
    """Plan buffers come from the library's stream-ordered pool.  A second plan made after
    the first is destroyed reuses that memory (free device memory does not drop again),
    solves bitwise like the first although its buffers still hold the first plan's data,
    and release_cached hands the cached memory back to the device."""
    S, ny, nz, C, Tn, K = 48, 128, 96, 8, 16, 4
    rng, phi, mask, maps = random_problem(53, S, ny, nz, C, Tn, K, 1)
    y = c64(crandn(rng, S, C, Tn, ny, nz) * mask[None, None] * 0.1)
    d = T.make_dims(ny, nz, C, Tn, K, nslices=S, block=8, lam=0.02, iters=4, seed=3)
    ws = T.workspace_bytes(d)
    assert ws > 200e6
    torch.cuda.synchronize()
    T.release_cached()
    free0 = torch.cuda.mem_get_info()[0]
    torch0 = torch.cuda.memory_reserved()
    outs, live = [], []
    for _ in range(2):
        with make_plan(T, phi, mask, maps, block=8, lam=0.02, iters=4, seed=3) as p:
            outs.append(host(p.solve(y, T.KSPACE_TE)))
            p.sync()
            live.append(torch.cuda.mem_get_info()[0])
    cached = torch.cuda.mem_get_info()[0]
    assert np.array_equal(outs[0], outs[1])
    assert free0 - live[0] > 0.9 * ws
    assert abs(live[1] - live[0]) < 0.1 * ws  # the second plan took no new memory
    assert free0 - cached > 0.9 * ws          # destroyed plans' memory stays cached
    T.release_cached()
    # what torch's own allocator kept of the solve outputs is not the plan pool's
    torch_kept = torch.cuda.memory_reserved() - torch0
    assert free0 - torch.cuda.mem_get_info()[0] - torch_kept < 0.1 * ws
