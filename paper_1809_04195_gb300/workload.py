"""Device-resident synthetic scans for throughput measurements and the serving driver.

Structure (basis, masks, 3D phantom, coil maps) comes from the seeded generator
t2sh_synth; the k-space is produced on the GPU by the library's own forward operator
(t2sh_forward, projected form) plus projected Gaussian noise drawn with torch.  These
inputs serve timing runs only; the parity tests build theirs with the FP64 oracle.
"""
from __future__ import annotations


def make_scan(sh, S: int, dev):
    """Device-resident synthetic scan: phi, mask, maps [S][C][M][ny][nz], projected k-space
    ytil [S][C][K][ny][nz] = Phi^T P (F S Phi alpha_true + w), scaled to max |ytil| = 1
    (alpha_true in the first map set, zero in the others)."""
    import numpy as np
    import torch

    import t2sh_synth as synth

    from . import t2sh
    phi, mask, te = synth.scan_common(sh)
    vol = synth.EllipsoidVolume.draw(synth.rng_for(sh.seed, 4, 0))
    N = sh.ny * sh.nz
    M = sh.nmaps
    maps = torch.empty((S, sh.ncoils, M, sh.ny, sh.nz), dtype=torch.complex64, device=dev)
    alpha = torch.zeros((S, M, sh.nbasis, sh.ny, sh.nz), dtype=torch.complex64, device=dev)
    for s in range(S):
        st = synth.slice_structure(sh, s, volume=vol)
        xt = synth.decay_series(st.rho, st.t2, te)
        a = np.einsum("tk,tyz->kyz", phi, xt)
        maps[s] = torch.from_numpy(st.maps.astype(np.complex64)).to(dev)
        alpha[s, 0] = torch.from_numpy(a.astype(np.complex64)).to(dev)  # image in the first map set
    phi_d = torch.from_numpy(phi.astype(np.float32)).to(dev)
    mask_d = torch.from_numpy(mask).to(dev)
    d = t2sh.make_dims(sh.ny, sh.nz, sh.ncoils, sh.nechoes, sh.nbasis, nslices=S, nmaps=M)
    with t2sh.Plan(d, phi_d, mask_d, maps) as p:
        ytil = p.forward(alpha, t2sh.KSPACE_PROJ)
    # sigma = 1 % of the largest echo-0 sample of the central slice
    c = min(S - 1, S // 2)
    d1 = t2sh.make_dims(sh.ny, sh.nz, sh.ncoils, sh.nechoes, sh.nbasis, nslices=1, nmaps=M)
    with t2sh.Plan(d1, phi_d, mask_d, maps[c:c + 1].contiguous()) as p:
        sig = 0.01 * float(p.forward(alpha[c:c + 1].contiguous(), t2sh.KSPACE_TE)[:, :, 0].abs().max())
    # projected noise Phi^T P w, w ~ CN(0, sigma^2) per echo, drawn echo by echo
    gen = torch.Generator(device=dev)
    gen.manual_seed(sh.seed)
    mk = mask_d.to(torch.float32).reshape(sh.nechoes, 1, 1, N)
    for s0 in range(0, S, 8):
        s1 = min(S, s0 + 8)
        acc = torch.zeros((s1 - s0, sh.ncoils, sh.nbasis, N), dtype=torch.complex64, device=dev)
        for t in range(sh.nechoes):
            w = torch.randn((s1 - s0, sh.ncoils, 1, N), dtype=torch.complex64, device=dev, generator=gen)
            acc += (sig * w * mk[t]) * phi_d[t].reshape(1, 1, sh.nbasis, 1)
        ytil[s0:s1] += acc.reshape(s1 - s0, sh.ncoils, sh.nbasis, sh.ny, sh.nz)
    ytil /= ytil.abs().max()
    del alpha
    return phi_d, mask_d, maps, ytil
