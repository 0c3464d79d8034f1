"""Test-side helpers: the oracle's synthetic acquisitions and a complex normal draw."""
from oracle.acquire import proj_scan, te_case  # noqa: F401


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
