"""Seeded synthetic inputs shared by the GPU path and the oracle (data only)."""
from . import scenes  # noqa: F401
from ._lib import bvh_build, bvh_validate, poisson_disc  # noqa: F401
