"""Seeded synthetic inputs (meshes, initial and boundary data) for the IPCS workloads.

Shared by the oracle, the tests and the benchmark; contains none of the
scheme's arithmetic."""
from . import meshes, problems  # noqa: F401
