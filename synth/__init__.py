"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

Input generation only: no force, integrator or energy arithmetic of the method
lives here.
"""
from .plummer import plummer, sample_active, ensemble, ensemble_member, salpeter_masses  # noqa: F401
