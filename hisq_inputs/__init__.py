"""Seeded synthetic inputs (fields and workload definitions) shared by tests and benchmarks.

Holds no Dslash or solver arithmetic; see `fields` for the generator definitions.
"""
from . import fields, workloads  # noqa: F401
