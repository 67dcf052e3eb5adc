"""Seeded synthetic workloads shared by the tests, the smoke check and the
benchmark.  No method arithmetic lives here (see ``workloads``)."""
from .workloads import (  # noqa: F401
    ACGT, GENERATORS, INDEX_SEED, Collection, Workload, documents, genome, genomes, make,
    random_bases, random_kmers, substring_queries, tiny, uneven,
)
