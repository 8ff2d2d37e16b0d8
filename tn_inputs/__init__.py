"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds tensor networks (Ising, random-entry lattices, dimer
covers, corner-double-line) and ordered approximate contraction trees, and
reads/writes their file formats.  It holds none of the contraction or
compression arithmetic of the method: both the CPU oracle and the CUDA
library consume what it writes.
"""
from .formats import Network, Tree, read_network, write_network, read_tree, write_tree  # noqa: F401
