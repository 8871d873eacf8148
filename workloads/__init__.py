"""Seeded synthetic inputs shared by the CPU oracle and the GPU binding.

Nothing here computes the superblock product, the Lanczos iteration or a
gradient: the modules only build operator blocks and random arrays.
"""
from .superblock import Pair, Superblock, seeded_normal

__all__ = ["Pair", "Superblock", "seeded_normal"]
