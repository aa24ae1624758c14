"""Seeded synthetic inputs shaped like the paper's planted (l,d) workloads.

This module holds no part of the motif finder's arithmetic: it only writes
ASCII DNA (and, for the protein alphabet, ASCII amino-acid letters).  Both
the CUDA library's tests/benchmark and the CPU oracle's tests draw their
inputs from here, so every comparison runs on identical bytes.
"""
from .planted import (CONFIGS, Instance, instance_for_config, mix_instances,  # noqa: F401
                      planted_instance, planted_protein)
