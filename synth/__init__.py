"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module only draws random numbers and arranges them with the symmetries the
inputs must have (Hermiticity, time reversal, momentum structure).  It holds none
of the method's arithmetic, so both the oracle and the GPU path can use it
without sharing any computation.
"""
from .gen import (Problem, make_problem, make_operator, kmesh_neg, pair_index, random_amplitudes,
                  random_probe, CONFIGS)

__all__ = ["Problem", "make_problem", "make_operator", "kmesh_neg", "pair_index", "random_amplitudes",
           "random_probe", "CONFIGS"]
