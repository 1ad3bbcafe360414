"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This package holds no arithmetic of the numerical method: it only samples closed-form
fields (meshes, coefficients, manufactured solutions and their sources) at nodes.
"""
from .rng import SplitMix64
from . import meshes, problems
from .problems import (Problem, SCHEME_CONSERVATIVE, SCHEME_PAPER, config1, config2,
                       config3, config4_instance, config5, continuity_problem,
                       parabolic_problem, paper_parabolic_e1, paper_continuity_e3,
                       CoupledPair, coupled_pair)
