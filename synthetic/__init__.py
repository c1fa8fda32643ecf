"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Nothing here computes any step of the filter: it draws ensembles, observation
networks, observation errors and the standard normals of the perturbed
observations from counter-based random streams.
"""
from .philox import normal_stream, philox4x32_10, uint32_stream, uniform_stream
from .workloads import WORKLOADS, Workload
from .fields import Inputs, make_inputs, draw_field, observation_indices, variable_of
from .cycling import CycleInputs, make_cycle_inputs, nature_run

__all__ = ["normal_stream", "philox4x32_10", "uint32_stream", "uniform_stream", "WORKLOADS",
           "Workload", "Inputs", "make_inputs", "draw_field", "observation_indices", "variable_of",
           "CycleInputs", "make_cycle_inputs", "nature_run"]
