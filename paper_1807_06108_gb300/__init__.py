"""GB300-native MPPI on jump-diffusion processes (information-theoretic MPC,
Wang, Williams & Theodorou).

The compute path lives in the CUDA library ``libmppi_jump.so`` built from
``csrc/``; :mod:`paper_1807_06108_gb300.mppi` is its ctypes binding and
:mod:`paper_1807_06108_gb300.workloads` describes seeded synthetic problems.
Importing this package loads nothing; importing ``mppi`` loads the library and
raises if it is missing.
"""

__all__ = ["workloads"]
