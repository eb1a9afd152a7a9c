"""gblbm: D2Q9 bounce-back lattice Boltzmann with per-step body forces
(momentum exchange in both operation orders and the discrete Reynolds transport
theorem of arXiv:2210.10377), as hand-written CUDA for sm_103a behind a C ABI.

``paper_2210_10377_gb300.binding`` loads the compiled library (libgblbm.so)
and raises if it is missing; nothing here falls back to a CPU implementation.
``paper_2210_10377_gb300.inputs`` names the workloads and draws seeded inputs.
"""
