"""B300-native Riccati sweep of the quasiclassical Eilenberger method
(SuperConga, arXiv 2205.15000): C-ABI library ``libsc.so`` + thin binding.

``paper_2205_15000_b300.sc`` loads the compiled library and raises if it is
missing; ``paper_2205_15000_b300.workloads`` builds seeded synthetic inputs.
"""
