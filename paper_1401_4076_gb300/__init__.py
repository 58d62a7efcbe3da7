"""GB300-native parallel multicanonical lattice gas (sm_103a CUDA behind a C ABI).

``paper_1401_4076_gb300.mucal`` is the ctypes binding of ``libmucal.so``;
``paper_1401_4076_gb300.workloads`` holds the seeded workload descriptions.
"""
