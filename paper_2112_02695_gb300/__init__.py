"""GB300-native fast-spectral Boltzmann collision operator (C ABI + binding).

`boltz` is the ctypes binding of libboltz.so (include/boltz.h); `workloads`
generates the seeded synthetic inputs; `build` compiles the library in-tree
for sm_103a.  Importing the package does not load the library; importing
`paper_2112_02695_gb300.boltz` does, and fails loudly if it is missing.
"""
