"""GB300-native (sm_103a) solver for effective thermal conductivity with the
D3Q7 MRT lattice Boltzmann model and an off-diagonal relaxation block
(Fang et al., arXiv 1503.08718).

The compute path is libmrtlbm.so (hand-written CUDA, C ABI in include/lbm.h);
`lbm` is its ctypes binding and `build` compiles it.  `inputs` draws the
seeded synthetic cells.
"""
