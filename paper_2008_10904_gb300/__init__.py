"""GB300-native matrix-free resolvent analysis by time marching.

Martini, Rodriguez, Towne & Cavalieri, "Efficient computation of global
resolvent modes": the direct and adjoint RK4 marches of a linear system,
forced by a Fourier series and analysed by a streaming DFT, for all
frequencies and a block of test vectors at once, plus the randomized-SVD
glue that turns them into gains and modes.

The compute path is librsv.so (CUDA, sm_103a) behind the C ABI declared in
include/rsv.h; `paper_2008_10904_gb300.rsv` binds it with the same names.
Build it with `paper_2008_10904_gb300.build.build()`.
"""
