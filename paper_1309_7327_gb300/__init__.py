"""GB300-native (sm_103a) hot path of the SMC method of Emmett, Zhang & Bell,
"High-Order Algorithms for Compressible Reacting Flow with Complex Chemistry"
(arXiv 1309.7327): the reacting compressible Navier-Stokes right-hand side
on 3-D structured boxes and the SDC / multirate-SDC sweeps that consume it.

* ``smc``   -- Python binding of the C-ABI library ``libsmc.so`` (argument
               marshalling only; every step runs in the CUDA kernels).
* ``synth`` -- seeded synthetic mechanisms, box layouts and fields.
* ``build`` -- compiles ``csrc/`` for sm_103a into ``libsmc.so``.
"""
