"""GB300-native hot path of the controllability method (CMCG) for time-harmonic
Maxwell's equations: DG time-domain period sweeps, their discrete adjoint, the
conjugate-gradient outer loop and the e^{i omega t} filter, behind the C ABI
declared in ``include/cmcg.h``.

Submodules are imported on demand: ``cmcg`` (the ctypes binding of
``libcmcg.so``), ``inputs`` (seeded synthetic workloads), ``build`` (compiles
the CUDA library).
"""
