"""B300 (sm_103a) implementation of one bounce of wavefront path tracing with the
normalized Russian roulette and splitting of "NRRS: Neural Russian Roulette and
Splitting" (arXiv 2510.07868), behind the C ABI of include/nrrs.h.

``paper_2510_07868_b300.nrrs`` is the ctypes binding (it needs libnrrs.so, built by
``paper_2510_07868_b300.build``); ``paper_2510_07868_b300.inputs`` draws the seeded
synthetic scenes and weights.
"""
