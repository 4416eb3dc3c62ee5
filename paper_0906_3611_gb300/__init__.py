"""GB300 (sm_103a) two-species soft-glassy lattice Boltzmann library.

The hot path (Benzi et al., arXiv:0906.3611, Sec. II: the fused
force + shifted-BGK + streaming step of both species' D2Q9 populations) runs
in hand-written CUDA kernels inside ``liblb.so``, behind the C ABI of
``include/lb.h``.  ``paper_0906_3611_gb300.lb`` is the ctypes binding with the
same names; ``paper_0906_3611_gb300.build`` compiles the library.
"""
__all__ = ["lb", "build"]
