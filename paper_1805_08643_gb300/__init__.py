"""GB300 (sm_103a) D3Q19 pseudopotential MRT lattice Boltzmann library.

Implements the per-time-step update of Li, Du, Fei, Luo and Yu,
"Three-dimensional non-orthogonal multiple-relaxation-time lattice Boltzmann
model for multiphase flows" (arXiv 1805.08643), for the paper's non-orthogonal
transformation matrix (Eq. 12) and the usual orthogonal one, as CUDA kernels
behind the C ABI of ``include/lbm.h``.

``Lattice`` (module ``lbm``) is the ctypes binding; ``thermo`` gives
coexistence densities for initial states; ``synth`` the seeded synthetic
workloads.  Importing ``lbm`` requires the built ``liblbm.so``.
"""

__all__ = ["lbm", "thermo", "synth"]


def __getattr__(name):
    if name in ("Lattice", "Rates", "LBMError"):
        from . import lbm

        return getattr(lbm, name)
    raise AttributeError(name)
