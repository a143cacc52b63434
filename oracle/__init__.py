"""FP64 CPU oracle for the D3Q19 pseudopotential MRT lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method of Li, Du, Fei, Luo and Yu, "Three-dimensional
non-orthogonal multiple-relaxation-time lattice Boltzmann model for multiphase
flows" (arXiv 1805.08643), written with numpy in float64.  It exists to check
the CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product package never does,
and it shares no code, table or constant with the CUDA sources.

Parity pins: every function is checked in ``tests/test_oracle_*.py`` against
something other than itself (the matrices the paper prints, closed forms,
invariants, Maxwell values the paper prints).  One reading stays unpinned
beyond physics-level agreement: the exact equilibria and forcing moments the
authors used for the *orthogonal* operator, which the paper does not print
(``lbm_oracle.meq_orth`` / ``forcing_orth``; see the module docstring).

``d3q15`` restates the D3Q15 non-orthogonal variant the paper says can be
built the same way (Sec. II A) but does not print; its readings are listed in
that module's docstring and pinned in ``tests/test_oracle_d3q15.py``.
"""
