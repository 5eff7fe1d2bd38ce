"""Plain, slow, FP64 CPU oracle for classical and all-floating FETI.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports, links or runs this
package; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` do.  It shares no code with the CUDA path: it has its own
element integrals, index maps, rigid-body modes, generalized inverses and
projected CG, written from the paper (Augustin, Holzapfel & Steinbach,
"Classical and all-floating FETI methods for the simulation of arterial
tissues"), section by section, with dense LAPACK / SuperLU as library steps.

Parity status per function is stated in each module header.
"""
