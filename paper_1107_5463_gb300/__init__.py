"""GB300 (sm_103a) checkerboard single-spin-flip Metropolis for O(n) lattice
spin models (Weigel & Yavors'kii, Physics Procedia 15, 2011, Section 2).

The compute path is the C-ABI library ``libspinmc.so`` built from ``csrc/``;
``paper_1107_5463_gb300.spinmc`` is its thin Python binding.  Importing this
package does not load the library; importing ``spinmc`` does, and fails loudly
if it has not been built.
"""
