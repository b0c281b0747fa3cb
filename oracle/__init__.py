"""Plain FP64 CPU oracle for the Recursive MRCM (arXiv 2009.07965).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or
executes this package: only the tests, the smoke check and the CPU-baseline
leg of the benchmark do.  It shares no code with the CUDA path; both draw
their inputs from the separate `inputs` package.

Modules (each function cites the passage of the paper it follows):
  geometry   leaves, interface segments and the Robin coefficient (Eqs.
             decomp.1-2, robin.beta, permeff; Section 4)
  fine       O1, the fine-scale lumped-RT0 / two-point-flux solve (Eqs.
             ellip.1-3; Section 2.2 on RT0 = conservative finite volumes)
  local      the local Robin problems and MMBFs (Eqs. 11.2-12.2, 11a-11b)
  mrcm       O2, the non-recursive MRCM with the global interface system
             (Eqs. linsys, brhs, final) -- the parity target
  recursive  the CPU Recursive MRCM (Algorithm 1, Eqs. particular.1-2)
  brute      monolithic dense solve of Eqs. 11.2-14.2 on tiny grids
  counts     number of MMBFs per decomposition (Table ntmmbfs)
  refine     double-double residual of Eqs. 11.2-14.2 and iterative
             refinement of the discrete solution
  dd         double-double helpers (TwoSum, Dekker's TwoProd)
  cnn        the surrogate network's 3 x 3 convolutions and their gradients
  mrcm3d     the 3D counterparts (Section 5.1): fine solve, box leaves,
             interface patches, local Robin problems and O2 over patches
"""
