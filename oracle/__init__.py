"""FP64 CPU oracle of the clustered-Potts PEPS branch-and-bound method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and
reference legs of ``bench.py`` use it.  It shares no code with the CUDA
library; the two meet only in the seeded generators of ``instances``.

The oracle is written step by step from the method of arXiv:2502.02317
(SpinGlassPEPS.jl), in plain NumPy (LAPACK SVD/QR as library primitives), with
no blocking, fusion or reordering beyond what each step states:

* ``tables``   -- Eq. 1 / Eq. 2 and Sec. 2: spins grouped into clusters, the
  local energy table of every cluster over all its states ("full spectrum")
  and the pairwise table of every grid edge, reduced to its distinct rows and
  columns with projectors (Sec. 3.1, "Sparsity"); for clusters of more than
  8 spins (Sec. 3.1.1: Pegasus, Zephyr) the sparse form, whose pairwise
  tables are over the coupled spins' configurations only.
* ``peps``     -- Sec. 2, Fig. 1(c): Boltzmann weights at inverse temperature
  beta and the row MPOs of the PEPS on the square and king's lattices
  (sparse factor graphs: classes over a cluster's interface configurations,
  site tensors by grouping the states' terms).
* ``boundary`` -- Sec. 2, Fig. 1(d) and Sec. 3.1 (``MpsParameters``,
  ``SVDTruncate``): bottom-up boundary MPSs by MPO-MPS zipper application with
  SVD truncation to bond dimension chi, then variational sweeps.
* ``search``   -- Sec. 2 and Sec. 3.1 (``SearchParameters``,
  ``merge_branches``): conditional marginals from the cached environments,
  branch merging on the boundary of the explored region, pruning to
  ``max_states``, exact energies of the final states, and the droplets
  (low-energy excitations) collected in the merges.
* ``lattice``  -- Sec. 3.1 (lattice transformations): the instance solved on
  each of the 8 rotations / reflections of the grid, states mapped back to
  the original sites, the best of 8 kept.
* ``metrics``  -- Fig. 3 (c), (f): the diversity of a set of solutions
  (within an approximation ratio of the best energy, pairwise more than N/2
  variables apart).
* ``exact``    -- pins that do not use any of the above: brute force over all
  spin configurations (<= 24 spins), spin-level row transfer matrices for
  width-3 Chimera strips (exact log Z and exact ground energy), and sums over
  the interface spins of large clusters (exact log Z, ground energy and the
  first cluster's marginal); ``bruteforce.c`` (loaded by ``native``) is the
  same brute force in C with OpenMP, for up to 30 spins.

Where the paper leaves a point open, the reading taken is stated in the
docstring of the function that implements it.
"""
