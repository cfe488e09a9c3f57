"""Plain FP64 CPU oracle of the tensor-network branch-and-bound method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
anything from here.  The CUDA library never calls it and shares no code with
it: the oracle builds every MPO column as a dense array straight from the
definition (a sum over cluster states of Boltzmann factors times index
deltas) and then runs textbook dense MPS algebra with numpy.

Modules
-------
energy  the exact Ising energy of Eq. (1) (int64 numerators)
potts   clustering of Ising spins into Potts variables (Sec. III, Eqs. 2-4)
peps    dense row MPOs, zipper + variational boundary MPS, log Z (Figs. 5-8, Eq. 9)
search  conditional marginals and branch-and-bound with boundary merging (Eqs. 5-8, Figs. 3, 6)
brute   exhaustive enumeration for tiny instances (test pins only)
"""
