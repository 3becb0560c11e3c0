"""Plain, slow FP64 CPU oracle for the simulated-bifurcation (SB) tracking path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything here. The
product path (the CUDA library and its Python binding) never imports, links or
runs this package, and this package imports nothing from the product.

Every function follows one passage of the paper (Okawa, Zeng, Tao, Yung,
"Quantum-Annealing-Inspired Algorithms for Track Reconstruction at High-Energy
Colliders", arXiv:2402.14718) and cites it by section / equation:

* ``philox``   -- Philox4x32-10 counter-based generator (Salmon et al., SC'11),
                  the published definition; used for the synthetic events and
                  the SB initial state.
* ``events``   -- synthetic barrel events standing in for the TrackML data
                  (section "Dataset"): helices in a 2 T solenoid, 10 layers.
* ``qubo``     -- doublets -> triplets (Eq. 16 cuts) -> consistent / conflicting
                  triplet pairs (Eq. 17) -> the QUBO of Eq. 13 as CSR.
* ``ising``    -- QUBO <-> Ising conversion (T = (1+s)/2), energies of Eq. 13.
* ``sb``       -- aSB / bSB / dSB time evolution, Eq. 1-12, symplectic Euler.
* ``bruteforce`` -- exhaustive ground state of Eq. 13 for N <= 22.
* ``tracks``   -- selected triplets -> doublets -> track candidates, and the
                  efficiency / purity of Eq. 18-19.
* ``ttt``      -- time-to-target (section "Results", Table 1 definition).
* ``adjoint``  -- reverse-mode gradient of the relaxed bSB energy.

Functions whose result has no independent pin say "parity unpinned" in their
docstring.
"""
