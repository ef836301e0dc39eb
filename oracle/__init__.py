"""CPU oracle for the tanTRG hot path (arXiv 2212.11973).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, dense FP64
restatement of what the GPU library computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and
``--impl reference``) may import it.  It shares no code with the CUDA
library under ``paper_2212_11973_gb300/`` and never imports it.

Modules
-------
model   lattice and snake order (Fig. 1(a)), the Hubbard Hamiltonian of Eq. 3
        (and its particle-hole symmetric form used in the DQMC appendix)
        built densely from second quantisation with a mode-level
        Jordan-Wigner transform, exact diagonalisation, U=0 closed forms.
mpo     the Hubbard MPO W as a finite automaton, dense tensors.
tantrg  the dense super-MPS tanTRG integrator: rho_h(beta0) = I - beta0 H/2,
        right canonicalisation, Lanczos exponential (Supplement, "Lanczos-
        based exponential method"), 1-TDVP sweeps (Supplement, "Procedure of
        1-TDVP"), 2-TDVP growth sweeps (Supplement, "2-TDVP in the initial
        stage"), bilayer measurements (Supplement, Choi transformation).

Pins: see tests/test_oracle_*.py.  Every function names the passage it
follows; where the paper is silent the reading taken is stated inline.
"""
