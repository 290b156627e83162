"""Plain FP64 CPU oracle for grouped-qubit MPS TEBD of the 2D TFIM.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its
Python binding, the batching/serving layers) may import, call or link anything
in this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is written from the paper (Mandra et al., "A Heuristic for Matrix Product
State Simulation of Out-of-Equilibrium Dynamics of Two-Dimensional Quantum Spin
Systems"), Sec. II (Eq. hamiltonian, Eq. trotter_step, Eq. initial_state,
Eq. z2_tot), Sec. III (TEBD with grouped sites, Eq. Z_tot, F_MPS,
Eq. Z_tot_via_F, Eq. z2_tot_rescaled, Table gamma_scaling), and shares no code
with the GPU path.

Modules
-------
model        TFIM parameters, theta_min, temperatures, PBC bonds.
layout       row grouping into blocks, snake order, bond bounds, gate schedule.
statevector  exact state-vector Trotter simulator (<= 24 qubits).
mps          plain MPS TEBD: dense SVD truncation per bond (numpy/LAPACK).
rescale      F and F^gamma rescaling, gamma_fit table.
xy           the XY-model workload of the Supplemental Material (open grid, one qubit per
             site, depth-7 Trotter step, Eq. xy_init, the signal of Eq. xy_signal): state
             vector and TEBD by SWAP routing.

The 3D variant (Supplemental Material, 3D TFIM section) is in model / layout / statevector / mps
(the ``Lz`` arguments).

Every function either has a pin in ``tests/test_oracle_*.py`` (closed forms,
symmetries, brute force, a library routine) or says "parity unpinned".
"""
