"""CPU oracle for MPS time evolution of the ab-initio electronic Schroedinger
equation (Frahm & Pfannkuche, "Ultrafast ab-initio Quantum Chemistry Using
Matrix Product States").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package; only the test-suite, the smoke check and
the benchmark's CPU-baseline and reference (``--impl reference``) legs use it.  It shares no code with the CUDA
implementation; the two meet only in the seeded input generators (``synth``).

* ``oracle.fci`` -- full configuration interaction in the occupation-number
  basis of Eq. (fci): the dense Hamiltonian of Eq. (hamil) built by literal
  second-quantised action, exact propagation by diagonalisation
  (Eq. time_evo_opera), the paper's RK4 (stages k1..k4, Eq. rk_add) and
  Krylov (Eqs. kry_orth, kry_non, krylov_evo) steps on vectors, and the
  one-body reduced density matrix of Section 3.2.
* ``oracle.mps`` -- the MPS algorithm of Section 2.2 step by step, on dense
  site tensors carrying (N, 2S_z) labels: variational fitting of Eq. (add_min)
  with the local linear problems solved by projecting the exact target vector
  onto the current left/right bases, RK4 and Krylov steps built from those
  fits, and SVD compression (Section 2.1).  It is only meant for small L.

All arithmetic is float64 / complex128.
"""
