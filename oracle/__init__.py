"""FP64 CPU oracle for the light-transport camera model (TEST INFRASTRUCTURE).

This package is test infrastructure only.  It is a plain, slow restatement of
the paper's model (McGaffin, Chen, Fessler, Sick, "A practical light transport
system model for chemiluminescence distribution reconstruction"), written in
numpy float64, against which the CUDA path is compared.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it.  It shares no code with the CUDA path and imports
nothing from the product package.

Modules
  optics     -- Table I ray maps and their composition (Sec. II-A)
  transport  -- 1-D transport entries: Table III (pillbox), Table II (Dirac),
                and an independent phase-space polygon-clipping evaluation
  camera     -- single-lens and plenoptic camera operators (Sec. II-C..F, III):
                explicit matrices, matrix-free forward/adjoint, sampled outputs
  rotation   -- rotated perspectives by three-pass shears (Sec. III-A)
  recon      -- the reconstruction algorithm of Table V (Sec. V)

Parity status: every function is pinned by a test in tests/test_oracle_*.py
against a value fixed independently of this code (closed forms, a second
geometric evaluation, brute-force quadrature, library solvers, invariants).
"""
