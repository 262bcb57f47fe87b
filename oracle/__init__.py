"""FP64 CPU oracle for the Gross-Pitaevskii split-step method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, calls or
links anything under this directory; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

The oracle is a plain, slow, obviously-correct restatement of what the paper
(Kobayashi et al., "Quantum turbulence simulations using the Gross-Pitaevskii
equation: HPC and new numerical benchmarks") computes, in float64/complex128,
written with numpy.  It has its own FFT (``oracle.fft``) and shares no code,
table or constant generator with the CUDA path.

Modules
-------
fft          recursive mixed-radix (2/3) DFT, forward/inverse, 1D and 3D
rng          counter-based SplitMix64 stream (Steele, Lea & Flood 2014)
scheme       parameters (Sec. 4.1), sub-flows and Strang steps (Sec. 4.3)
diagnostics  N, E, hydrodynamic split, Helmholtz split, spectra (Sec. 3.4-3.5, 4.1)
initial      SRP (Sec. 5.3) and RVR (Sec. 5.4) initial conditions
adjoint      vector-Jacobian products of the split step (no counterpart in the paper)
argle        imaginary-time ARGLE step, E_v, Taylor-Green and ABC start fields (Sec. 4.2, 5.1-5.2)
structure    velocity and longitudinal structure functions (Sec. 3.5)
helicity     helicity and regularised helicity with their spectra (Sec. 3.6)

Pinning: every public function is checked by ``tests/test_oracle_*.py``
against brute force, closed forms, invariants or library routines; the one
function that has no such pin says "parity unpinned" in its docstring.
"""
