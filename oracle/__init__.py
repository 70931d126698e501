"""FP64 CPU oracle for the SD-OCT model-based reconstruction (ISAM forward model,
its adjoint, the proximal steps and FISTA).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct numpy in float64 that
restates the paper's definitions.  Only the test-suite, the package smoke check
and the benchmark's CPU-baseline leg may import it; the library itself never
does, and it shares no code with the CUDA path (inputs come from the seeded
workload generators, which hold no reconstruction arithmetic).

Modules:
  isam     -- system operator Phi and its adjoint (Sec. 2.1, Eqs. for_model /
              back_model), both as a direct non-uniform DFT and as the
              Kaiser-Bessel NUFFT the paper uses; the paper's Hilbert-form
              back-projection and the literal zero-pad / DFT form of Phi.
  wavelet  -- orthonormal Daubechies wavelet (4 vanishing moments) built by
              spectral factorisation, and its periodic 2-D transform.
  fista    -- penalties, proximal maps, power iteration, ISTA and FISTA
              (Sec. 2.2-2.3, Eq. alg).
  tv       -- isotropic total variation (Sec. 2.2) and its prox by fast gradient
              projection on the dual.
  evaluate -- the evaluation loop of Sec. 3: direct ISAM on interpolated
              measurements, the NCC of Eq. ncc, the golden-section lambda search.
  volume   -- the ISAM operator of a 3-D volume (both lateral axes), direct sum.
"""
