"""FP64 CPU oracle of the Allegro edge hot path -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously correct definition that the CUDA
path is checked against.  Only the tests, the smoke check of the package entry
module and the CPU-baseline leg of the benchmark may import it; the product
path never does, and the CUDA path shares no code with it (no kernels, helpers,
tables or constant generators).  The only shared module is `synth`, which
draws seeded inputs and holds none of the method's arithmetic.

Contents and the passages they follow (arXiv 2304.10061):
  neighbors  ordered pairs (i, j, image shift) within r_c -- Sec. "Allegro"
             (per-ordered-pair energies) and "Species-dependent cutoffs".
  so3        real spherical harmonics, real-basis Wigner-3j coupling tensors,
             tensor-product path enumeration and the fused path tensor --
             Eq. (1) ("eq:tp") and Sec. "Optimized tensor product".
  allegro    the model: energy decomposition (Sec. "Allegro"), two-body MLP,
             embedding, env weights, environment sum (Eq. 1, second line),
             tensor product, latent MLP, edge-energy MLP, FP64 final stage
             (Sec. "Mixed-precision calculations"); forces and virial by
             torch autograd.
  verlet     velocity-Verlet integration (Sec. "Problem Overview").
  zbl        the ZBL screened nuclear repulsion of the production potential
             (Sec. "Training details").

Where the paper is silent the oracle takes one stated reading (basis,
envelope, normalisations, path weights, sign conventions), restated in the
docstring of the function that uses it.
"""
