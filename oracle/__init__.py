"""FP64 CPU oracle for the FIFA-GP Gibbs step (Moran & Wheeler, arXiv 2006.06537).

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously correct
restatement of what the GPU path computes, written from the paper:

* ``detmath``  -- the deterministic exponential and the two covariance kernels
                  (squared exponential of Sec. 2.1 / Sec. 4.1, Matern-5/2).
* ``rng``      -- Philox4x32-10 counter-based generator (Salmon et al. 2011),
                  Box-Muller normals, Marsaglia-Tsang gamma draws.
* ``tree``     -- the HODLR partition tree of Sec. 3.2 (recursive 2x2 split).
* ``aca``      -- partial-pivoted cross approximation of an off-diagonal block
                  (the "partial-pivoted LU" of the proof of Lemma 1).
* ``hodlr``    -- assembly of the HODLR matrix, its dense reconstruction,
                  the matrix-vector product and the shift M~ = s C~ + I.
* ``factor``   -- symmetric factorization A = W W^T (SI, HODLR decomposition
                  and factorization), log-determinant (SI, determinant
                  computation), application of W, W^T, W^-1, W^-T and solve.
* ``sampler``  -- Algorithm 1 draw of f, and one Gibbs iteration (Sec. 4.1).
* ``dense``    -- the exact dense Gaussian-process posterior of Eq. (gp_posterior),
                  the exact conjugate conditionals and the KL divergence of the
                  proof of Theorem 4.1.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package. The product path (the CUDA library and its Python
binding) never imports it, and this package never imports the product.
"""
