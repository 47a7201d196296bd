"""FP64 CPU oracle for the precomputed random walker of Andrews & Hamarneh, "Adaptable
Precomputation for Random Walker Image Segmentation and Registration" (arXiv 1607.04174).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import anything from this package.  The product path (the
CUDA library and its Python binding) never imports, calls or links it, and this package never
imports the product: the two share no code.  The only shared module is ``synth`` (seeded input
generators, no random-walker arithmetic).

Every function follows the paper's notation and cites the section / equation it restates.  All
arithmetic is float64 (NumPy / SciPy); no blocking, fusion or reordering beyond what the cited
definition states.  Modules:

* ``graph``     image graph, Eq. (W), D, L = D - W (Sec. II-A); normalized Laplacian (Sec. II-C)
* ``priors``    Gaussian-fit priors P from the seeds (Sec. IV-A)
* ``exact``     basic RW: the linear system Eq. (rw_eq) (Sec. II-A), normalized form (Sec. II-C)
* ``eig``       smallest eigenpairs of L or L-hat, Eq. (L_eigs) (Sec. II-B)
* ``fastrw``    fast RW, Eqs. (E_def)-(Fs) (Sec. II-B), factored and dense-block restatements
* ``adaptive``  number of eigenvectors from the seeds, Eq. (alpha_1), and from priors, Eq. (g)
                (Sec. III-A)
* ``refine``    k damped-Jacobi (default) or Jacobi-preconditioned CG steps on Eq. (rw_eq)
                from a starting guess (a refinement the paper does not have)
* ``update``    Rayleigh-quotient eigenvalue update, Eq. (z_ray) (Sec. III-B); edge edits
* ``aggregate`` super-vertex aggregation of the basis, Eqs. (q_agg_1), (q_agg_2) (Sec. III-C)
* ``adjoint``   gradients of a loss on U w.r.t. edge weights and beta through the exact solve
* ``registration`` displacement labels, patch-difference priors and the unseeded solve
                (Sec. II-A, III-A-2, IV-B)
* ``pipeline``  the whole online solve composed from the pieces above

Parity notes: the parts without a pin beyond this code itself say so in their docstrings
("parity unpinned").
"""
