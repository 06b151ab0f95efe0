"""Plain FP64 CPU oracle for the randomized low-rank decomposition.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code,
constants table or helper with the CUDA path; the two meet only in the seeded
input generators (``paper_2307_15572_gb300.synth``), which hold none of the
method's arithmetic.

Every routine here is written for obviousness, not speed: numpy FP64, library
primitives (matmul, Householder QR, LAPACK SVD) as single steps, and no
blocking, fusion or reordering beyond what the cited passage states.

Sources:
  * the paper, "Randomized matrix decompositions" paragraph, Eq. (1) and the
    three-step scheme of Fig. 1 (random projection + QR, thin SVD of the
    projected matrix, lift of the left factor), oversampling p = l - R_SVD;
  * Halko, Martinsson & Tropp, SIAM Review 53 (2011), which the paper names as
    the basis of its method: subspace (power) iteration with
    re-orthogonalisation (their Alg. 4.4) and the expected-error bound of their
    Thm. 10.5 (used as a pin in the tests);
  * Yu, Gu & Li, SIAM J. Matrix Anal. Appl. 39 (2018), blocked randQB_EI, for
    the tolerance-driven adaptive loop;
  * Salmon, Moraes, Dror & Shaw, SC'11, for the Philox4x32-10 counter-based
    generator that fixes the random test matrix.

Parity status per function is listed in each module's header.
"""


