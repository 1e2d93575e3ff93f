"""FP64 CPU oracle for the fast graph Fourier transform (Lu & Ortega,
"Fast Graph Fourier Transforms Based on Graph Symmetry and Bipartition").

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
the test suite, the smoke check in ``__graft_entry__`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA path: the
only common module is ``gft_workloads``, which draws inputs and holds none of
the transform's arithmetic.

Everything is plain, slow and in float64:

* ``graph``    -- Laplacian from weights and back (Eqs. 3-5), involutions and
                  phi-symmetry (Definitions 1-2), the permuted butterfly matrix
                  B_phi (Eq. 20), block diagonalisation (Thm. 3) and the
                  closed-form weights of G+ / G- (Thm. 4).
* ``jacobi``   -- cyclic-by-row Jacobi eigensolver (Golub & Van Loan's
                  symmetric Schur rotations), the solver behind every basis.
* ``gft``      -- the dense GFT (eigenvectors of L, ascending eigenvalues),
                  the paper's stage-by-stage decomposition (Sec. IV-C and the
                  recursion at its end), the fast basis U = B_1...B_S diag(U_k),
                  and dense / staged application to signal batches.
* ``right_haar`` -- the right Haar stage of bipartite graphs (Sec. III-A,
                  Lemma 1, Thms. 1-2): the two sub-transforms E and F and the
                  output-side Haar units.
* ``approx``   -- approximate GFT by greedy layers of Jacobi rotations, alone
                  and after the Haar stages (Haar + approximate GFT, Sec. VI-B).
* ``givens``   -- layered Givens rotations (Eq. 1, Fig. 1) for the learned
                  surrogate: forward, loss and central finite differences.
* ``metrics``  -- the error measures RE (Eq. 23), delta and epsilon (Sec. VI-B).

Parity status of each function is stated in its docstring; every function
has a pin in ``tests/test_oracle_*.py``.  The paper's operation counts are
pinned where its runtime table fixes them; the 25-joint skeleton's printed
counts are not reproduced ("parity unpinned", see the design notes).
"""
from . import graph, jacobi, gft, givens, metrics, right_haar, approx  # noqa: F401
