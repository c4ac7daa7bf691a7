"""Plain, slow FP64 CPU oracle for the sketch-and-solve least-squares path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (the CUDA library and its Python binding) never imports, calls or
links anything here, and this package imports nothing from the product.

What it computes follows "Sketch 'n Solve" (arXiv 2409.14309):

* the least-squares problem  min_x ||A x - b||^2  (Eq. 1, Sec. 1.3);
* the reduced problem  min ||S A x^ - S b||^2  with S in R^{d x m} (Sec. 1.3);
* the method's steps: generate S, form SA and Sb, solve on SA (Sec. 1.2);
* the sketch families the paper names: Clarkson-Woodruff / CountSketch (the
  default, Sec. 1.2.2), Gaussian and subsampled randomized Hadamard (Sec. 1.2.1);
* sketch-and-precondition (SAP-SAS, Sec. 2.1), whose fixed point is the exact
  least-squares solution x*.

Where the paper is silent (hash, signs, scaling, the Gaussian generator, SRHT
sampling, the meaning of "relative residual") the oracle follows the readings
written in each module's docstring.  Every function is pinned by a test in
``tests/test_oracle_*.py`` against something other than itself, except the
LSQR iteration count, which is "parity unpinned" (only its fixed point is
pinned).
"""
