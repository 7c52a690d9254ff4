"""Oracle for the DPVO differentiable bundle-adjustment layer.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import, call or execute anything in this
package.  It shares no code, header, table or helper with the CUDA path in
``paper_2208_04726_b300/``; the two meet only in the seeded scene generator
(``paper_2208_04726_b300/scenes.py``), which holds none of the method's arithmetic.

Contents
--------
``dense_gn``      plain FP64 Gauss-Newton that solves the full dense normal
                  equations (no Schur complement), Sec. 3.1 Eq. 6.
``schur``         FP64 Schur-complement solve of the same normal equations, used
                  only to pin the dense solve and to inspect the reduced pose system.
``unrolled_grad`` FP64 torch-autograd twin of the unrolled iterations, written
                  independently of ``dense_gn``, giving the reference gradient of a
                  loss on the final state w.r.t. targets and weights.
``pose_loss``     FP64 pose supervision loss of Sec. 3.4 (Eq. 7): a matrix-logarithm
                  form with central-difference gradients, and a differentiable torch
                  form for the gradient through the unrolled twin.
``corr``          the correlation features of Sec. 3.2 (Eq. 4): the definition written out,
                  and the correlation-volume form the paper names as equivalent.
``window``        the sliding optimisation window of Sec. 3.3 (constant-velocity pose,
                  median-depth patches, dropping the oldest frame, the patch-graph
                  edges and their reprojection targets), in numpy.

Parity unpinned: nothing here is checked against the authors' implementation,
which is not available; every pin is mathematical (finite differences, exact
recovery, closed forms, library least squares, invariances).
"""
