"""CPU oracle for approximate tensor-network contraction (test infrastructure).

Plain, slow, FP64 numpy restatement of what the GPU library computes, used
only by the tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg
of ``bench.py``.  The product path never imports it.  It shares no code with
the CUDA library: both sides only read the same network and tree files
written by ``tn_inputs``.

Modules:
  approx  -- Algorithm 1 over an explicit ordered tree: pairwise contraction
             (Eq. 1 as a matrix product over the shared bonds) and bond
             compression (QR of A, LQ of B, SVD of R_A R_B truncated to chi,
             sqrt(sigma) absorbed into both sides; Eq. "svd"), with an exact
             power-of-two running log-norm.
  exact   -- independent references: brute-force sums over spin / edge
             configurations, row transfer matrices, closed forms, perfect
             matching counts, and full einsum contraction of tiny networks.
  gauge   -- compression in the tree gauge of distance r (Algorithm 2's
             spanning tree, QR inwards on virtual copies, projector form).
  grad    -- d log|Z| / d T_v: the same schedule re-run with its operands
             kept, then walked backwards (matrix-product adjoints, the exact
             power-of-two rescale, and the adjoint of the truncated SVD of
             X = A B for each compression), in plain numpy FP64.

Every function states the passage of the paper it follows.  Where the paper
is silent the reading used is stated in the docstring.
"""
