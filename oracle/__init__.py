"""CPU oracle for affinity propagation and its partition / landmark variants.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 statement of
what the method computes (Algorithms 1-3 of Xia et al., "Local and global
approaches of affinity propagation clustering for large scale data").  Only
the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never calls it, and it shares no
code with the CUDA library.

Modules:
  ap    -- Algorithm 1 (Eq. 1-4, damping, decisions, outputs) in two forms:
           the literal triple loop and the top-2 / column-sum form.
  pap   -- Algorithm 2 (partition, sub-runs, block-diagonal merge, warm start).
  lap   -- Algorithm 3: Steps 1-2 (landmark AP, nearest-exemplar assignment), Steps 1-4
           (gate, recursion, merge) and Step 4's refinement of the centre set.
  mlp   -- the learned warm-start network (features, forward, backward, Adam).
  rng   -- splitmix64, restated independently of the CUDA path.

Parity status: every function is pinned by a ``-m "not gpu"`` test except
``mlp.row_features``' scaling choice and Table 1's "accuracy", which the
paper leaves undefined ("parity unpinned").
"""
