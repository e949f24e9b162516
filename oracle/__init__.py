"""FP64 CPU oracle of the vMAP training step.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (CPU-baseline leg and the
``--impl reference`` arm) may import it. The CUDA library never calls into
it, and it never calls into the CUDA library.

Modules:
  philox     Philox4x32-10 (Salmon et al., SC'11), the counter-based generator
             both sides implement independently.
  vmap_step  sampling (Eq. 1-2), encoding, MLP, occupancy rendering (Eq. 3),
             losses (Eq. 4-5), backward, Adam, the vectorised step, query.
  evaluate   held-out depth rendering used for the depth-L1 metric.
  hypernet   the warm-start set-encoder hypernetwork, forward and backward.

Parity status per function: every function listed above is pinned by tests
under tests/ (test_oracle_*.py) against closed forms, invariants, finite
differences, brute force or an independent library routine.
"""
