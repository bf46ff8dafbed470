"""B300-native dual-regularized LQR solver and the interior-point method
around it.

Modules (each a thin ctypes binding of the CUDA library _lib/librlqr.so,
built in-tree by csrc/build.py; no CPU fallback):
  rlqr    -- include/rlqr.h: factor / solve / residual, batched and ragged
             solves, cross-stage variables, diagonal Delta_i, horizon shards
  ipm     -- include/rlqr_ipm.h: the batched regularized IPM on the
             cart-double-pendulum
  mlp     -- include/rlqr_mlp.h: the IPM's learned warm start
  shard   -- the multi-rank protocol of the horizon-sharded solve
  inputs  -- seeded synthetic workloads (no arithmetic of the method)
"""
