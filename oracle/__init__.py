"""FP64 CPU oracle for the sparse SH codec: TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy restatements of what the codec computes,
written from the paper ("Smaller and Faster 3DGS via Post-Training Dictionary
Learning"): the dictionary-learning objective (Eq. 1), OMP sparse coding and the
alternating dictionary update (Sec. 2.1), decoding radiance straight from the
sparse codes (Sec. 2.2), plus the learned support proposal network.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  The product path (the CUDA library and its Python
binding) never imports it and shares no code with it.

Modules
  sh     real spherical harmonics of degree 1..3 from associated Legendre
         functions; dense SH evaluation; decode = dense evaluation of D alpha
  omp    OMP with Householder-QR least squares recomputed at every step
  mod    MOD dictionary update (ridge-regularised least squares in D with the
         codes fixed), dead-atom refill, and the alternating learning loop
  brute  best s-subset by enumeration (tiny inputs only)
  mlp    support-proposal MLP: forward, backward, BCE loss, Adam step, and the
         candidate-restricted OMP with its fallback rule

Every function is pinned by `-m "not gpu"` tests against closed forms, library
routines, invariants or brute force; see the pin list in each module header.
"""
