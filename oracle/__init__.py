"""FP64 CPU oracle of the partitioned bidomain step with spectral deferred
correction (Algorithm 2 of the paper) -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

This package is the correctness authority for the CUDA library.  It is a
plain, slow, double-precision restatement of the paper's equations written
independently of the CUDA path: the two share no code, no tables and no
helpers.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the library never calls it and has no CPU fallback.

Modules
  fem       P1 stiffness / mass assembly (Sec. 3.2, Eqs. (3.6)-(3.9))
  lr91      Luo-Rudy 1991 membrane model (Sec. 2, "Luo-Rudy model")
  tp06      ten Tusscher-Panfilov 2006 epicardial model (Sec. 2, "Ten Tusscher model")
  cell      node vector field, complex-step Jacobian, rest state
  bidomain  ROS2 (Eqs. (3.13)-(3.14)), SDC correction (Eq. (3.20)),
            Algorithm 2 generalised to Gauss-Lobatto nodes, activation times

Parity status of each function is stated in its module docstring.
"""
