"""FP64 CPU oracle for one MPPI iteration with covariance-variable importance sampling.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs do.  It shares no code, header,
table or constant generator with the CUDA path in ``paper_1509_01149_b300``.

It is the plain, slow, obviously correct statement of what the CUDA path
computes, written from the paper (Williams, Aldrich, Theodorou, "Model
Predictive Path Integral Control using Covariance Variable Importance
Sampling"):

* ``philox``  -- the counter-based noise (Philox4x32-10 from Salmon et al.,
  SC'11, and Box-Muller), turned into delta-u = sqrt(nu) chol(Sigma) eps, the
  exploration noise of Theorem 1 with A = sqrt(nu) I (Sec. III-C).
* ``systems`` -- the three synthetic plants and their state costs (Sec. V
  analogues) in FP64, vectorised over samples.
* ``mppi``    -- path cost S~ with the importance-sampling running cost q~
  (Sec. III-C, the reduced q~), the min-shifted exponential weights, the
  reward-weighted update (Eq. App_PI) and the shift of Algorithm 1.
* ``mlp``     -- the learned-dynamics surrogate (forward, backward, Adam) in FP64.

Parity status per function is listed in each module header.  Pins live in
``tests/test_oracle_pins.py`` and are run with ``pytest -m "not gpu"``.
"""
