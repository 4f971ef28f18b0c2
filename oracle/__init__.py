"""Plain FP64 CPU oracle for the neural GCDF hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
calls this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path:
both sides read their inputs from the seeded generators in ``synth`` and
nothing else.

Contents
  mlp      network input (Sec. III-C: concat of p and q), MLP forward, the
           hand-derived reverse input Jacobian and the sin/cos chain rule,
           evaluated on the *un-split* input so the CUDA path's first-layer
           split (an exact re-association) is tested rather than assumed.
  reduce   per-waypoint min / soft-min / hinge collision cost and gradient
           over the pairs of Eq. (11) / the stacked vector of Eq. (14).
  robot    synthetic capsule robots, their signed distance f_s (Eq. 1) and
           the brute-force GCDF of Definition 1 over a sampled zero-level set
           (Eq. 8, second form), with the closed-form gradient of Theorem 1.
  planner  the trajectory optimisation of Sec. IV-A (Eq. 10 with the velocity
           controls eliminated, the l1 GCDF penalty of Eq. 12) as a fixed
           number of Levenberg-Marquardt steps preconditioned by the
           tridiagonal Hessian of the smooth terms (FP64 Cholesky).
  sparse   the spatial partition of Sec. IV-A (planar range of the reference
           base), the dense->sparse GCDF Jacobian of Eq. (17)/(18) and the
           single-step projection of Theorem 1.
  fit      per-sample field values and their vector-Jacobian products with
           respect to the weights and q (first order: the distance loss of
           Table I; second order: losses on grad_q f).
  labels   labelled (q, p, f) samples of a capsule robot's sampled GCDF
           (the data generation of Sec. III-C), for fitting on exact labels.
  metrics  the relative-error measures used by every parity test.

Every function states the passage it follows.  Parity pins live in
``tests/test_oracle_*.py``.
"""
from . import mlp, reduce, robot, metrics, planner, sparse, fit  # noqa: F401
