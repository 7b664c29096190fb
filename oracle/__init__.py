"""CPU FP64 oracle for the multilevel entropic-risk gradient hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import anything
from this package.  The product path (``paper_2606_09291_gb300``) never
imports it and shares no code, table or constant generator with it.

The oracle is a plain, slow, step-by-step restatement of the method of
Baumgarten, Guth, Schneiderhan, Vanzan, "Multilevel Stochastic Gradient
Descent for Risk-Averse PDE-Constrained Optimization":

* ``philox``     counter-based normal draws xi (Salmon et al., SC'11), the
                 random input of Sec. 2 / Sec. 5 (iid across samples and levels,
                 Sec. 2.2 after eq:delta-notation).
* ``kl``         Karhunen-Loeve modes of the 1D exponential covariance and the
                 log-normal coefficient at cell centres (Sec. 5 field model; the
                 exponential covariance is the workload's own choice).
* ``fem``        assembled Q1 stiffness / mass matrices by Gauss quadrature,
                 control operator B and its adjoint (eq:sys, Sec. 5).
* ``solve``      sparse direct solve and plain PCG (Sec. 5 solves the state and
                 adjoint PDEs; any exact-to-tolerance solver gives the same
                 discrete solution).
* ``mlmc``       per-sample X, Y (eq:definition_Xell_Yell), level differences
                 (eq:delta-notation), pairwise Chan merge (Algorithm 1,
                 PairwiseUpdate), MLMC sums (eq:ml_estimator_numerator/
                 denominator), gradient (eq:gradient_estimator) and the
                 projected step (eq:gradientdescentMLMC).
* ``controller`` adaptive batch size and level (eq:sec-order-sum,
                 eq:optimal-batch-size, eq:squared-bias-estimate-mlmc,
                 eq:optimal-level, eq:mse-estimate-mlmc).

Everything is float64 numpy / scipy.  Parity status per function is stated in
each module header; the pins live in ``tests/test_oracle_*.py``.
"""
