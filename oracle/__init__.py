"""FP64 CPU oracle for the batched Lax / PDHG Hamilton-Jacobi solver.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or links
anything in this directory: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path;
the only thing both sides read is ``paper_1803_01215_gb300.workloads`` (seeded
input draws, no arithmetic of the method).

Contents
  counter_rng  splitmix64 used as a counter-based generator for the random
               initial guess (Section 6: x^0 within 0.1 of the target in the
               max-norm, p^0 within 0.1 of zero).
  families     the Hamiltonians H(x, p), their p-proximal maps, gradients and
               the quadratic terminal cost g (Section 2, H = max_u{<f,p> - L}),
               including the eikonal family c(x)|p|_2 of Section 6.1 (shrink_2
               dual step; the negative equation through phi = -psi).
  lax_pdhg     Algorithm 1 (Lax formula, backward Euler) with the concrete
               updates of Section 5.3 and the loop of Appendix Algorithm A.1,
               and the value fval of Eq. (disclaxBE).
  hopf_pdhg    Algorithm 2 (Hopf formula, backward Euler, Eq. dischopf) as the
               appendix's Hopf tutorial algorithm: the joint prox of g* and
               delta H at j = 1, x_0 eliminated through the conjugate of g.
  lax_schemes  the Lax saddle problem with forward Euler (Eq. disclaxFE) and
               the trapezoid average of the two Euler forms, costates indexed
               by interval as in Eq. disclaxFE, same PDHG steps as lax_pdhg.
  game_schemes Algorithm 3 with the forward-Euler and trapezoid forms (the
               averaging Section 7 proposes for the Lax discretisations).
  retry        rounds for the points that reach the iteration cap (the
               paper's sigma raise and reruns, Sections 6.1 and 6.2).
  game_pdhg    Algorithm 3 (Lax form for differential games, Eq.
               discgenlaxhopfdg) for Section 6.2's difference-of-norms game:
               shrink_2 dual steps for both players, a descent step for the
               minimiser and an ascent step for the maximiser.

Pins: see tests/test_oracle_pins.py, tests/test_oracle_hopf_pins.py,
tests/test_oracle_eikonal_pins.py, tests/test_oracle_game_pins.py and
tests/test_oracle_schemes_pins.py, tests/test_oracle_game_schemes_pins.py
and tests/test_oracle_retry_pins.py.  Closed form (quadratic H), discrete
Riccati (linear drift), direct collocation (tanh drift), the discrete
characteristic (KKT) equations with complex-step derivatives of an H written
independently from the quadcopter dynamics, the primal/dual value identity, and
brute-force search for tiny cases.
"""
