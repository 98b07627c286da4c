"""FP64 CPU oracle for the multi-moment vortex method (MMVM) right-hand side.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_1010_2475_gb300``); the only module both
sides use is ``mmvm_inputs``, which draws seeded states and holds none of the
method's arithmetic.

What it computes (Uminsky, Wayne & Barbaro, "A multi-moment vortex method for
2D viscous fluids", arXiv:1010.2475), in plain float64 numpy, following the
paper's own order of steps:

* ``coefficients``: the projection prefactor c_k (eq:coefficient), the
  closed forms H_1, H_2 (Appendix A.1, after eq:Fullint), the literal double
  sums Gamma^I, Gamma^II (eq:FinalSingleI, eq:FinalSingleII) and their sum
  Gamma-tilde (eq:moment_evolutionFinish).
* ``pair_jet``: the cross-term kernel H^B(alpha; s) = D^alpha V_00(b; sqrt(2)
  lambda) at b = s (Appendix A.2, the display after eq:FinalCrossII).  The
  paper gives no closed form for s != 0; the oracle evaluates the defining
  derivative through the integral F(x) = int_0^1 exp(-x t) dt of the Gaussian
  core factor (1 - exp(-x))/x, differentiated under the integral sign and
  summed by Gauss quadrature.
* ``rhs``: the full right-hand side A + B + C (eq:Final_CrossCoef) with the
  centroid velocity eq:xjdot_Final, the literal coefficient-tensor form for
  small orders and the regrouped velocity-jet form (the paper's own
  intermediate step before the Gaussian self-convolution, Appendix A.1) for
  large problems, and classic RK4 with lambda(t)^2 = lambda_0^2 + 4 nu t
  (eq:phi00) at the stage times.

Readings of the paper taken here (each is pinned by a test, see
``tests/test_oracle_*.py``):

* separation s_{j,j'} = x^j - x^{j'} (eq:xjdotA's definition; the other sign
  printed after eq:mom_multi in Section 2.2 fails first-moment conservation
  and the brute-force Biot-Savart quadrature);
* in the cross term B the binomial (vorticity) index l belongs to the target
  particle j and the velocity index m to the source j' (the derivation in
  Appendix A.1 puts the l-derivatives on omega^j); the printed labelling
  M^{j'}[l] M^j[m] fails the same two checks;
* Gamma^II integrates the second velocity component (H_2), as its last line
  states;
* the self pair is left out of the centroid sum (eq:xjdot excludes it; its
  value is zero by antisymmetry);
* every sum is truncated at total order <= M (the Galerkin truncation of
  Section 2.1.2).

Parity status: every function here is pinned (closed forms, invariants,
brute-force quadrature, high-precision differentiation); none is "parity
unpinned".
"""
