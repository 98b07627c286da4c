// FP64 coefficient tables of the MMVM finish step, generated on the host.
//
// In units where c = 2 lambda^2 = 1 (scaled moments a_l = M_l c^{-|l|/2}, and
// the stream-function correlation Psi[beta] of the pair kernel), the moment
// equation of eq:Final_CrossCoef becomes
//   dM_k/dt = c^{|k|/2 - 1} [ sum_l a_l sum_beta coef(k,l,beta) Psi_tot[beta]
//                             + (X_1 a_{k-e1} + X_2 a_{k-e2}) / M_00 ]
// where the (k, l, beta, coef) entries collect the (i, q) double sums of
// eq:FinalSingleI (Gamma^I, velocity component 1, W_1[g] = -Psi[g + e2]) and
// eq:FinalSingleII (Gamma^II, component 2, W_2[g] = Psi[g + e1]) times the
// projection prefactor c_k (eq:coefficient):
//   Gamma^I : coef = -(-1)^{|k|+|l|} C(l1,i) C(l2,q) 4^{i+q+1-|k|} / ((k1-i-1)! (k2-q)!)
//             beta = (k1+l1-2i-1, k2+l2-2q+1)
//   Gamma^II: coef = +(-1)^{|k|+|l|} C(l1,i) C(l2,q) 4^{i+q+1-|k|} / ((k1-i)! (k2-q-1)!)
//             beta = (k1+l1-2i+1, k2+l2-2q-1)
// (the lambda powers of eq:FinalSingleI/II, c_k and the velocity scaling all
// combine into the single factor c^{|k|/2-1}).  Psi_tot adds the self pair,
// Psi_self[beta] = sum_m a_m psi0[m + beta], with psi0 the jet at the origin
// of the stream function of a Gaussian vortex (c = 1):
//   psi0[(2p, 2q)] = -(1/4pi) (-1)^{p+q} [(2p)!/p!] [(2q)!/q!] / (p+q),  p+q >= 1,
// and 0 for any odd index (the closed forms H_1, H_2 of Appendix A.1 are its
// first derivatives: H_1(a) = -psi0[a+e2], H_2(a) = psi0[a+e1]).
#pragma once

#include <vector>

namespace mmvm {

struct FinishTables {
  int M = 0, K = 0, NB = 0, NJ = 0;
  std::vector<int> k_off;    // K+1 offsets into the entry arrays, grouped by k
  std::vector<int> e_l;      // moment column l
  std::vector<int> e_b;      // Psi column beta (bcol)
  std::vector<double> e_c;   // coefficient
  std::vector<double> psi0;  // psi0 for |alpha| <= NJ, column q(|alpha|) + alpha_2
};

// entries = false leaves out the (k, l, beta) entries (their number grows
// like M^6; the separable single-particle path does not use them).
FinishTables build_finish_tables(int M, bool entries = true);

// Factors of the separable single-particle path (self_high.cu): binom is
// row-major (M+1) x (M+1), binom[l][q] = C(l, q); g[j] = 4^{-j} / j!, j <= M;
// cg[(l (M+1) + k) (M+1) + q] = binom[l][q] * g[k - q] (the FP64 product, 0
// for q > min(l, k)), so that the passes do one multiply-add per term.
struct SeparableTables {
  std::vector<double> binom, g, cg;
};
SeparableTables build_separable_tables(int M);

}  // namespace mmvm
