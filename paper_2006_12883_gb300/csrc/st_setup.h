// Collocation setup data (host, double precision results of long double work).
#pragma once

#include <complex>

#include "../../include/st.h"

#ifndef MAXM
#define MAXM ST_MAX_M
#endif

namespace st {

struct Colloc {
  int M;
  double tau[MAXM];
  double Q[MAXM][MAXM];
  double K[MAXM][MAXM];               // DG matrix of Eq. (2.9), unit interval
  std::complex<double> lam[MAXM];     // eigenvalues of Q (ordered, see st.h)
  std::complex<double> V[MAXM][MAXM];
  std::complex<double> Vinv[MAXM][MAXM];
  double Pt[2 * MAXM][MAXM];          // slab-bisection prolongation
  double Rt[MAXM][2 * MAXM];          // slab-bisection restriction
  double QI_ie[MAXM][MAXM], QI_lu[MAXM][MAXM], QE[MAXM][MAXM];
};

// 0 on success, negative on failure.
int colloc_setup(int M, Colloc* out);

// M-coarsening between the Radau node sets of one slab (Section 5.2, SMMG):
// P (Mf x Mc) evaluates the coarse nodal polynomial at the fine nodes,
// R (Mc x Mf) = Kc^{-1} P^T Kf restricts collocation-form residuals.
// 0 on success, negative on failure.
int node_transfer_setup(int Mf, int Mc, double P[MAXM][MAXM], double R[MAXM][MAXM]);

// X (Mto x Mfrom): the nodal polynomial on the Mfrom Radau nodes evaluated
// at the Mto Radau nodes (value restriction / interpolation between node
// sets).  0 on success.
int node_eval_setup(int Mfrom, int Mto, double X[MAXM][MAXM]);

}  // namespace st
