// Drives the host-side collocation setup (st_setup.cpp) for every node count
// and every pair of node sets, for a build with AddressSanitizer and
// UndefinedBehaviorSanitizer.  Exits 0 when every call succeeds and the
// results satisfy identities that hold exactly in real arithmetic: the rows
// of Q sum to the nodes (Q integrates constants), the node-set restriction
// is a left inverse of the prolongation, and the value map between equal
// node sets is the identity.
#include <cmath>
#include <cstdio>

#include "st_setup.h"

int main() {
  int bad = 0;
  for (int M = 1; M <= ST_MAX_M; ++M) {
    st::Colloc c;
    if (st::colloc_setup(M, &c) != 0) {
      std::printf("colloc_setup(%d) failed\n", M);
      ++bad;
      continue;
    }
    for (int i = 0; i < M; ++i) {
      double row = 0.0;
      for (int j = 0; j < M; ++j) row += c.Q[i][j];
      if (std::fabs(row - c.tau[i]) > 1e-13) {
        std::printf("M=%d row %d of Q sums to %.17g, node %.17g\n", M, i, row, c.tau[i]);
        ++bad;
      }
    }
  }
  for (int Mf = 1; Mf <= ST_MAX_M; ++Mf)
    for (int Mc = 1; Mc <= Mf; ++Mc) {
      double P[MAXM][MAXM] = {}, R[MAXM][MAXM] = {}, X[MAXM][MAXM] = {};
      if (st::node_transfer_setup(Mf, Mc, P, R) != 0 || st::node_eval_setup(Mf, Mc, X) != 0) {
        std::printf("node transfers %d -> %d failed\n", Mf, Mc);
        ++bad;
        continue;
      }
      for (int a = 0; a < Mc; ++a)
        for (int b = 0; b < Mc; ++b) {
          double rp = 0.0;
          for (int k = 0; k < Mf; ++k) rp += R[a][k] * P[k][b];
          if (std::fabs(rp - (a == b ? 1.0 : 0.0)) > 1e-11) {
            std::printf("(R P)[%d][%d] = %.17g for %d -> %d\n", a, b, rp, Mf, Mc);
            ++bad;
          }
          if (Mf == Mc && std::fabs(X[a][b] - (a == b ? 1.0 : 0.0)) > 1e-13) {
            std::printf("value map %d -> %d not the identity\n", Mf, Mc);
            ++bad;
          }
        }
    }
  std::printf(bad ? "FAILED %d\n" : "ok\n", bad);
  return bad ? 1 : 0;
}
