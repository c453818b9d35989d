// The Anderson small solve (pd_aa_solve.cuh) compiled as host C++: the
// unrolled forms for windows of 1 to 5 columns and the run-time form used
// above that, behind one C entry point for the CPU tests.
#define __device__
#define __forceinline__ inline
#include "../../paper_2605_14526_b300/csrc/pd_aa_solve.cuh"

using namespace pdk;

extern "C" {
int aa_max_window() { return kMaxAA; }

// G: [kMaxAA][kMaxAA] row-major (only the leading nc x nc block is read);
// any_form = 1 takes the run-time form for every nc
int aa_solve_host(int nc, int any_form, const double* G, const double* rhs, double* gam, double* gn) {
  bool ok = false;
  double g2 = 0.0;
  if (any_form || nc > 5) {
    ok = aa_solve_any(nc, G, rhs, gam, g2);
  } else {
    switch (nc) {
      case 1: ok = aa_solve<1>(G, rhs, gam, g2); break;
      case 2: ok = aa_solve<2>(G, rhs, gam, g2); break;
      case 3: ok = aa_solve<3>(G, rhs, gam, g2); break;
      case 4: ok = aa_solve<4>(G, rhs, gam, g2); break;
      default: ok = aa_solve<5>(G, rhs, gam, g2); break;
    }
  }
  *gn = g2;
  return ok ? 1 : 0;
}
}
