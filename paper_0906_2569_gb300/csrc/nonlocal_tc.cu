// Nonlocal contractions of the mixed-precision path.
#include <cuda_runtime.h>

#include "hpsi_internal.h"

namespace hpsi {

int mixed_prepare_beta(Context& c, Problem& p) {
  (void)c;
  (void)p;
  return HPSI_OK;
}

int nonlocal_apply_mixed(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd) {
  return nonlocal_apply_fp64(c, p, psi, hpsi, nbnd);
}

}  // namespace hpsi
