// Sparse (CSR) operator support.
#include "lsrn_internal.h"

namespace lsrn {

lsrn_status csr_plan_setup(Plan* p, const lsrn_matrix* A, bool host) {
  (void)p;
  (void)A;
  (void)host;
  return LSRN_ERR_UNSUPPORTED;
}

}  // namespace lsrn
