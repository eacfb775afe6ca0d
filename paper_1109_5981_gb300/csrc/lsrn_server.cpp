// Serving front end (request queue with admission by device-memory budget).
#include "lsrn.h"

extern "C" {

lsrn_status lsrn_server_create(size_t hbm_budget_bytes, int32_t max_slots, lsrn_server_t* out) {
  (void)hbm_budget_bytes;
  (void)max_slots;
  if (out) *out = nullptr;
  return LSRN_ERR_UNSUPPORTED;
}
lsrn_status lsrn_submit(lsrn_server_t s, const lsrn_matrix* A, const double* b,
                        const lsrn_options* opt, int32_t solver, uint64_t* ticket) {
  (void)s; (void)A; (void)b; (void)opt; (void)solver; (void)ticket;
  return LSRN_ERR_UNSUPPORTED;
}
lsrn_status lsrn_poll(lsrn_server_t s, uint64_t ticket, double* x_out, lsrn_info* info) {
  (void)s; (void)ticket; (void)x_out; (void)info;
  return LSRN_ERR_UNSUPPORTED;
}
lsrn_status lsrn_server_destroy(lsrn_server_t s) {
  (void)s;
  return LSRN_OK;
}

}  // extern "C"
