// pending.cu -- entry points declared in ibm.h whose implementation is not
// built yet; each reports IBM_ERR_UNSUPPORTED.
#include "plan.h"
using namespace ibm;
extern "C" {
int ibm_batch_create(int, const int *, const double *, int, int, ibm_batch *) {
  return set_error(IBM_ERR_UNSUPPORTED, "ibm_batch_create: not built");
}
int ibm_batch_destroy(ibm_batch) { return set_error(IBM_ERR_UNSUPPORTED, "not built"); }
int ibm_batch_poisson(ibm_batch, const void *const *, void *const *, void *) {
  return set_error(IBM_ERR_UNSUPPORTED, "not built");
}
int ibm_server_create(size_t, int, int, ibm_server *) { return set_error(IBM_ERR_UNSUPPORTED, "not built"); }
int ibm_server_destroy(ibm_server) { return set_error(IBM_ERR_UNSUPPORTED, "not built"); }
int ibm_submit(ibm_server, const ibm_request *, uint64_t *) { return set_error(IBM_ERR_UNSUPPORTED, "not built"); }
int ibm_poll(ibm_server, uint64_t, ibm_result *) { return set_error(IBM_ERR_UNSUPPORTED, "not built"); }
int ibm_wait(ibm_server, uint64_t, double, ibm_result *) { return set_error(IBM_ERR_UNSUPPORTED, "not built"); }
int ibm_cancel(ibm_server, uint64_t) { return set_error(IBM_ERR_UNSUPPORTED, "not built"); }
}
