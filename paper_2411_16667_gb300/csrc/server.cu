// Continuous-batching server entry points (see include/opmos.h).
#include "opmos.h"

extern "C" {

int opmos_server_create(const opmos_graph* const*, uint32_t, const opmos_options*, opmos_server** out) {
  if (out) *out = nullptr;
  return OPMOS_ERR_INVALID_ARG;
}
int opmos_server_submit(opmos_server*, uint32_t, uint32_t, uint32_t, uint32_t, uint64_t*) {
  return OPMOS_ERR_INVALID_ARG;
}
int opmos_server_poll(opmos_server*, uint64_t, opmos_result** out) {
  if (out) *out = nullptr;
  return OPMOS_ERR_INVALID_ARG;
}
void opmos_server_destroy(opmos_server*) {}

}  // extern "C"
