// Request server (placeholder until the serving loop lands).
#include "sf_internal.h"

extern "C" {
int sf_server_create(int64_t, int, sf_server** out) {
  if (out) *out = nullptr;
  sf::set_error("server not built yet");
  return SF_EUNSUPPORTED;
}
int sf_server_submit(sf_server*, sf_plan*, const uint64_t*, int64_t, const sf_path_sel*, uint64_t*) {
  return SF_EUNSUPPORTED;
}
int sf_server_wait(sf_server*, uint64_t, int, double*) { return SF_EUNSUPPORTED; }
int sf_server_cancel(sf_server*, uint64_t) { return SF_EUNSUPPORTED; }
int sf_server_times(sf_server*, uint64_t, double*, double*) { return SF_EUNSUPPORTED; }
void sf_server_destroy(sf_server*) {}
}
