// Entry points whose subsystems are not built yet.
#include "mrn_internal.h"

extern "C" {
int mrn_server_create(const mrn_server_opts*, mrn_server**) { return MRN_EUNSUPPORTED; }
int mrn_server_submit(mrn_server*, const mrn_view*, const mrn_view*, uint64_t*) { return MRN_EUNSUPPORTED; }
int mrn_server_poll(mrn_server*, uint64_t, int*, int*) { return MRN_EUNSUPPORTED; }
int mrn_server_wait(mrn_server*, uint64_t, uint64_t, int*) { return MRN_EUNSUPPORTED; }
int mrn_server_stats_get(mrn_server*, mrn_server_stats*) { return MRN_EUNSUPPORTED; }
void mrn_server_destroy(mrn_server*) {}
}
