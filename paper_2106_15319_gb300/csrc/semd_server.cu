// Continuous-batching request server of the GB300 Serial-EMD library.
#include "semd_runtime.h"

extern "C" {

semd_status serial_emd_server_create(const semd_params *, size_t, int, semd_server_t *out)
{
    if (out)
        *out = nullptr;
    return SEMD_EUNSUPPORTED;
}

semd_status serial_emd_submit(semd_server_t, const semd_request *, uint64_t *)
{
    return SEMD_EUNSUPPORTED;
}

semd_status serial_emd_poll(semd_server_t, uint64_t, semd_result *) { return SEMD_EUNSUPPORTED; }

void serial_emd_server_destroy(semd_server_t) {}

const char *serial_emd_server_last_error(semd_server_t) { return "server not built"; }

} // extern "C"
