// server.cu -- continuous-batching restoration server (C ABI).
#include "plan.hpp"

using namespace eecmg;

extern "C" {

eecmg_status eecmg_server_create(size_t, int, eecmg_server_t* out) {
    if (out) *out = nullptr;
    return set_error(EECMG_ERR_UNSUPPORTED, "eecmg_server_create: server not available in this build");
}
eecmg_status eecmg_server_submit(eecmg_server_t, eecmg_plan_t, const float*, float*, uint64_t*) {
    return set_error(EECMG_ERR_UNSUPPORTED, "eecmg_server_submit: server not available in this build");
}
eecmg_status eecmg_server_poll(eecmg_server_t, uint64_t, int*, double*) {
    return set_error(EECMG_ERR_UNSUPPORTED, "eecmg_server_poll: server not available in this build");
}
eecmg_status eecmg_server_drain(eecmg_server_t) {
    return set_error(EECMG_ERR_UNSUPPORTED, "eecmg_server_drain: server not available in this build");
}
eecmg_status eecmg_server_destroy(eecmg_server_t) { return EECMG_OK; }

}  // extern "C"
