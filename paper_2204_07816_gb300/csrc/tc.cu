// Tensor-core (tcgen05) path: placeholder until the kernels land.
#include "internal.h"

namespace nqs {

bool tc_supported(const Problem &, std::string *why) { if (why) *why = "tensor-core path not built"; return false; }
size_t tc_packed_bytes(const Problem &) { return 16; }
int launch_tc_pack(const Problem &, const double *, void *, const LaunchEnv &env) {
    *env.msg = "tensor-core path not built";
    return NQS_ERR_UNSUPPORTED;
}
int launch_logpsi_tc(const Problem &, const double *, const void *, const int8_t *, int64_t, double *, const LaunchEnv &env) {
    *env.msg = "tensor-core path not built";
    return NQS_ERR_UNSUPPORTED;
}
int launch_eloc_tc(const Problem &, const double *, const void *, const int8_t *, const double *, int64_t, double *,
                   const LaunchEnv &env) {
    *env.msg = "tensor-core path not built";
    return NQS_ERR_UNSUPPORTED;
}
int launch_sample_tc(const Problem &, const double *, const void *, int8_t *, int, uint64_t, uint64_t, int, int, int,
                     int8_t *, double *, const LaunchEnv &env) {
    *env.msg = "tensor-core path not built";
    return NQS_ERR_UNSUPPORTED;
}

}  // namespace nqs
