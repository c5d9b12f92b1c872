// tcgen05 tensor-core path (placeholder until the sm_103a kernels land).
#include "gp_internal.cuh"

namespace gp {

bool tc_available() { return false; }
size_t tc_points_bytes(int64_t, int) { return 0; }
int tc_prepare_points(const KP<float> &, const float *, int64_t, void *, TcPoints *, cudaStream_t) {
    set_error("tensor-core path not built");
    return GP_ERR_UNSUPPORTED;
}
size_t tc_mvm_workspace(int64_t, int64_t, int) { return 0; }
int tc_mvm(const TcMvmArgs &, void *, size_t, cudaStream_t) {
    set_error("tensor-core path not built");
    return GP_ERR_UNSUPPORTED;
}
size_t tc_grad_workspace(int64_t, int, int) { return 0; }
int tc_grad(const GradArgs<float> &, void *, size_t, cudaStream_t) {
    set_error("tensor-core path not built");
    return GP_ERR_UNSUPPORTED;
}

}  // namespace gp
