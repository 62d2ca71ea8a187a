// k_tc.cu -- tcgen05 tensor-core MLP (placeholder until the kernel lands).
#include "nv_internal.cuh"

bool tc_supported(const NetDesc &) { return false; }

nv_status launch_mlp_tc_ext(const nv_ctx *, int, const MlpArgs &, const int *, int, int64_t, double *) {
  return nv_fail(NV_ERR_UNSUPPORTED, "tensor-core MLP not built");
}

nv_status launch_mlp_tc(const nv_ctx *c, int mode, const MlpArgs &a) {
  return launch_mlp_tc_ext(c, mode, a, nullptr, 1, a.n, nullptr);
}
