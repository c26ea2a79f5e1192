// Temporary launchers for paths still being written.
#include "kernels.h"

namespace wrf {

size_t deform_bwd_ws_layout(int n, int Q, const MlpView &m, DeformWs *fw, DeformBwdWs *bw,
                            char *base) {
    size_t s = deform_ws_layout(n, Q, m.n_layers, fw, base);
    if (bw) *bw = DeformBwdWs{};
    return s;
}

cudaError_t launch_mlp_bwd(const SceneView &, const MlpView &, const GridView &, int,
                           const DeformWs &, const DeformBwdWs &, const float *, float *const *,
                           float *const *, float *, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace wrf
