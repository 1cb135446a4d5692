#include "mlp.cuh"

namespace relcp {

relcp_status mlp_guess(MlpState& m, int64_t, const int*, const int*, View<3, const double>, View<4, const double>,
                       View<3, const double>, const double*, cudaStream_t) {
    (void)m;
    set_error("learned guess not loaded");
    return RELCP_ERR_STATE;
}

void mlp_release(MlpState& m, cudaStream_t s) { m.guess.release(s); }

}  // namespace relcp
