// Learned SNSD initial guess (BF16 MLP): state and entry points (mlp.cu).
#pragma once

#include "relcp_internal.cuh"

namespace relcp {

struct MlpState {
    bool loaded = false;
    DBuf<double> guess;  // 3 x npairs start normals
};

relcp_status mlp_guess(MlpState& m, int64_t npairs, const int* pa, const int* pb, View<3, const double> x,
                       View<4, const double> q, View<3, const double> axes, const double box[3], cudaStream_t s);
void mlp_release(MlpState& m, cudaStream_t s);

}  // namespace relcp
