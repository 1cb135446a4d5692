// Learned SNSD initial guess: a 13 -> 128 -> 128 -> 128 -> 5 MLP (padded to
// 16 inputs and 8 outputs) evaluated and trained with BF16 tensor-core
// kernels (mma.sync m16n8k16, FP32 accumulation).  mlp.cu.
#pragma once

#include "relcp_internal.cuh"

namespace relcp {

constexpr int kMlpIn = RELCP_MLP_IN;
constexpr int kMlpHid = RELCP_MLP_HID;
constexpr int kMlpOut = RELCP_MLP_OUT;
constexpr int kMlpParams = RELCP_MLP_NPARAMS;

// parameter offsets in the FP32 parameter vector (row-major W[out][in])
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpHid * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpHid;
constexpr int kOffB2 = kOffW2 + kMlpHid * kMlpHid;
constexpr int kOffW3 = kOffB2 + kMlpHid;
constexpr int kOffB3 = kOffW3 + kMlpHid * kMlpHid;
constexpr int kOffW4 = kOffB3 + kMlpHid;
constexpr int kOffB4 = kOffW4 + kMlpOut * kMlpHid;
static_assert(kOffB4 + kMlpOut == kMlpParams, "parameter layout");

struct MlpState {
    bool loaded = false;
    DBuf<float> params;  // FP32 parameters
    DBuf<unsigned char> image;  // the forward kernel's shared-memory image of params (mlp_pack_launch)
    DBuf<double> guess;  // 3 x npairs start normals (world frame; zero = no guess)
};

// features (and optionally targets from SNSD outputs) of listed pairs
struct MlpFeatArgs {
    int64_t npairs;
    const int32_t* pa;
    const int32_t* pb;
    int64_t pstride;
    View<3, const double> x;
    View<4, const double> q;
    View<3, const double> axes;
    double box[3];
    const double* box_dev;  // if set, the box is read here (device) instead
    const double* snsd;  // null, or per-pair (phi, n[3], ...) with stride snsd_s between pairs
    int64_t snsd_s, snsd_c;  // pair stride and component stride of `snsd`
    float* feat;         // npairs x 16
    float* targets;      // npairs x 4 (n in a's frame, phi / scale) or null
    // optional subset: row k < *count_dev holds pair idx[k] (idx == nullptr: row p = pair p)
    const int* idx;
    const int* count_dev;
};
relcp_status mlp_features_launch(const MlpFeatArgs& a, cudaStream_t s);
// the forward kernel's packed network image (RELCP_MLP image bytes) from FP32 params
relcp_status mlp_pack_launch(const float* params, unsigned char* image, cudaStream_t s);
// rows: npairs, or *count_dev (<= npairs) when count_dev is given; a failed
// weight copy sets DEV_TIMEOUT in *status (may be null)
relcp_status mlp_forward_launch(int64_t npairs, const unsigned char* image, const float* feat, float* out,
                                cudaStream_t s, const int* count_dev = nullptr, int* status = nullptr);
size_t mlp_image_bytes();

relcp_status mlp_train_step(int64_t B, float* params, float* am, float* av, const float* feat, const float* targets,
                            const relcp_mlp_train_config& tc, float* grad_out, double* loss_out, cudaStream_t s);

// start normals guess(., k) for the pairs idx[k], k < *count_dev (idx == nullptr:
// all npairs pairs); npairs bounds the count
// min_count: with fewer rows (*count_dev) the network does not run and
// *ran (if given) is set to 0, else to 1; *declined (if given) counts the
// pairs whose start the network declined (trust logit <= 0: a cold start)
relcp_status mlp_guess(MlpState& m, int64_t npairs, const int* pa, const int* pb, View<3, const double> x,
                       View<4, const double> q, View<3, const double> axes, const double box[3], cudaStream_t s,
                       const int* idx = nullptr, const int* count_dev = nullptr, int* status = nullptr,
                       const double* box_dev = nullptr, int64_t min_count = 0, int* ran = nullptr,
                       int* declined = nullptr);
void mlp_release(MlpState& m, cudaStream_t s);

}  // namespace relcp
