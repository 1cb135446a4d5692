// Argument blocks of the per-body and per-row step kernels (step_kernels.cu).
// Every array is structure-of-arrays: component k of item i at base[k*n + i]
// (rows: base[k*cap + r]).
#pragma once

#include "relcp_internal.cuh"

namespace relcp {

struct PrepArgs {
    int64_t n;
    int dynamics;
    double dt, drag_xi, density, strain_rate;
    double box[3];
    const double* x;
    double* q;  // normalised in place
    const double* axes;
    const double* vel;
    const double* fext;
    double* P;
    double* K;
    float* Kf;  // FP32 mirror of K (mixed path)
    double* rb;
    double* ufree;
};

struct RowsArgs {
    int64_t npairs, nbodies;
    const int* pa;
    const int* pb;
    const int* flags;
    const int* scan;
    const double* snsd;  // 10 x npairs: phi, n, r_a, r_b
    int64_t base, cap;
    int rec_index;
    double c, strain_rate;
    double box[3];
    const double* x;      // C^k positions (A_0 offsets)
    const double* ufree;  // A_0 offsets
    const double* uc;     // appended offsets: K D gamma of the last LCP
    const double* K;
    int* ia;
    int* ib;
    int* rec;
    int* pair;
    double* geom;   // 9 x cap
    float* geomf;   // 9 x cap FP32 mirror (mixed path) or null
    double* q;
    float* qf;      // FP32 mirror of q (mixed path) or null
    double* diag;
    double* invd;   // 1 / A_aa (FP64 path) or null
    float* invdf;   // 1 / A_aa (mixed path) or null
    double* gamma;  // warm start of new rows set to 0 (FP64 path) or null
    float* gammaf;  // same for the mixed path or null
    int* nrows_dev; // set to base + number of flagged pairs
    int* status;
    // warm start of A_0 rows from the previous step's A_0 rows (sorted keys
    // (a << 32) | b with their final gamma); prev_n = 0 disables it
    int64_t prev_n;
    const long long* prev_keys;
    const double* prev_gamma;
};

struct SaveWarmArgs {
    const int* nrows0_dev;  // number of A_0 rows (device)
    const int* ia;
    const int* ib;
    const double* gamma;    // FP64 path or null
    const float* gammaf;    // mixed path or null
    long long* keys;
    double* gout;
};

struct TrialArgs {
    int64_t n;
    double dt;
    const double* x;
    const double* q;
    const double* axes;
    const double* ufree;
    const double* uc;
    double* xt;
    double* qt;
    double* Pt;
    double* ustep;
};

struct AcceptArgs {
    int64_t n;
    int inertial;
    double box[3];
    const double* xt;
    const double* qt;
    const double* ustep;
    double* x;
    double* q;
    double* vel;
};

relcp_status prep_launch(const PrepArgs& a, cudaStream_t s);
relcp_status flag_le_launch(int64_t np, const double* phi, double thr, int* flags, cudaStream_t s);
relcp_status rows_launch(const RowsArgs& a, cudaStream_t s);
relcp_status trial_launch(const TrialArgs& a, cudaStream_t s);
relcp_status accept_launch(const AcceptArgs& a, cudaStream_t s);
relcp_status wrap_launch(int64_t n, double* x, const double box[3], cudaStream_t s);
relcp_status save_warm_launch(const SaveWarmArgs& a, int64_t cap, cudaStream_t s);

}  // namespace relcp
