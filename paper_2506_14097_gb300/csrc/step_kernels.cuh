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
    double* geom;  // 9 x cap
    double* q;
    double* diag;
    double* gamma;
    int* status;
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
relcp_status max_blocks_launch(int nblocks, const double* v, double* out, cudaStream_t s);
relcp_status iters_max_launch(int64_t np, const int* it, int* out, cudaStream_t s);
relcp_status wrap_launch(int64_t n, double* x, const double box[3], cudaStream_t s);

}  // namespace relcp
