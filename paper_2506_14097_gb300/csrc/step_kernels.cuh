// Argument blocks of the per-body and per-row step kernels (step_kernels.cu).
// Every array is structure-of-arrays: component k of item i at base[k*n + i]
// (rows: base[k*cap + r]).
#pragma once

#include "relcp_internal.cuh"

namespace relcp {

struct PrepArgs {
    int64_t n;
    int dynamics;
    int shape;  // RELCP_SHAPE_*: the shape record written to P
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
    float* ufreef;  // FP32 mirror of U_free (mixed path) or null
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
    int planar;  // RELCP_OVERDAMPED_2D: rows keep their u_x, u_y, omega_z entries only
    double c, strain_rate;
    double box[3];
    const double* x;      // C^k positions (A_0 offsets)
    const double* ufree;  // A_0 offsets
    const double* uc;     // appended offsets: K D gamma of the last LCP
    const double* K;
    // mixed path (all three set): the row's torques, rate and diagonal in FP32
    // from FP32 mirrors of U_free and K; only Phi + c rate stays FP64
    const float* ufreef;
    const float* Kf;
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
    int* nrows0_dev;  // if set, also receives that count (|A_0|)
    unsigned long long* clear3;  // if set, three words zeroed (the per-level fields of the next trial)
    int* status;
    const double* box_dev;  // if set, the box is read here (device) instead of `box`
    // A_0 only: warm start per pair (null: 0) and the pair -> row map (-1: no row)
    const double* gamma0;
    int* rowof;
};

// C^k values of the pairs that were candidates in the previous step: the SNSD
// result of that step's last overlap test (same configuration) and the final
// gamma of the pair's A_0 row; need[p] = 1 for the pairs still to evaluate
struct ReuseArgs {
    int64_t npairs;         // capacity (SoA stride of s0, gamma0)
    const int* np_dev;      // number of pairs (device)
    const int* pv;          // pair -> cached-list entry
    const PairMemo* memo;   // per entry
    int stamp_prev;         // stamp of the previous step (no memo matches a negative stamp)
    const int* stamp_prev_dev;  // if set, read here (device) instead
    int reuse_snsd;
    int use_gamma;
    const double* sprev;    // previous step's last trial SNSD output, 10 x sprev_stride (SoA)
    int64_t sprev_stride;
    int64_t nprev;          // pairs of the previous step
    double* s0;             // SNSD output at C^k, 10 x npairs (SoA)
    int* it0;               // Newton iterations at C^k (0 for reused pairs)
    double* gamma0;         // per pair
    int* list;              // pairs to evaluate, in no particular order (each pair's result does not
                            // depend on its position in the list)
    int* count;             // their number (zeroed before the launch)
};

struct MemoSaveArgs {
    int64_t npairs;         // capacity
    const int* np_dev;      // number of pairs (device)
    const int* pv;
    const int* rowof;
    const double* gamma;    // FP64 path or null
    const float* gammaf;    // mixed path or null
    int stamp;
    PairMemo* memo;
};

struct TrialArgs {
    int64_t n;
    int shape;  // RELCP_SHAPE_*: the shape record written to Pt
    double dt;
    // optional look-ahead of the cached pair list (xb == nullptr: none): the
    // largest |min_image(x_t - sfac xb)| in box `la_box`, atomicMax of its bits
    const double* xb;
    double sfac[3], la_box[3];
    const double* sfac_dev;    // if set: sfac and la_box read here (device) instead
    const double* la_box_dev;
    unsigned long long* la_dmax;  // bits of the largest squared displacement (atomic max)
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
    // optional: the next step's prep on the accepted state, in the same pass
    // (next.n == 0: none)
    PrepArgs next;
    // overdamped, with K, Kf and rb computed for the current semi-axes and
    // config: the next prep keeps them, takes q as the trial normalised it
    // and P = Pt (the shape matrix of the accepted trial orientation), so
    // only U_free is recomputed
    int keep;
    const double* Pt;
    const double* xt;
    const double* qt;
    const double* ustep;
    double* x;
    double* q;
    double* vel;
};

relcp_status prep_launch(const PrepArgs& a, cudaStream_t s);
// flags[p] = (p < *np_dev && phi[p] <= thr) for p < cap (zeros past the count)
relcp_status flag_le_launch(int64_t cap, const int* np_dev, const double* phi, double thr, int* flags, cudaStream_t s);
relcp_status rows_launch(const RowsArgs& a, cudaStream_t s);
relcp_status trial_launch(const TrialArgs& a, cudaStream_t s);
relcp_status accept_launch(const AcceptArgs& a, cudaStream_t s);

// Body state in from a row-major staging block [x 3 | q 4 | axes 3 | vel 6 |
// fext 6] per body (22 doubles), transposed into the SoA arrays with x
// wrapped into the box.  With `compare`, *changed gets bit 0 if x, q, vel or
// fext differ (bitwise) from what the arrays held, bit 1 if the axes differ.
struct LoadArgs {
    int64_t n;
    const double* stage;
    double* x;
    double* q;
    double* axes;
    double* vel;
    double* fext;
    double box[3];
    int compare;
    int* changed;
};
relcp_status load_bodies_launch(const LoadArgs& a, cudaStream_t s);

// Body state read in place from the caller's row-major arrays (device memory,
// or host memory the device reaches through the host page tables): x n x 3,
// q n x 4, axes n x 3, vel / fext n x 6 (null: zeros).
struct BodyIn {
    const double* x;
    const double* q;
    const double* axes;
    const double* vel;
    const double* fext;
};
// validation and comparison, writing nothing to the state
struct BodyCheck {
    unsigned long long bad_key;  // min over invalid bodies of (index << 4 | reasons), all ones: none;
                                 // reasons 1: |q| not 1 within 1e-6, 2: position not finite,
                                 // 4: semi-axis not > 0 or not finite, 8: velocity / force not finite
    unsigned long long rbmax_bits;  // bits of the largest semi-axis
    int changed;                    // as LoadArgs::changed
    int pad;
};
struct CheckArgs {
    int64_t n;
    BodyIn in;
    const double* x;  // current SoA state (compared when `compare`)
    const double* q;
    const double* axes;
    const double* vel;
    const double* fext;
    double box[3];
    int compare;
    double* stage;  // the rows copied out as load_bodies_launch reads them (22 doubles per body)
    BodyCheck* out;
};
relcp_status check_bodies_launch(const CheckArgs& a, cudaStream_t s);
// x, q, vel (SoA) into the caller's row-major arrays (any may be null)
relcp_status store_direct_launch(int64_t n, const double* x, const double* q, const double* vel, double* ox,
                                 double* oq, double* ov, cudaStream_t s);
// x (3), q (4), vel (6) of every body into a row-major block (13 doubles per
// body; a null source is skipped and its columns are left unwritten)
relcp_status store_bodies_launch(int64_t n, const double* x, const double* q, const double* vel, double* out,
                                 cudaStream_t s);
relcp_status reuse_launch(const ReuseArgs& a, cudaStream_t s);
relcp_status memo_save_launch(const MemoSaveArgs& a, cudaStream_t s);

}  // namespace relcp
