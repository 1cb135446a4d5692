// C ABI of the ReLCP library: context lifecycle, the time step of Algorithm 1
// and the stateless per-step entry points.  See include/relcp.h.
//
// One step (Algorithm 1; inertial variant Eq. relcp_inertial):
//   prep -> broad phase -> SNSD at C^k -> A_0 = {Phi <= phi_skin} ->
//   loop { LCP (persistent BB projected gradient) -> trial C_{n+1} ->
//          SNSD at C_{n+1} (warm-started from the C^k normals) + FP64 overlap
//          test -> stop if no pair has Phi < -eps_NCP (Eq. gap_stopping_rule)
//          -> append one frozen-normal, pulled-back row per violating pair }
//   -> accept C^{k+1}.
// The host reads three counts per recursion (pairs, rows, violators) to size
// buffers and decide the loop; everything else stays on the device.
#include <atomic>
#include <chrono>
#include <cmath>
#include <climits>
#include <functional>
#include <cstdarg>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "relcp_internal.cuh"
#include "step_kernels.cuh"
#include "mlp.cuh"

namespace relcp {

static thread_local char g_err[1024] = "";
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

relcp_status status_from_device(int bits) {
    if (bits & DEV_TIMEOUT) return RELCP_ERR_TIMEOUT;
    if (bits & DEV_CAPACITY) return RELCP_ERR_CAPACITY;
    if (bits & DEV_NEWTON) return RELCP_ERR_NEWTON;
    if (bits & DEV_LCP_NOT_CONVERGED) return RELCP_ERR_NOT_CONVERGED;
    return RELCP_OK;
}

int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

// FP64 -> FP32 and back, element by element (the stateless LCP call's
// one-time conversions)
__global__ void narrow_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
__global__ void widen_kernel(const float* __restrict__ in, double* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}
static unsigned conv_blocks(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}
relcp_status narrow_launch(const double* in, float* out, int64_t n, cudaStream_t s) {
    note_launch();
    narrow_kernel<<<conv_blocks(n), 256, 0, s>>>(in, out, n);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}
relcp_status widen_launch(const float* in, double* out, int64_t n, cudaStream_t s) {
    note_launch();
    widen_kernel<<<conv_blocks(n), 256, 0, s>>>(in, out, n);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

}  // namespace relcp

using namespace relcp;

// Device-side scalars of one step, read by the host in one copy at each
// recursion decision.
struct DevStep {
    int nrows;          // rows currently in the LCP (set by the row kernel)
    int status;         // DEV_* bits
    int newton_max;     // largest Newton iteration count
    int nrows0;         // |A_0| (copied from nrows after the first LCP)
    unsigned long long iters0;      // Newton iterations summed over the pairs at C^k
    LcpDevResult lcp;   // iterations and residual of the last LCP
    int c0_evals;       // pairs evaluated at C^k (the others reused the previous step's values)
    int np;             // candidate pairs of the step
    int guess_on;       // the learned start seeded this step's C^k evaluation
    int declined;       // pairs whose learned start the network declined (cold start)
    // per recursion level (cleared together before each trial)
    unsigned long long maxov_bits;  // bits of the largest overlap at the last trial
    unsigned long long la_dmax;     // bits of the largest squared displacement of the trial positions since the list build
    int nviol;                      // violators of the last overlap test
    int pad;
};

// the per-step scalars and the step's device-side counters in one block, so
// that the start of a step uploads both with one copy (the DevStep half of
// the pinned upload image stays zero)
struct StepBlock {
    StepConst k;
    DevStep d;
};

// a captured first level of a step (see step_once)
struct StepGraph {
    std::vector<uintptr_t> key;
    bool uncapturable = false;
    cudaGraphExec_t pre = nullptr, post = nullptr;  // before and after the LCP launch
    long long nkernels = 0;
};

struct relcp_ctx {
    relcp_config cfg{};
    cudaStream_t s = nullptr;
    int64_t n = 0;
    bool has_bodies = false;
    double box[3] = {0, 0, 0};
    double rb_max = 0.0;
    // body state and per-step body arrays (SoA)
    DBuf<double> x, q, axes, vel, fext, P, K, rb, ufree, uc, ustep, xt, qt, Pt;
    // pairs
    DBuf<int> pa, pb;
    int64_t npairs = 0;
    DBuf<double> s0, s1;  // SNSD outputs at C^k and at the trial (10 x npairs)
    DBuf<int> it0, it1, flags, fscan;
    DBuf<StepBlock> sblk;      // StepConst + DevStep on the device
    StepBlock* hup = nullptr;  // pinned upload image (DevStep half zero)
    DevStep* hstep = nullptr;  // pinned host copy (asynchronous readback)
    // rows (capacity rcap, SoA)
    int64_t nrows = 0, nrows0 = 0, rcap = 0;
    DBuf<int> r_ia, r_ib, r_rec, r_pair;
    DBuf<double> r_geom, r_q, r_diag, r_gamma, r_invd;
    DBuf<float> r_geomf, r_gammaf, r_qf, Kf, r_invdf, ufreef;
    BroadphaseScratch bp;
    LcpScratch lcp;
    ScanScratch scan;
    MlpState mlp;
    relcp_step_stats stats{};
    int64_t steps_done = 0;
    std::vector<cudaEvent_t> events;  // phase-timing event pool
    // carried between steps: the last overlap test's SNSD output at the
    // accepted configuration (= the next C^k) and the per-pair memo of the
    // cached candidate list (bp.memo), stamped with the step number
    DBuf<double> s1prev;
    int64_t nprev = 0, sprev_stride = 0;
    // the previous step checked the cached pair list against the positions it
    // accepted (= this step's C^k): la_ok says the check is current, la_rebuild
    // whether the list must be rebuilt; with la_ok && !la_rebuild the broad
    // phase needs no host round trip
    bool la_ok = false, la_rebuild = true;
    bool prepped = false;  // the last accept pass also ran the next step's prep
    double* hstage = nullptr;  // pinned staging of the body state (relcp_set_bodies / relcp_get_bodies)
    size_t hstage_cap = 0;
    DBuf<double> dstage;       // its device counterpart
    bool pageable_ok = false;  // the device reads / writes pageable host memory (host page tables)
    DBuf<BodyCheck> dcheck;    // relcp_set_bodies' validation result
    BodyCheck* hcheck = nullptr;  // pinned
    std::vector<StepGraph> graphs;
    int stamp = 0;         // stamp written by the last completed step
    bool memo_ok = false;  // memo and s1prev describe the current state
    bool snsd_ok = false;  // s1prev may stand in for the SNSD at C^k
    DBuf<double> gamma0;   // per pair: warm start of its A_0 row
    DBuf<int> idx, rowof;  // pairs to evaluate at C^k (unordered); pair -> A_0 row
};

namespace {

relcp_status check_config(const relcp_config* c) {
    if (!c) return set_error("config is NULL"), RELCP_ERR_INVALID_ARG;
    if (c->dynamics != RELCP_INERTIAL && c->dynamics != RELCP_OVERDAMPED && c->dynamics != RELCP_OVERDAMPED_2D)
        return set_error("dynamics must be RELCP_INERTIAL, RELCP_OVERDAMPED or RELCP_OVERDAMPED_2D"),
               RELCP_ERR_INVALID_ARG;
    if (c->precision != RELCP_FP64 && c->precision != RELCP_MIXED)
        return set_error("precision must be RELCP_FP64 or RELCP_MIXED"), RELCP_ERR_INVALID_ARG;
    if (c->guess != RELCP_GUESS_COLD && c->guess != RELCP_GUESS_MLP)
        return set_error("guess must be RELCP_GUESS_COLD or RELCP_GUESS_MLP"), RELCP_ERR_INVALID_ARG;
    if (!(c->dt > 0) || !(c->eps_ncp > 0) || !(c->skin >= 0) || !(c->lcp_tol > 0) || c->lcp_max_iter < 1 ||
        c->max_recursion < 0 || c->max_recursion > 4096)
        return set_error("dt, eps_ncp, lcp_tol > 0; skin >= 0; lcp_max_iter >= 1; 0 <= max_recursion <= 4096"),
               RELCP_ERR_INVALID_ARG;
    if (c->shape != RELCP_SHAPE_ELLIPSOID && c->shape != RELCP_SHAPE_SPHEROCYLINDER)
        return set_error("shape must be RELCP_SHAPE_ELLIPSOID or RELCP_SHAPE_SPHEROCYLINDER"), RELCP_ERR_INVALID_ARG;
    if (c->shape == RELCP_SHAPE_SPHEROCYLINDER && c->dynamics == RELCP_INERTIAL)
        return set_error("spherocylinders are stepped with the overdamped laws only"), RELCP_ERR_INVALID_ARG;
    if (c->dynamics != RELCP_INERTIAL && !(c->drag_xi > 0))
        return set_error("drag_xi must be > 0"), RELCP_ERR_INVALID_ARG;
    if (c->dynamics == RELCP_INERTIAL && !(c->density > 0))
        return set_error("density must be > 0"), RELCP_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (!(c->box[k] >= 0)) return set_error("box sides must be >= 0"), RELCP_ERR_INVALID_ARG;
    if (c->strain_rate != 0.0) {
        if (c->dynamics != RELCP_OVERDAMPED || !(c->box[0] > 0 && c->box[1] > 0 && c->box[2] > 0))
            return set_error("strain_rate needs overdamped dynamics and a fully periodic box"), RELCP_ERR_INVALID_ARG;
    }
    if (c->n_scenes != 1 && c->n_scenes != 0)
        return set_error("n_scenes must be 1 (use relcp_batched_* for many scenes)"), RELCP_ERR_INVALID_ARG;
    return RELCP_OK;
}

template <class T>
relcp_status move_rows(DBuf<T>& dst, DBuf<T>& src, int comps, int64_t nc, int64_t oldcap, int64_t m, cudaStream_t s) {
    DBuf<T> nb;
    RELCP_TRY(nb.ensure((size_t)(comps * nc), s));
    if (m > 0 && src.p)
        for (int k = 0; k < comps; ++k)
            RELCP_CUDA(cudaMemcpyAsync(nb.p + k * nc, src.p + k * oldcap, m * sizeof(T), cudaMemcpyDeviceToDevice, s));
    src.release(s);
    dst = nb;
    return RELCP_OK;
}

// grow the row buffers to hold `need` rows, keeping the first c->nrows
relcp_status grow_rows(relcp_ctx* c, int64_t need) {
    const bool mixed = c->cfg.precision == RELCP_MIXED;
    if (need <= c->rcap && (!mixed || c->r_geomf.p)) return RELCP_OK;
    int64_t nc = need > c->rcap ? need + need / 2 + 64 : c->rcap;
    cudaStream_t s = c->s;
    const int64_t m = c->nrows, oc = c->rcap;
    RELCP_TRY(move_rows(c->r_ia, c->r_ia, 1, nc, oc, m, s));
    RELCP_TRY(move_rows(c->r_ib, c->r_ib, 1, nc, oc, m, s));
    RELCP_TRY(move_rows(c->r_rec, c->r_rec, 1, nc, oc, m, s));
    RELCP_TRY(move_rows(c->r_pair, c->r_pair, 1, nc, oc, m, s));
    RELCP_TRY(move_rows(c->r_geom, c->r_geom, 9, nc, oc, m, s));
    RELCP_TRY(move_rows(c->r_q, c->r_q, 1, nc, oc, m, s));
    RELCP_TRY(move_rows(c->r_diag, c->r_diag, 1, nc, oc, m, s));
    RELCP_TRY(move_rows(c->r_gamma, c->r_gamma, 1, nc, oc, m, s));
    RELCP_TRY(move_rows(c->r_invd, c->r_invd, 1, nc, oc, m, s));
    if (mixed) {
        RELCP_TRY(move_rows(c->r_invdf, c->r_invdf, 1, nc, oc, m, s));
        RELCP_TRY(move_rows(c->r_geomf, c->r_geomf, 9, nc, oc, m, s));
        RELCP_TRY(move_rows(c->r_gammaf, c->r_gammaf, 1, nc, oc, m, s));
        RELCP_TRY(move_rows(c->r_qf, c->r_qf, 1, nc, oc, m, s));
    }
    c->rcap = nc;
    return RELCP_OK;
}

// CUDA events of the optional per-phase timing, recorded on the context
// stream and read only after a stream synchronisation.  Events come from a
// per-context pool, created once.
// CUDA-event timing of a step: per-phase marks (RELCP_FLAG_PHASE_TIMING) and/or
// events around the LCP kernel launches only (take(), also with
// RELCP_FLAG_LCP_TIMING)
struct PhaseTimer {
    std::vector<cudaEvent_t>* pool = nullptr;
    bool on = false;       // per-phase marks
    bool kernels = false;  // kernel events (take)
    cudaStream_t s{};
    int k = 0;
    relcp_status start(bool phases, bool lcp_only, cudaStream_t st, std::vector<cudaEvent_t>* p) {
        on = phases;
        kernels = phases || lcp_only;
        s = st;
        k = 0;
        pool = p;
        return RELCP_OK;
    }
    cudaEvent_t next() {
        if (k >= (int)pool->size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool->push_back(e);
        }
        return (*pool)[k];
    }
    int mark() {
        if (!on) return -1;
        cudaEvent_t e = next();
        if (!e) return -1;
        cudaEventRecord(e, s);
        return k++;
    }
    // both events must have completed (call after a stream synchronisation)
    float ms(int a, int b) {
        float t = 0.f;
        if (kernels && a >= 0 && b >= 0) cudaEventElapsedTime(&t, (*pool)[a], (*pool)[b]);
        return t;
    }
    // an unrecorded event for a callee to record (index returned in *idx)
    cudaEvent_t take(int* idx) {
        *idx = -1;
        if (!kernels) return nullptr;
        cudaEvent_t e = next();
        if (!e) return nullptr;
        *idx = k;
        ++k;
        return e;
    }
    void stop() { on = kernels = false; }
};

// Key of a captured step graph: everything the level-0 launches depend on
// (buffer addresses, capacities, modes).  A step whose key was seen before runs
// the graph of that key; the second sighting captures it.
static void step_key(relcp_ctx* c, int64_t PC, std::vector<uintptr_t>& key) {
    key.clear();
    auto add = [&](const void* p) { key.push_back((uintptr_t)p); };
    key.push_back((uintptr_t)PC);
    key.push_back((uintptr_t)c->n);
    key.push_back((uintptr_t)c->rcap);
    key.push_back((uintptr_t)c->sprev_stride);
    key.push_back((uintptr_t)(c->memo_ok ? 1 : 0) | (uintptr_t)(c->snsd_ok ? 2 : 0) | (uintptr_t)(c->mlp.loaded ? 4 : 0));
    const void* ptrs[] = {c->x.p, c->q.p, c->axes.p, c->vel.p, c->fext.p, c->P.p, c->K.p, c->Kf.p, c->ufreef.p, c->rb.p,
                          c->ufree.p, c->uc.p, c->ustep.p, c->xt.p, c->qt.p, c->Pt.p, c->s0.p, c->s1.p, c->s1prev.p,
                          c->it0.p, c->it1.p, c->flags.p, c->fscan.p, c->gamma0.p, c->idx.p, c->rowof.p, c->pa.p,
                          c->pb.p, c->bp.pv.p, c->bp.memo.p, c->bp.vpa.p, c->bp.vpb.p, c->bp.vflag.p, c->bp.vscan.p,
                          c->bp.xb.p, c->r_ia.p, c->r_ib.p, c->r_rec.p, c->r_pair.p, c->r_geom.p, c->r_geomf.p,
                          c->r_q.p, c->r_qf.p, c->r_diag.p, c->r_gamma.p, c->r_gammaf.p, c->r_invd.p, c->r_invdf.p,
                          c->lcp.inc_count.p, c->lcp.inc_off.p, c->lcp.inc_tmp.p, c->lcp.inc.p, c->lcp.packf.p,
                          c->lcp.packd.p, c->lcp.partials.p, c->scan.tiles.p, c->scan.ctr.p, c->bp.scan.tiles.p,
                          c->bp.scan.ctr.p, c->lcp.scan.tiles.p, c->lcp.scan.ctr.p, c->mlp.image.p, c->mlp.guess.p,
                          c->sblk.p, c->hstep, c->hup};
    for (const void* q : ptrs) add(q);
    for (size_t k = 0; k < 2 && k < c->events.size(); ++k) add(c->events[k]);
}

static void destroy_graph(StepGraph& g) {
    if (g.pre) cudaGraphExecDestroy(g.pre);
    if (g.post) cudaGraphExecDestroy(g.post);
    g.pre = g.post = nullptr;
}

void drop_graphs(relcp_ctx* c) {
    for (auto& g : c->graphs) destroy_graph(g);
    c->graphs.clear();
}

// The learned SNSD start runs on a step only when at least this many pairs are
// evaluated at C^k.  With the previous step's values carried over, a step
// typically evaluates tens of new pairs (a few thousand at most on the
// compaction), and for those the network's fixed latency (one tile through
// three 128-wide layers, about 10 us) exceeds the Newton iterations it saves
// (the cold seeds converge in at most four); they take the cold seeds, with
// the same converged result.  Such steps do not launch the network at all.
constexpr int64_t kLearnedMinPairs = 4096;

relcp_status step_once(relcp_ctx* c) {
    const auto h0 = std::chrono::steady_clock::now();
    double wait_ms = 0.0;
    cudaStream_t s = c->s;
    const relcp_config& cfg = c->cfg;
    const int64_t n = c->n;
    relcp_step_stats st{};
    st.n_bodies = n;
    const double dt = cfg.dt;
    double box0[3], box1[3];
    for (int k = 0; k < 3; ++k) {
        box0[k] = c->box[k];
        box1[k] = box0[k] > 0 ? box0[k] * (1.0 + cfg.strain_rate * dt) : 0.0;
    }
    const bool mixed = cfg.precision == RELCP_MIXED;
    PhaseTimer tm;
    RELCP_TRY(tm.start((cfg.flags & RELCP_FLAG_PHASE_TIMING) != 0, (cfg.flags & RELCP_FLAG_LCP_TIMING) != 0, s,
                       &c->events));
    std::vector<std::pair<int, int>> snsd_marks, lcp_marks, lcpk_marks;
    DevStep* ds = &c->sblk.p->d;
    const bool memo_ok = c->memo_ok;
    const bool prepped = c->prepped;

    // per-step scalars, read by the kernels from device memory
    StepConst& sk = c->hup->k;
    for (int k = 0; k < 3; ++k) {
        sk.box0[k] = box0[k];
        sk.box1[k] = box1[k];
    }
    if (!broadphase_lookahead_params(c->bp, n, box1, sk.sfac))
        for (int k = 0; k < 3; ++k) sk.sfac[k] = 1.0;
    sk.stamp_prev = memo_ok ? c->stamp : -1;
    sk.pad = 0;
    const double* box0_dev = c->sblk.p->k.box0;
    const double* box1_dev = c->sblk.p->k.box1;

    // bodies: normalised q, P, K, rb, U_free
    PrepArgs pa{};
    pa.n = n;
    pa.dynamics = cfg.dynamics;
    pa.shape = cfg.shape;
    pa.dt = dt;
    pa.drag_xi = cfg.drag_xi;
    pa.density = cfg.density;
    pa.strain_rate = cfg.strain_rate;
    for (int k = 0; k < 3; ++k) pa.box[k] = box0[k];
    pa.x = c->x.p;
    pa.q = c->q.p;
    pa.axes = c->axes.p;
    pa.vel = c->vel.p;
    pa.fext = c->fext.p;
    pa.P = c->P.p;
    pa.K = c->K.p;
    pa.Kf = nullptr;
    pa.ufreef = nullptr;
    if (mixed) {
        RELCP_TRY(c->Kf.ensure((size_t)(7 * (n > 0 ? n : 1)), s));
        RELCP_TRY(c->ufreef.ensure((size_t)(6 * (n > 0 ? n : 1)), s));
        pa.Kf = c->Kf.p;
        pa.ufreef = c->ufreef.p;
    }
    pa.rb = c->rb.p;
    pa.ufree = c->ufree.p;
    c->prepped = false;
    if (cfg.fault_inject & RELCP_FAULT_ROW_CAPACITY) {
        set_error("row capacity exhausted (injected fault)");
        tm.stop();
        return RELCP_ERR_CAPACITY;
    }

    // broad phase.  When the previous step's look-ahead showed the cached list
    // complete for these positions, the exact filter and compaction run with
    // the pair count left on the device (and the whole first level of the
    // step can be a replayed CUDA graph); otherwise the synchronous path
    // checks the bound and rebuilds the list if needed.  Per-pair work runs
    // over the list's capacity PC (also the SoA stride of pair arrays) and
    // stops at the device count.
    View<3, const double> xv = View<3, const double>::soa(c->x.p, n);
    const int rebuilds_before = c->bp.rebuilds;
    const bool fast_bp = c->la_ok && !c->la_rebuild && n >= 2 &&
                         verlet_bound_holds(c->bp, n, box0, c->rb_max, cfg.skin, 0.0);
    c->la_ok = false;  // set again when this step completes
    int t_begin = -1, t_bp = -1;
    // every buffer of the step sized before any launch (nothing allocates
    // inside a captured region)
    auto reserve = [&](int64_t PC) -> relcp_status {
        const int64_t npa = PC > 0 ? PC : 1;
        RELCP_TRY(c->s0.ensure(10 * npa, s));
        RELCP_TRY(c->s1.ensure(10 * npa, s));
        RELCP_TRY(c->it0.ensure(npa, s));
        RELCP_TRY(c->it1.ensure(npa, s));
        RELCP_TRY(c->flags.ensure(npa, s));
        RELCP_TRY(c->fscan.ensure(npa + 1, s));
        RELCP_TRY(c->gamma0.ensure(npa, s));
        RELCP_TRY(c->idx.ensure(npa, s));
        RELCP_TRY(c->rowof.ensure(npa, s));
        c->nrows = 0;
        RELCP_TRY(grow_rows(c, npa));
        if (cfg.guess == RELCP_GUESS_MLP && c->mlp.loaded) RELCP_TRY(c->mlp.guess.ensure((size_t)(3 * npa), s));
        RELCP_TRY(lcp_reserve(c->lcp, npa, n, mixed, s));
        RELCP_TRY(scan_reserve(c->scan, npa, s));
        RELCP_TRY(scan_reserve(c->bp.scan, c->bp.vn > 0 ? c->bp.vn : 1, s));
        RELCP_TRY(scan_reserve_tiles(c->bp.scan, broadphase_filter_tiles(c->bp.vn > 0 ? c->bp.vn : 1), s));
        return RELCP_OK;
    };
    auto head = [&]() -> relcp_status {
        // StepConst and a zeroed DevStep in one copy
        RELCP_CUDA(cudaMemcpyAsync(c->sblk.p, c->hup, sizeof(StepBlock), cudaMemcpyHostToDevice, s));
        if (!prepped) RELCP_TRY(prep_launch(pa, s));
        return RELCP_OK;
    };
    int64_t PC = 0;
    if (fast_bp) {
        PC = c->bp.vn;
        RELCP_TRY(reserve(PC));
    } else {
        t_begin = tm.mark();
        RELCP_TRY(head());
        int64_t np_host = 0;
        RELCP_TRY(broadphase_cached(n, c->x.p, c->rb.p, c->rb_max, box0, cfg.skin, c->pa, c->pb, &np_host, c->bp, s));
        PC = (n >= 2) ? c->bp.vn : 0;
        RELCP_TRY(reserve(PC));
        t_bp = tm.mark();
    }
    st.pair_list_rebuilt = c->bp.rebuilds != rebuilds_before;
    const int* npd = PC > 0 ? c->bp.vscan.p + PC : nullptr;  // device pair count
    const int64_t np = PC;  // grid sizes and strides of the per-pair work

    auto snsd_out = [&](DBuf<double>& o, DBuf<int>& it) {
        SnsdOut so;
        so.phi = o.p;
        so.phi_s = 1;
        so.n = View<3, double>::soa(o.p + np, np);
        so.ra = View<3, double>::soa(o.p + 4 * np, np);
        so.rb = View<3, double>::soa(o.p + 7 * np, np);
        so.iters = it.p;
        return so;
    };

    // C^k values a pair keeps from the previous step (the SNSD of its last
    // overlap test, evaluated at this very configuration, and the final gamma
    // of its A_0 row); idx lists the pairs still to evaluate
    c->memo_ok = false;  // set again once this step has saved its memo
    const int* count_dev = &ds->c0_evals;
    ReuseArgs ru{};
    ru.npairs = np;
    ru.np_dev = npd;
    ru.pv = c->bp.pv.p;
    ru.memo = c->bp.memo.p;
    ru.stamp_prev = sk.stamp_prev;
    ru.stamp_prev_dev = &c->sblk.p->k.stamp_prev;
    ru.reuse_snsd = c->snsd_ok && !(cfg.flags & RELCP_FLAG_NO_SNSD_REUSE);
    ru.use_gamma = !(cfg.flags & RELCP_FLAG_NO_WARM_START);
    ru.sprev = c->s1prev.p;
    ru.sprev_stride = c->sprev_stride;
    ru.nprev = c->nprev;
    ru.s0 = c->s0.p;
    ru.it0 = c->it0.p;
    ru.gamma0 = c->gamma0.p;
    ru.list = c->idx.p;
    ru.count = &ds->c0_evals;  // zeroed with the rest of DevStep at the start of the step

    // SNSD at C^k for the listed pairs
    // (spherocylinder pairs are closed-form: no Newton start to learn)
    const bool learned = cfg.guess == RELCP_GUESS_MLP && c->mlp.loaded && np > 0 && cfg.shape == RELCP_SHAPE_ELLIPSOID;
    SnsdArgs sa{};
    sa.shape = cfg.shape;
    sa.npairs = np;
    sa.pa = c->pa.p;
    sa.pb = c->pb.p;
    sa.pstride = 1;
    sa.x = xv;
    sa.P = View<6, const double>::soa(c->P.p, n);
    for (int k = 0; k < 3; ++k) sa.box[k] = box0[k];
    sa.box_dev = box0_dev;
    sa.guess.c[0] = sa.guess.c[1] = sa.guess.c[2] = nullptr;
    sa.guess.s = 1;
    sa.idx = c->idx.p;
    sa.count_dev = count_dev;
    if (learned) {
        sa.guess = View<3, const double>::soa(c->mlp.guess.p, np);
        sa.guess_on = &ds->guess_on;
    }
    sa.mixed = mixed ? 1 : 0;
    sa.newton_cap = (cfg.fault_inject & RELCP_FAULT_NEWTON_ITERS) ? 1 : 0;
    sa.out = snsd_out(c->s0, c->it0);
    sa.eps = 0.0;
    sa.viol = nullptr;
    sa.maxov_bits = nullptr;
    sa.newton_max = &ds->newton_max;
    sa.iters_sum = &ds->iters0;
    sa.status = &ds->status;

    // A_0: rows for the pairs with Phi(C^k) <= phi_skin
    RowsArgs ra{};
    ra.npairs = np;
    ra.nbodies = n;
    ra.pa = c->pa.p;
    ra.pb = c->pb.p;
    ra.flags = c->flags.p;
    ra.scan = c->fscan.p;
    ra.snsd = c->s0.p;
    ra.base = 0;
    ra.rec_index = 0;
    ra.c = dt;
    ra.planar = cfg.dynamics == RELCP_OVERDAMPED_2D;
    ra.strain_rate = cfg.strain_rate;
    for (int k = 0; k < 3; ++k) ra.box[k] = box0[k];
    ra.box_dev = box0_dev;
    ra.x = c->x.p;
    ra.ufree = c->ufree.p;
    ra.ufreef = pa.ufreef;
    ra.Kf = pa.Kf;
    ra.uc = c->uc.p;
    ra.K = c->K.p;
    ra.nrows_dev = &ds->nrows;
    ra.nrows0_dev = &ds->nrows0;
    // the trial's per-level fields (largest overlap, look-ahead displacement,
    // violator count + pad) are cleared by each level's row kernel
    static_assert(offsetof(DevStep, la_dmax) == offsetof(DevStep, maxov_bits) + 8 &&
                      offsetof(DevStep, nviol) == offsetof(DevStep, maxov_bits) + 16,
                  "per-level fields of DevStep must be three consecutive words");
    ra.clear3 = &ds->maxov_bits;
    ra.status = &ds->status;
    ra.gamma0 = c->gamma0.p;
    ra.rowof = c->rowof.p;
    auto bind_rows = [&](RowsArgs& r) {
        r.cap = c->rcap;
        r.ia = c->r_ia.p;
        r.ib = c->r_ib.p;
        r.rec = c->r_rec.p;
        r.pair = c->r_pair.p;
        r.geom = c->r_geom.p;
        r.geomf = mixed ? c->r_geomf.p : nullptr;
        r.q = c->r_q.p;
        r.qf = mixed ? c->r_qf.p : nullptr;
        r.diag = c->r_diag.p;
        const bool jac = (cfg.flags & RELCP_FLAG_JACOBI) != 0;  // 1 / A_aa is only used by the Jacobi metric
        r.invd = (!mixed && jac) ? c->r_invd.p : nullptr;
        r.invdf = (mixed && jac) ? c->r_invdf.p : nullptr;
        r.gamma = mixed ? nullptr : c->r_gamma.p;
        r.gammaf = mixed ? c->r_gammaf.p : nullptr;
    };
    bind_rows(ra);
    int64_t m_bound = np;  // rows <= m_bound until the host learns the count

    // LCP on the current rows (row buffers may move when rows are appended)
    auto make_pr = [&](LcpProblem& pr) {
        pr = LcpProblem{};
        pr.m_cap = m_bound;
        pr.nrows_dev = &ds->nrows;
        pr.nbodies = n;
        pr.ia = c->r_ia.p;
        pr.ib = c->r_ib.p;
        for (int k = 0; k < 9; ++k)
            pr.geom[k] = mixed ? (const void*)(c->r_geomf.p + k * c->rcap) : (const void*)(c->r_geom.p + k * c->rcap);
        pr.q = c->r_q.p;
        pr.qr = mixed ? (const void*)c->r_qf.p : (const void*)c->r_q.p;
        pr.diag = c->r_diag.p;
        pr.invd = nullptr;
        if (cfg.flags & RELCP_FLAG_JACOBI) pr.invd = mixed ? (const void*)c->r_invdf.p : (const void*)c->r_invd.p;
        for (int k = 0; k < 7; ++k) {
            pr.K[k] = c->K.p + k * n;
            pr.Kr[k] = mixed ? (const void*)(c->Kf.p + k * n) : (const void*)(c->K.p + k * n);
        }
        pr.c = dt;
        pr.mixed = mixed ? 1 : 0;
        pr.tol = cfg.lcp_tol;
        pr.refine = (cfg.flags & RELCP_FLAG_NO_LCP_REFINE) ? 0 : 1;
        pr.max_iter = (cfg.fault_inject & RELCP_FAULT_LCP_ITERS) ? 1 : cfg.lcp_max_iter;
        if (cfg.fault_inject & RELCP_FAULT_LCP_TIMEOUT) {
            pr.wait_ns = kFaultWaitNs;
            pr.fault_skip_block = 1;
        }
        pr.gamma = mixed ? (void*)c->r_gammaf.p : (void*)c->r_gamma.p;
        for (int k = 0; k < 6; ++k) pr.uc[k] = c->uc.p + k * n;
        pr.result = &ds->lcp;
        pr.status = &ds->status;
    };

    // trial configuration and overlap test (the list look-ahead for the next
    // step folded into the trial pass: the cached list against these trial
    // positions, accepted if the recursion stops here, in the next box)
    TrialArgs ta{};
    ta.shape = cfg.shape;
    ta.n = n;
    ta.dt = dt;
    ta.x = c->x.p;
    ta.q = c->q.p;
    ta.axes = c->axes.p;
    ta.ufree = c->ufree.p;
    ta.uc = c->uc.p;
    ta.xt = c->xt.p;
    ta.qt = c->qt.p;
    ta.Pt = c->Pt.p;
    ta.ustep = c->ustep.p;
    ta.xb = nullptr;
    if (broadphase_lookahead_params(c->bp, n, box1, ta.sfac)) {
        ta.xb = c->bp.xb.p;
        for (int k = 0; k < 3; ++k) ta.la_box[k] = box1[k];
        ta.sfac_dev = c->sblk.p->k.sfac;
        ta.la_box_dev = box1_dev;
        ta.la_dmax = &ds->la_dmax;
    }
    SnsdArgs sb = sa;
    sb.idx = nullptr;
    sb.count_dev = npd;
    sb.x = View<3, const double>::soa(c->xt.p, n);
    sb.P = View<6, const double>::soa(c->Pt.p, n);
    for (int k = 0; k < 3; ++k) sb.box[k] = box1[k];
    sb.box_dev = box1_dev;
    sb.guess = View<3, const double>::soa(c->s0.p + np, np);  // warm start: normals at C^k
    sb.out = snsd_out(c->s1, c->it1);
    sb.eps = cfg.eps_ncp;
    sb.viol = c->flags.p;
    sb.maxov_bits = &ds->maxov_bits;
    sb.nviol = &ds->nviol;
    sb.iters_sum = nullptr;
    sb.newton_max = &ds->newton_max;

    int k0 = -1, k1 = -1, lcp_l0 = -1;
    LcpProblem pr;
    // the persistent LCP launch between its timing events
    auto lcp_mid = [&]() -> relcp_status {
        pr.ev_before = tm.take(&k0);
        pr.ev_after = tm.take(&k1);
        int blocks = 0;
        RELCP_TRY(lcp_run(pr, c->lcp, &blocks, s));
        lcpk_marks.push_back({k0, k1});
        return RELCP_OK;
    };
    // after the LCP: trial, overlap test, readback
    auto post_lcp = [&]() -> relcp_status {
        // (the per-level fields were cleared by the level's row kernel, or with
        // the whole DevStep at the start of the step)
        RELCP_TRY(trial_launch(ta, s));
        {
            int e0 = tm.mark();
            RELCP_TRY(snsd_launch(sb, s));
            snsd_marks.push_back({e0, tm.mark()});
        }
        RELCP_CUDA(cudaMemcpyAsync(c->hstep, ds, sizeof(DevStep), cudaMemcpyDeviceToHost, s));
        return RELCP_OK;
    };
    // one recursion level from the LCP to the readback
    auto level_tail = [&]() -> relcp_status {
        make_pr(pr);
        int l0 = tm.mark();
        RELCP_TRY(lcp_build_csr(pr, c->lcp, s));
        RELCP_TRY(lcp_mid());
        lcp_marks.push_back({l0, tm.mark()});
        return post_lcp();
    };
    // level 0 after the broad phase, up to the LCP's incidence CSR
    auto level0_pre = [&]() -> relcp_status {
        if (np > 0) {
            if (!fast_bp) RELCP_CUDA(cudaMemcpyAsync(&ds->np, npd, sizeof(int), cudaMemcpyDeviceToDevice, s));
            RELCP_TRY(reuse_launch(ru, s));
            // (a step that carries the previous step's values evaluates only the
            // pairs new to the list, far fewer than kLearnedMinPairs: the
            // network is not launched at all then; its flag stays 0)
            if (learned && !ru.reuse_snsd)
                RELCP_TRY(mlp_guess(c->mlp, np, c->pa.p, c->pb.p, xv, View<4, const double>::soa(c->q.p, n),
                                    View<3, const double>::soa(c->axes.p, n), box0, s, c->idx.p, count_dev,
                                    &ds->status, box0_dev,
                                    (cfg.flags & RELCP_FLAG_LEARNED_ALWAYS) ? 1 : kLearnedMinPairs, &ds->guess_on,
                                    &ds->declined));
        }
        {
            int e0 = tm.mark();
            RELCP_TRY(snsd_launch(sa, s));
            snsd_marks.push_back({e0, tm.mark()});
        }
        if (np > 0) {
            RELCP_TRY(flag_le_launch(np, npd, c->s0.p, cfg.phi_skin, c->flags.p, s));
            RELCP_TRY(exclusive_scan(c->flags.p, c->fscan.p, np, c->scan, s));
            RELCP_TRY(rows_launch(ra, s));
        }
        make_pr(pr);
        lcp_l0 = tm.mark();
        return lcp_build_csr(pr, c->lcp, s);
    };
    // the first level with the fast broad phase, up to the LCP's CSR
    auto level0_fast_pre = [&]() -> relcp_status {
        t_begin = tm.mark();
        RELCP_TRY(head());
        RELCP_TRY(broadphase_filter_async(n, c->x.p, c->rb.p, box0, box0_dev, cfg.skin, c->pa, c->pb, c->bp, s,
                                          &ds->np));
        t_bp = tm.mark();
        return level0_pre();
    };
    auto run_direct = [&](bool fast) -> relcp_status {
        RELCP_TRY(fast ? level0_fast_pre() : level0_pre());
        RELCP_TRY(lcp_mid());
        lcp_marks.push_back({lcp_l0, tm.mark()});
        return post_lcp();
    };
    // capture fn into *out; false when the stream cannot be captured or the
    // capture fails (nothing of fn has run then)
    auto capture = [&](const std::function<relcp_status()>& fn, cudaGraphExec_t* out, long long* nk) -> bool {
        *out = nullptr;
        const long long l_before = relcp_kernel_launches();
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        const relcp_status r = fn();
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &graph);
        *nk += relcp_kernel_launches() - l_before;
        note_launches(-(relcp_kernel_launches() - l_before));  // captured, not run
        bool ok = r == RELCP_OK && e == cudaSuccess && graph && cudaGraphInstantiate(out, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            *out = nullptr;
            (void)cudaGetLastError();
        }
        return ok;
    };
    if (!fast_bp) {
        RELCP_TRY(run_direct(false));
    } else if (!(cfg.flags & RELCP_FLAG_GRAPH) || (cfg.flags & RELCP_FLAG_PHASE_TIMING) || !prepped ||
               s == nullptr || s == cudaStreamLegacy) {
        // (the legacy default stream cannot be captured)
        RELCP_TRY(run_direct(true));
    } else {
        // replay the captured graphs of this configuration (before and after
        // the LCP launch, which stays between its timing events), capture them
        // on the configuration's second sighting, run directly on the first
        std::vector<uintptr_t> key;
        step_key(c, PC, key);
        StepGraph* g = nullptr;
        for (auto& e : c->graphs)
            if (e.key == key) g = &e;
        if (!g) {
            if (c->graphs.size() >= 4) {
                destroy_graph(c->graphs.front());
                c->graphs.erase(c->graphs.begin());
            }
            c->graphs.push_back(StepGraph{key, false, nullptr, nullptr, 0});
            RELCP_TRY(run_direct(true));
        } else if (g->uncapturable) {
            RELCP_TRY(run_direct(true));
        } else {
            if (!g->pre) {
                long long nk = 0;
                bool ok = capture(level0_fast_pre, &g->pre, &nk);
                if (ok) ok = capture(post_lcp, &g->post, &nk);
                if (ok) {
                    g->nkernels = nk;
                } else {
                    destroy_graph(*g);
                    g->uncapturable = true;
                }
                snsd_marks.clear();
                lcp_marks.clear();
                lcpk_marks.clear();
            }
            if (g->pre) {
                make_pr(pr);
                st.graph_replayed = 1;
                RELCP_CUDA(cudaGraphLaunch(g->pre, s));
                RELCP_TRY(lcp_mid());
                RELCP_CUDA(cudaGraphLaunch(g->post, s));
                note_launches(g->nkernels);
            } else {
                RELCP_TRY(run_direct(true));
            }
        }
    }

    int depth = 0;
    int lcp_iters_total = 0;
    relcp_status step_status = RELCP_OK;
    DevStep hs{};
    int t_last = tm.mark();
    for (;;) {
        {
            const auto w0 = std::chrono::steady_clock::now();
            RELCP_CUDA(cudaStreamSynchronize(s));
            wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
        }
        hs = *c->hstep;
        const int nv = np > 0 ? hs.nviol : 0;
        c->npairs = hs.np;
        c->nrows = hs.nrows;
        if (depth == 0) c->nrows0 = hs.nrows;
        if (depth < RELCP_MAX_DEPTH_STATS) {
            st.lcp_iters[depth] = (int)hs.lcp.iterations;
            st.rows_per_rec[depth] = hs.nrows;
        }
        lcp_iters_total += (int)hs.lcp.iterations;
        if (tm.kernels && hs.nrows > 0) {
            st.ms_lcp_kernel += tm.ms(k0, k1);
            st.lcp_alg_bytes += lcp_bytes_per_iter(hs.nrows, n, mixed) * (hs.lcp.iterations + 1);
            st.lcp_launches += 1;
        }
        if (hs.status & DEV_TIMEOUT) {
            set_error("a device wait timed out (LCP grid barrier or prefix-sum look-back)");
            tm.stop();
            return RELCP_ERR_TIMEOUT;
        }
        if (nv == 0) break;
        if (depth >= cfg.max_recursion) {
            step_status = RELCP_ERR_RECURSION_LIMIT;
            break;
        }
        ++depth;
        // positions of the appended rows (the violator flags of the last test)
        RELCP_TRY(exclusive_scan(c->flags.p, c->fscan.p, np, c->scan, s));
        RELCP_TRY(grow_rows(c, c->nrows + nv));
        RowsArgs rb2 = ra;
        rb2.gamma0 = nullptr;
        rb2.rowof = nullptr;
        rb2.nrows0_dev = nullptr;
        bind_rows(rb2);
        rb2.snsd = c->s1.p;
        rb2.base = c->nrows;
        rb2.rec_index = depth;
        RELCP_TRY(rows_launch(rb2, s));
        m_bound = c->nrows + nv;
        RELCP_TRY(level_tail());
        t_last = tm.mark();
    }

    // memo for the next step: every candidate pair's final A_0 gamma (0 without
    // a row) and its index in this step's last overlap test, whose SNSD output
    // (s1, at the configuration accepted below) becomes s1prev
    if (np > 0) {
        MemoSaveArgs ms{};
        ms.npairs = np;
        ms.np_dev = npd;
        ms.pv = c->bp.pv.p;
        ms.rowof = c->rowof.p;
        ms.gamma = mixed ? nullptr : c->r_gamma.p;
        ms.gammaf = mixed ? c->r_gammaf.p : nullptr;
        ms.stamp = (c->stamp + 1) & 0x3fffffff;
        ms.memo = c->bp.memo.p;
        RELCP_TRY(memo_save_launch(ms, s));
    }
    std::swap(c->s1, c->s1prev);
    c->sprev_stride = np;
    c->nprev = hs.np;
    c->stamp = (c->stamp + 1) & 0x3fffffff;
    c->memo_ok = true;
    c->snsd_ok = true;
    // the last look-ahead was taken at the configuration accepted below
    c->la_ok = true;
    c->la_rebuild =
        !verlet_bound_holds(c->bp, n, box1, c->rb_max, cfg.skin, std::sqrt(__builtin_bit_cast(double, hs.la_dmax)));

    // accept C^{k+1} (no synchronisation: the next call queues behind it)
    AcceptArgs aa{};
    aa.n = n;
    aa.inertial = cfg.dynamics == RELCP_INERTIAL;
    for (int k = 0; k < 3; ++k) aa.box[k] = box1[k];
    aa.xt = c->xt.p;
    aa.qt = c->qt.p;
    aa.ustep = c->ustep.p;
    aa.x = c->x.p;
    aa.q = c->q.p;
    aa.vel = c->vel.p;
    // the next step's prep in the same pass, on the accepted state in the next box
    aa.next = pa;
    for (int k = 0; k < 3; ++k) aa.next.box[k] = box1[k];
    aa.keep = cfg.dynamics != RELCP_INERTIAL;
    aa.Pt = c->Pt.p;
    RELCP_TRY(accept_launch(aa, s));
    c->prepped = true;
    for (int k = 0; k < 3; ++k) c->box[k] = box1[k];
    relcp_status dstat = status_from_device(hs.status);
    if (step_status == RELCP_OK) step_status = dstat;
    st.n_rows = c->nrows;
    st.n_rows0 = c->nrows0;
    st.depth = depth;
    st.status = step_status;
    st.lcp_iters_total = lcp_iters_total;
    st.newton_iters_max = hs.newton_max;
    st.newton_iters_c0 = (int64_t)hs.iters0;
    st.n_pairs = hs.np;
    st.snsd_c0_evaluated = hs.c0_evals;
    st.guess_used = learned ? hs.guess_on : 0;
    st.newton_fallbacks = (learned && hs.guess_on) ? hs.declined : 0;
    st.lcp_residual = hs.lcp.residual;
    st.max_overlap = __builtin_bit_cast(double, hs.maxov_bits);
    for (int k = 0; k < 3; ++k) st.box[k] = c->box[k];
    if (tm.on) {
        st.ms_broadphase = tm.ms(t_begin, t_bp);
        st.ms_total = tm.ms(t_begin, t_last);
        for (size_t m = 0; m < snsd_marks.size(); ++m) {
            st.ms_snsd_kernel += tm.ms(snsd_marks[m].first, snsd_marks[m].second);
            st.snsd_launches += 1;
            st.snsd_evals += m == 0 ? hs.c0_evals : hs.np;  // the first launch is the C^k evaluation
        }
        st.ms_snsd = st.ms_snsd_kernel;
        for (auto& mk : lcp_marks) st.ms_lcp += tm.ms(mk.first, mk.second);
        st.ms_augment = st.ms_total - st.ms_broadphase - st.ms_snsd - st.ms_lcp;
    }
    tm.stop();
    c->steps_done += 1;
    st.steps_done = c->steps_done;
    st.host_wait_ms = wait_ms;
    st.host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h0).count();
    c->stats = st;
    return step_status;
}


}  // namespace

extern "C" {

const char* relcp_last_error(void) { return relcp::g_err; }

int64_t relcp_kernel_launches(void) { return (int64_t)relcp::g_launches.load(); }

relcp_status relcp_version(int32_t* major, int32_t* minor, int32_t* sm_count) {
    if (major) *major = 1;
    if (minor) *minor = 0;
    if (sm_count) *sm_count = device_sm_count();
    return RELCP_OK;
}

relcp_status relcp_create(const relcp_config* cfg, void* cuda_stream, relcp_ctx** out) {
    if (!out) return set_error("out is NULL"), RELCP_ERR_INVALID_ARG;
    *out = nullptr;
    RELCP_TRY(check_config(cfg));
    relcp_ctx* c = new relcp_ctx();
    c->cfg = *cfg;
    c->s = (cudaStream_t)cuda_stream;
    for (int k = 0; k < 3; ++k) c->box[k] = cfg->box[k];
    relcp_status st = c->sblk.ensure(1, c->s);
    if (st == RELCP_OK && cudaMallocHost((void**)&c->hstep, sizeof(DevStep)) != cudaSuccess) {
        set_error("pinned allocation failed");
        st = RELCP_ERR_CUDA;
    }
    if (st == RELCP_OK) st = c->dcheck.ensure(1, c->s);
    if (st == RELCP_OK && cudaMallocHost((void**)&c->hcheck, sizeof(BodyCheck)) != cudaSuccess) {
        set_error("pinned allocation failed");
        st = RELCP_ERR_CUDA;
    }
    if (st == RELCP_OK) {
        int dev = 0, pma = 0, pht = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, dev);
        cudaDeviceGetAttribute(&pht, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev);
        c->pageable_ok = pma == 1 && pht == 1;
    }
    if (st == RELCP_OK && cudaMallocHost((void**)&c->hup, sizeof(StepBlock)) != cudaSuccess) {
        set_error("pinned allocation failed");
        st = RELCP_ERR_CUDA;
    }
    if (st == RELCP_OK) std::memset(c->hup, 0, sizeof(StepBlock));
    if (st == RELCP_OK) {
        // the context's prefix sums report a look-back timeout in the step's status word
        c->scan.status = c->bp.scan.status = c->lcp.scan.status = &c->sblk.p->d.status;
    }
    if (st != RELCP_OK) {
        c->sblk.release(c->s);
        c->dcheck.release(c->s);
        if (c->hstep) cudaFreeHost(c->hstep);
        if (c->hup) cudaFreeHost(c->hup);
        if (c->hcheck) cudaFreeHost(c->hcheck);
        delete c;
        return st;
    }
    *out = c;
    return RELCP_OK;
}

relcp_status relcp_set_config(relcp_ctx* c, const relcp_config* cfg) {
    if (!c) return set_error("ctx is NULL"), RELCP_ERR_INVALID_ARG;
    RELCP_TRY(check_config(cfg));
    // the carried SNSD values hold for the current box and precision only
    bool box_same = true;
    for (int k = 0; k < 3; ++k)
        if (cfg->box[k] != c->box[k]) box_same = false;
    if (!box_same || cfg->precision != c->cfg.precision || cfg->skin != c->cfg.skin) c->snsd_ok = false;
    // the config's box is the current box (it follows the compaction), the rest
    // is compared with the config in force
    relcp_config a = *cfg, b = c->cfg;
    for (int k = 0; k < 3; ++k) a.box[k] = b.box[k] = 0.0;
    if (!box_same || std::memcmp(&a, &b, sizeof(relcp_config)) != 0) {
        c->la_ok = false;  // the broad phase checks its cached list again
        c->prepped = false;
        drop_graphs(c);
    }
    c->cfg = *cfg;
    for (int k = 0; k < 3; ++k) c->box[k] = cfg->box[k];
    return RELCP_OK;
}

relcp_status after_set_bodies(relcp_ctx* c, int64_t n, bool same_n, int changed, double rbmax);

// the per-body state and scratch arrays for n bodies
static relcp_status ensure_body_arrays(relcp_ctx* c, int64_t n) {
    cudaStream_t s = c->s;
    const int64_t na = n > 0 ? n : 1;
    RELCP_TRY(c->x.ensure(3 * na, s));
    RELCP_TRY(c->q.ensure(4 * na, s));
    RELCP_TRY(c->axes.ensure(3 * na, s));
    RELCP_TRY(c->vel.ensure(6 * na, s));
    RELCP_TRY(c->fext.ensure(6 * na, s));
    RELCP_TRY(c->P.ensure(6 * na, s));
    RELCP_TRY(c->K.ensure(7 * na, s));
    RELCP_TRY(c->rb.ensure(na, s));
    RELCP_TRY(c->ufree.ensure(6 * na, s));
    RELCP_TRY(c->uc.ensure(6 * na, s));
    RELCP_TRY(c->ustep.ensure(6 * na, s));
    RELCP_TRY(c->xt.ensure(3 * na, s));
    RELCP_TRY(c->qt.ensure(4 * na, s));
    RELCP_TRY(c->Pt.ensure(6 * na, s));
    return RELCP_OK;
}

// pinned host staging for the body state (grown on demand)
static relcp_status ensure_hstage(relcp_ctx* c, size_t count) {
    if (c->hstage_cap >= count && c->hstage) return RELCP_OK;
    if (c->hstage) cudaFreeHost(c->hstage);
    c->hstage = nullptr;
    c->hstage_cap = 0;
    const size_t nc = count + count / 4 + 64;
    if (cudaMallocHost((void**)&c->hstage, nc * sizeof(double)) != cudaSuccess) {
        set_error("pinned allocation of %zu doubles failed", nc);
        return RELCP_ERR_CUDA;
    }
    c->hstage_cap = nc;
    return RELCP_OK;
}

relcp_status relcp_set_bodies(relcp_ctx* c, int64_t n, const int32_t* scene_offsets, const double* x,
                              const double* q, const double* semi_axes, const double* vel, const double* f_ext,
                              const double* dt_per_scene, int32_t ptr_kind) {
    if (!c) return set_error("ctx is NULL"), RELCP_ERR_INVALID_ARG;
    if (n < 0 || n > (int64_t)1 << 28) return set_error("n out of range"), RELCP_ERR_INVALID_ARG;
    if (scene_offsets || dt_per_scene)
        return set_error("scene_offsets / dt_per_scene must be NULL for a single-scene context"),
               RELCP_ERR_INVALID_ARG;
    if (ptr_kind != RELCP_PTR_HOST && ptr_kind != RELCP_PTR_DEVICE)
        return set_error("bad ptr_kind"), RELCP_ERR_INVALID_ARG;
    if (n > 0 && (!x || !q || !semi_axes)) return set_error("x, q, semi_axes required"), RELCP_ERR_INVALID_ARG;
    cudaStream_t s = c->s;
    const bool same_n = c->has_bodies && c->n == n;
    const bool direct = ptr_kind == RELCP_PTR_DEVICE || (c->pageable_ok && !(c->cfg.flags & RELCP_FLAG_HOST_STAGING));
    if (direct && n > 0) {
        // the device reads the caller's arrays in place: one pass validates,
        // compares with the current state and copies the rows to the device
        // stage, writing nothing to the state; the load follows only for a
        // valid, changed state
        RELCP_TRY(ensure_body_arrays(c, n));
        RELCP_TRY(c->dstage.ensure((size_t)(22 * n), s));
        for (int k = 0; k < 3; ++k) c->box[k] = c->cfg.box[k];
        BodyCheck init{};
        init.bad_key = ~0ull;
        *c->hcheck = init;
        RELCP_CUDA(cudaMemcpyAsync(c->dcheck.p, c->hcheck, sizeof(BodyCheck), cudaMemcpyHostToDevice, s));
        CheckArgs ca{};
        ca.n = n;
        ca.in = BodyIn{x, q, semi_axes, vel, f_ext};
        ca.x = c->x.p;
        ca.q = c->q.p;
        ca.axes = c->axes.p;
        ca.vel = c->vel.p;
        ca.fext = c->fext.p;
        for (int k = 0; k < 3; ++k) ca.box[k] = c->box[k];
        ca.compare = same_n ? 1 : 0;
        ca.stage = c->dstage.p;
        ca.out = c->dcheck.p;
        RELCP_TRY(check_bodies_launch(ca, s));
        RELCP_CUDA(cudaMemcpyAsync(c->hcheck, c->dcheck.p, sizeof(BodyCheck), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaStreamSynchronize(s));  // the caller's arrays are free again after this
        const BodyCheck chk = *c->hcheck;
        if (chk.bad_key != ~0ull) {
            const int bits = (int)(chk.bad_key & 15);
            const long long i = (long long)(chk.bad_key >> 4);
            const char* why = (bits & 1)   ? "quaternion norm is not 1"
                              : (bits & 2) ? "position not finite"
                              : (bits & 4) ? "semi-axes must be finite and > 0"
                                           : "velocity / force not finite";
            return set_error("body %lld: %s", i, why), RELCP_ERR_INVALID_ARG;
        }
        const int changed = same_n ? chk.changed : 3;
        if (changed) {
            LoadArgs la{};
            la.n = n;
            la.stage = c->dstage.p;
            la.x = c->x.p;
            la.q = c->q.p;
            la.axes = c->axes.p;
            la.vel = c->vel.p;
            la.fext = c->fext.p;
            for (int k = 0; k < 3; ++k) la.box[k] = c->box[k];
            la.compare = 0;
            la.changed = nullptr;
            RELCP_TRY(load_bodies_launch(la, s));
            RELCP_CUDA(cudaMemsetAsync(c->ustep.p, 0, 6 * n * sizeof(double), s));
        }
        return after_set_bodies(c, n, same_n, changed, __builtin_bit_cast(double, chk.rbmax_bits));
    }
    // otherwise the caller's rows are gathered into one pinned row-major block
    // of 22 doubles per body: x 3 | q 4 | axes 3 | vel 6 | fext 6
    RELCP_TRY(ensure_hstage(c, (size_t)(22 * (n > 0 ? n : 1))));
    double* st = c->hstage;
    if (n > 0) {
        if (ptr_kind == RELCP_PTR_DEVICE) RELCP_CUDA(cudaStreamSynchronize(s));
        auto gather = [&](const double* src, int w, int off) -> relcp_status {
            if (!src) {
                for (int64_t i = 0; i < n; ++i)
                    for (int k = 0; k < w; ++k) st[22 * i + off + k] = 0.0;
                return RELCP_OK;
            }
            if (ptr_kind == RELCP_PTR_DEVICE) {
                RELCP_CUDA(cudaMemcpy2D(st + off, 22 * sizeof(double), src, w * sizeof(double), w * sizeof(double),
                                        (size_t)n, cudaMemcpyDeviceToHost));
            } else {
                for (int64_t i = 0; i < n; ++i)
                    for (int k = 0; k < w; ++k) st[22 * i + off + k] = src[w * i + k];
            }
            return RELCP_OK;
        };
        RELCP_TRY(gather(x, 3, 0));
        RELCP_TRY(gather(q, 4, 3));
        RELCP_TRY(gather(semi_axes, 3, 7));
        RELCP_TRY(gather(vel, 6, 10));
        RELCP_TRY(gather(f_ext, 6, 16));
    }
    double rbmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double* r = st + 22 * i;
        double qq = 0;
        for (int k = 0; k < 4; ++k) qq += r[3 + k] * r[3 + k];
        if (!(fabs(sqrt(qq) - 1.0) <= 1e-6))
            return set_error("body %lld: quaternion norm %.17g is not 1", (long long)i, sqrt(qq)),
                   RELCP_ERR_INVALID_ARG;
        for (int k = 0; k < 3; ++k) {
            if (!std::isfinite(r[k])) return set_error("body %lld: position not finite", (long long)i), RELCP_ERR_INVALID_ARG;
            if (!(r[7 + k] > 0) || !std::isfinite(r[7 + k]))
                return set_error("body %lld: semi-axes must be finite and > 0", (long long)i), RELCP_ERR_INVALID_ARG;
            rbmax = r[7 + k] > rbmax ? r[7 + k] : rbmax;
        }
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(r[10 + k]))
                return set_error("body %lld: velocity / force not finite", (long long)i), RELCP_ERR_INVALID_ARG;
    }
    // what the step's carried data still holds depends on what changed: a
    // bitwise comparison with the current state, on the device
    const int64_t na = n > 0 ? n : 1;
    RELCP_TRY(ensure_body_arrays(c, n));
    RELCP_TRY(c->dstage.ensure((size_t)(22 * na), s));
    int changed = 3;
    if (n > 0) {
        for (int k = 0; k < 3; ++k) c->box[k] = c->cfg.box[k];
        RELCP_CUDA(cudaMemcpyAsync(c->dstage.p, st, 22 * n * sizeof(double), cudaMemcpyHostToDevice, s));
        RELCP_CUDA(cudaMemsetAsync(&c->sblk.p->d.status, 0, sizeof(int), s));
        LoadArgs la{};
        la.n = n;
        la.stage = c->dstage.p;
        la.x = c->x.p;
        la.q = c->q.p;
        la.axes = c->axes.p;
        la.vel = c->vel.p;
        la.fext = c->fext.p;
        for (int k = 0; k < 3; ++k) la.box[k] = c->box[k];
        la.compare = same_n ? 1 : 0;
        la.changed = &c->sblk.p->d.status;  // scratch word, cleared above and by the next step
        RELCP_TRY(load_bodies_launch(la, s));
        RELCP_CUDA(cudaMemcpyAsync(&c->hstep->status, &c->sblk.p->d.status, sizeof(int), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaMemsetAsync(c->ustep.p, 0, 6 * n * sizeof(double), s));
        RELCP_CUDA(cudaStreamSynchronize(s));  // the pinned staging is reused by the next call
        if (same_n) changed = c->hstep->status;
    }
    return after_set_bodies(c, n, same_n, changed, rbmax);
}

// what the context keeps after new bodies: everything for an unchanged state;
// the pair list (guarded by its displacement check) and the warm starts for
// moved bodies; nothing for other bodies or shapes
relcp_status after_set_bodies(relcp_ctx* c, int64_t n, bool same_n, int changed, double rbmax) {
    if (!same_n || (changed & 2)) {
        // other bodies or other shapes: nothing carried over
        c->memo_ok = false;
        c->bp.valid = false;
        c->rb_max = rbmax;
    }
    if (changed) {
        // the carried SNSD values, the list look-ahead, the prepared body
        // operators and the captured graphs hold only for the state they were
        // made for; the cached pair list (guarded by its displacement check)
        // and the warm-start gammas (a start only) stay
        c->snsd_ok = false;
        c->la_ok = false;
        c->prepped = false;
        drop_graphs(c);
    }
    c->n = n;
    c->has_bodies = true;
    c->steps_done = 0;
    c->nrows = 0;
    if (changed) c->npairs = 0;
    return RELCP_OK;
}

relcp_status relcp_get_bodies_impl(relcp_ctx* c, double* x, double* q, double* vel, int32_t ptr_kind) {
    const int64_t n = c->n;
    if (n == 0) return RELCP_OK;
    cudaStream_t s = c->s;
    const double* vsrc = c->steps_done > 0 ? c->ustep.p : c->vel.p;
    if (ptr_kind == RELCP_PTR_DEVICE || (c->pageable_ok && !(c->cfg.flags & RELCP_FLAG_HOST_STAGING))) {
        // written in place into the caller's arrays
        RELCP_TRY(store_direct_launch(n, c->x.p, c->q.p, vsrc, x, q, vel, s));
        RELCP_CUDA(cudaStreamSynchronize(s));
        return RELCP_OK;
    }
    RELCP_TRY(c->dstage.ensure((size_t)(22 * n), s));
    RELCP_TRY(ensure_hstage(c, (size_t)(13 * n)));
    RELCP_TRY(store_bodies_launch(n, x ? c->x.p : nullptr, q ? c->q.p : nullptr, vel ? vsrc : nullptr,
                                  c->dstage.p, s));
    RELCP_CUDA(cudaMemcpyAsync(c->hstage, c->dstage.p, 13 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    RELCP_CUDA(cudaStreamSynchronize(s));
    const double* r0 = c->hstage;
    auto put = [&](double* dst, int w, int off) -> relcp_status {
        if (!dst) return RELCP_OK;
        if (ptr_kind == RELCP_PTR_DEVICE) {
            RELCP_CUDA(cudaMemcpy2D(dst, w * sizeof(double), r0 + off, 13 * sizeof(double), w * sizeof(double),
                                    (size_t)n, cudaMemcpyHostToDevice));
        } else {
            for (int64_t i = 0; i < n; ++i)
                for (int k = 0; k < w; ++k) dst[w * i + k] = r0[13 * i + off + k];
        }
        return RELCP_OK;
    };
    RELCP_TRY(put(x, 3, 0));
    RELCP_TRY(put(q, 4, 3));
    RELCP_TRY(put(vel, 6, 7));
    return RELCP_OK;
}

relcp_status relcp_step(relcp_ctx* c, int32_t nsteps) {
    if (!c) return set_error("ctx is NULL"), RELCP_ERR_INVALID_ARG;
    if (!c->has_bodies) return set_error("relcp_set_bodies has not been called"), RELCP_ERR_STATE;
    if (nsteps < 1) return set_error("nsteps must be >= 1"), RELCP_ERR_INVALID_ARG;
    if (c->cfg.guess == RELCP_GUESS_MLP && !c->mlp.loaded)
        return set_error("guess = RELCP_GUESS_MLP needs relcp_load_mlp first"), RELCP_ERR_STATE;
    for (int k = 0; k < nsteps; ++k) {
        relcp_status st = step_once(c);
        if (st != RELCP_OK) return st;
    }
    return RELCP_OK;
}

relcp_status relcp_get_bodies(relcp_ctx* c, double* x, double* q, double* vel, int32_t ptr_kind) {
    if (!c) return set_error("ctx is NULL"), RELCP_ERR_INVALID_ARG;
    if (!c->has_bodies) return set_error("no bodies"), RELCP_ERR_STATE;
    if (ptr_kind != RELCP_PTR_HOST && ptr_kind != RELCP_PTR_DEVICE) return set_error("bad ptr_kind"), RELCP_ERR_INVALID_ARG;
    return relcp_get_bodies_impl(c, x, q, vel, ptr_kind);
}

relcp_status relcp_get_box(relcp_ctx* c, double* box3) {
    if (!c || !box3) return set_error("NULL argument"), RELCP_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k) box3[k] = c->box[k];
    return RELCP_OK;
}

relcp_status relcp_stats(relcp_ctx* c, relcp_step_stats* out) {
    if (!c || !out) return set_error("NULL argument"), RELCP_ERR_INVALID_ARG;
    *out = c->stats;
    return RELCP_OK;
}

relcp_status relcp_get_pairs(relcp_ctx* c, int32_t* pairs, double* phi0, int64_t cap, int64_t* n_out,
                             int32_t ptr_kind) {
    (void)ptr_kind;
    if (!c || !n_out) return set_error("NULL argument"), RELCP_ERR_INVALID_ARG;
    *n_out = c->npairs;
    if (c->npairs > cap) return RELCP_ERR_CAPACITY;
    const int64_t np = c->npairs;
    if (np == 0) return RELCP_OK;
    cudaStream_t s = c->s;
    if (pairs) {
        RELCP_CUDA(cudaMemcpy2DAsync(pairs, 2 * sizeof(int), c->pa.p, sizeof(int), sizeof(int), np, cudaMemcpyDefault, s));
        RELCP_CUDA(cudaMemcpy2DAsync(pairs + 1, 2 * sizeof(int), c->pb.p, sizeof(int), sizeof(int), np, cudaMemcpyDefault, s));
    }
    if (phi0) RELCP_CUDA(cudaMemcpyAsync(phi0, c->s0.p, np * sizeof(double), cudaMemcpyDefault, s));
    RELCP_CUDA(cudaStreamSynchronize(s));
    return RELCP_OK;
}

relcp_status relcp_get_rows(relcp_ctx* c, int32_t* ids, double* geom, double* gamma, int64_t cap, int64_t* n_out,
                            int32_t ptr_kind) {
    (void)ptr_kind;
    if (!c || !n_out) return set_error("NULL argument"), RELCP_ERR_INVALID_ARG;
    *n_out = c->nrows;
    if (c->nrows > cap) return RELCP_ERR_CAPACITY;
    const int64_t m = c->nrows;
    if (m == 0) return RELCP_OK;
    cudaStream_t s = c->s;
    if (ids) {
        const int* src[4] = {c->r_ia.p, c->r_ib.p, c->r_rec.p, c->r_pair.p};
        for (int k = 0; k < 4; ++k)
            RELCP_CUDA(cudaMemcpy2DAsync(ids + k, 4 * sizeof(int), src[k], sizeof(int), sizeof(int), m, cudaMemcpyDefault, s));
    }
    if (geom) {
        for (int k = 0; k < 9; ++k)
            RELCP_CUDA(cudaMemcpy2DAsync(geom + k, 11 * sizeof(double), c->r_geom.p + k * c->rcap, sizeof(double),
                                         sizeof(double), m, cudaMemcpyDefault, s));
        RELCP_CUDA(cudaMemcpy2DAsync(geom + 9, 11 * sizeof(double), c->r_q.p, sizeof(double), sizeof(double), m,
                                     cudaMemcpyDefault, s));
        RELCP_CUDA(cudaMemcpy2DAsync(geom + 10, 11 * sizeof(double), c->r_diag.p, sizeof(double), sizeof(double), m,
                                     cudaMemcpyDefault, s));
    }
    if (gamma) {
        if (c->cfg.precision == RELCP_MIXED && c->r_gammaf.p) {
            std::vector<float> gf((size_t)m);
            RELCP_CUDA(cudaMemcpyAsync(gf.data(), c->r_gammaf.p, m * sizeof(float), cudaMemcpyDeviceToHost, s));
            RELCP_CUDA(cudaStreamSynchronize(s));
            std::vector<double> gd(gf.begin(), gf.end());
            RELCP_CUDA(cudaMemcpyAsync(gamma, gd.data(), m * sizeof(double), cudaMemcpyDefault, s));
        } else {
            RELCP_CUDA(cudaMemcpyAsync(gamma, c->r_gamma.p, m * sizeof(double), cudaMemcpyDefault, s));
        }
    }
    RELCP_CUDA(cudaStreamSynchronize(s));
    return RELCP_OK;
}

relcp_status relcp_get_contact_velocity(relcp_ctx* c, double* uc, int32_t ptr_kind) {
    (void)ptr_kind;
    if (!c || !uc) return set_error("NULL argument"), RELCP_ERR_INVALID_ARG;
    const int64_t n = c->n;
    if (n == 0) return RELCP_OK;
    for (int k = 0; k < 6; ++k)
        RELCP_CUDA(cudaMemcpy2DAsync(uc + k, 6 * sizeof(double), c->uc.p + k * n, sizeof(double), sizeof(double), n,
                                     cudaMemcpyDefault, c->s));
    RELCP_CUDA(cudaStreamSynchronize(c->s));
    return RELCP_OK;
}

relcp_status relcp_load_mlp(relcp_ctx* c, const float* params, int32_t ptr_kind) {
    if (!c || !params) return set_error("NULL argument"), RELCP_ERR_INVALID_ARG;
    RELCP_TRY(c->mlp.params.ensure(RELCP_MLP_NPARAMS, c->s));
    RELCP_CUDA(cudaMemcpyAsync(c->mlp.params.p, params, RELCP_MLP_NPARAMS * sizeof(float),
                               ptr_kind == RELCP_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->s));
    RELCP_TRY(c->mlp.image.ensure(mlp_image_bytes(), c->s));
    RELCP_TRY(mlp_pack_launch(c->mlp.params.p, c->mlp.image.p, c->s));
    RELCP_CUDA(cudaStreamSynchronize(c->s));
    c->mlp.loaded = true;
    return RELCP_OK;
}

void relcp_destroy(relcp_ctx* c) {
    if (!c) return;
    cudaStream_t s = c->s;
    cudaStreamSynchronize(s);
    drop_graphs(c);
    DBuf<double>* dbs[] = {&c->x, &c->q, &c->axes, &c->vel, &c->fext, &c->P, &c->K, &c->rb, &c->ufree, &c->uc,
                           &c->ustep, &c->xt, &c->qt, &c->Pt, &c->s0, &c->s1, &c->r_geom, &c->r_q, &c->r_diag,
                           &c->r_gamma};
    for (auto* b : dbs) b->release(s);
    DBuf<int>* ibs[] = {&c->pa, &c->pb, &c->it0, &c->it1, &c->flags, &c->fscan, &c->r_ia, &c->r_ib, &c->r_rec,
                        &c->r_pair, &c->bp.cell_of, &c->bp.cell_count, &c->bp.cell_start, &c->bp.cell_cursor,
                        &c->bp.cell_body, &c->bp.pair_count, &c->bp.pair_off, &c->bp.vpa, &c->bp.vpb, &c->bp.vflag, &c->bp.vscan};
    for (auto* b : ibs) b->release(s);
    c->r_geomf.release(s);
    c->r_gammaf.release(s);
    c->r_qf.release(s);
    c->Kf.release(s);
    c->ufreef.release(s);
    c->r_invd.release(s);
    c->r_invdf.release(s);
    c->sblk.release(s);
    c->dstage.release(s);
    c->dcheck.release(s);
    c->bp.xb.release(s);
    c->bp.dmax.release(s);
    c->s1prev.release(s);
    c->gamma0.release(s);
    c->idx.release(s);
    c->rowof.release(s);
    c->bp.memo.release(s);
    c->bp.memo_old.release(s);
    c->bp.vpa_old.release(s);
    c->bp.vpb_old.release(s);
    c->bp.pv.release(s);
    release(c->lcp, s);
    release(c->scan, s);
    release(c->bp.scan, s);
    mlp_release(c->mlp, s);
    cudaStreamSynchronize(s);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    if (c->hstep) cudaFreeHost(c->hstep);
    if (c->hup) cudaFreeHost(c->hup);
    if (c->hstage) cudaFreeHost(c->hstage);
    if (c->hcheck) cudaFreeHost(c->hcheck);
    delete c;
}

// ---------------------------------------------------------------------------
// stateless entry points
// ---------------------------------------------------------------------------
relcp_status relcp_broadphase(int64_t n, const double* x, const double* rb, const double* box3, double skin,
                              int32_t* pairs, int64_t cap, int64_t* n_out, void* stream) {
    if (!n_out || !box3 || (n > 0 && (!x || !rb))) return set_error("NULL argument"), RELCP_ERR_INVALID_ARG;
    if (n < 0 || !(skin >= 0)) return set_error("bad n or skin"), RELCP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    BroadphaseScratch sc;
    DBuf<int> pa, pb;
    int64_t np = 0;
    relcp_status st = broadphase(n, View<3, const double>::aos(x, 3), rb, 0.0, box3, skin, pa, pb, &np, sc, s);
    if (st == RELCP_OK) st = scan_error(sc.scan, s);
    *n_out = np;
    if (st == RELCP_OK && np > cap) st = RELCP_ERR_CAPACITY;
    if (st == RELCP_OK && np > 0) {
        cudaError_t e1 = cudaMemcpy2DAsync(pairs, 2 * sizeof(int), pa.p, sizeof(int), sizeof(int), np,
                                           cudaMemcpyDeviceToDevice, s);
        cudaError_t e2 = cudaMemcpy2DAsync(pairs + 1, 2 * sizeof(int), pb.p, sizeof(int), sizeof(int), np,
                                           cudaMemcpyDeviceToDevice, s);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            set_error("pair copy failed: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
            st = RELCP_ERR_CUDA;
        }
    }
    DBuf<int>* bufs[] = {&pa, &pb, &sc.cell_of, &sc.cell_count, &sc.cell_start, &sc.cell_cursor, &sc.cell_body,
                         &sc.pair_count, &sc.pair_off};
    for (auto* b : bufs) b->release(s);
    release(sc.scan, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == RELCP_OK) st = RELCP_ERR_CUDA;
    return st;
}

relcp_status relcp_snsd_eval(int64_t npairs, const int32_t* pairs, int64_t n, const double* x, const double* q,
                             const double* axes, const double* box3, int32_t precision, double* out, int32_t* iters,
                             void* stream) {
    if (npairs < 0 || n < 0 || !box3 || (npairs > 0 && (!pairs || !x || !q || !axes || !out)))
        return set_error("bad argument"), RELCP_ERR_INVALID_ARG;
    if (precision != RELCP_FP64 && precision != RELCP_MIXED) return set_error("bad precision"), RELCP_ERR_INVALID_ARG;
    if (npairs == 0) return RELCP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<double> P;
    DBuf<int> status;
    RELCP_TRY(P.ensure(6 * (n > 0 ? n : 1), s));
    RELCP_TRY(status.ensure(1, s));
    RELCP_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), s));
    RELCP_TRY(shape_launch(n, View<4, const double>::aos(q, 4), View<3, const double>::aos(axes, 3),
                           View<6, double>::soa(P.p, n), s));
    SnsdArgs a{};
    a.npairs = npairs;
    a.pa = pairs;
    a.pb = pairs + 1;
    a.pstride = 2;
    a.x = View<3, const double>::aos(x, 3);
    a.P = View<6, const double>::soa(P.p, n);
    for (int k = 0; k < 3; ++k) a.box[k] = box3[k];
    a.guess.c[0] = a.guess.c[1] = a.guess.c[2] = nullptr;
    a.guess.s = 1;
    a.mixed = precision == RELCP_MIXED;
    a.out.phi = out;
    a.out.phi_s = 10;
    a.out.n = View<3, double>::aos(out + 1, 10);
    a.out.ra = View<3, double>::aos(out + 4, 10);
    a.out.rb = View<3, double>::aos(out + 7, 10);
    a.out.iters = iters;
    a.status = status.p;
    a.maxov_bits = nullptr;
    a.newton_max = nullptr;
    a.iters_sum = nullptr;
    relcp_status st = snsd_launch(a, s);
    int bits = 0;
    if (st == RELCP_OK) {
        RELCP_CUDA(cudaMemcpyAsync(&bits, status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    P.release(s);
    status.release(s);
    RELCP_CUDA(cudaStreamSynchronize(s));
    if (st != RELCP_OK) return st;
    return status_from_device(bits);
}

relcp_status relcp_lcp_solve(int64_t nrows, int64_t nbodies, const int32_t* ia, const int32_t* ib,
                             const double* geom, const double* qv, const double* K, double c, int32_t precision,
                             double tol, int32_t max_iter, double* gamma, double* uc, relcp_lcp_info* info,
                             void* stream) {
    if (nrows < 0 || nbodies < 0 || !info || (nrows > 0 && (!ia || !ib || !geom || !qv || !gamma)) ||
        (nbodies > 0 && (!K || !uc)))
        return set_error("bad argument"), RELCP_ERR_INVALID_ARG;
    if (!(tol > 0) || max_iter < 1 || !(c > 0)) return set_error("tol, c > 0 and max_iter >= 1"), RELCP_ERR_INVALID_ARG;
    if (precision != RELCP_FP64 && precision != RELCP_MIXED) return set_error("bad precision"), RELCP_ERR_INVALID_ARG;
    if (nrows > ((int64_t)1 << 29)) return set_error("too many rows"), RELCP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool mixed = precision == RELCP_MIXED;
    const int64_t m = nrows, nb = nbodies, ma = m > 0 ? m : 1, nba = nb > 0 ? nb : 1;
    // SoA copies of the rows (in the solve precision) and of K; diagonal
    DBuf<double> gd, kd, diag, ucd, gam;
    DBuf<float> gf, gamf, qf, kf;
    DBuf<int> cnt;
    DBuf<LcpDevResult> res;
    DBuf<int> dst;
    LcpScratch sc;
    relcp_status st = RELCP_OK;
    auto fail = [&](relcp_status e) {
        st = e;
        return e;
    };
    do {
        if (fail(gd.ensure(9 * ma, s)) || fail(kd.ensure(7 * nba, s)) || fail(diag.ensure(ma, s)) ||
            fail(ucd.ensure(6 * nba, s)) || fail(cnt.ensure(1, s)) || fail(res.ensure(1, s)) ||
            fail(dst.ensure(1, s)))
            break;
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 9 && e == cudaSuccess && m > 0; ++k)
            e = cudaMemcpy2DAsync(gd.p + k * m, sizeof(double), geom + k, 9 * sizeof(double), sizeof(double), m,
                                  cudaMemcpyDeviceToDevice, s);
        for (int k = 0; k < 7 && e == cudaSuccess && nb > 0; ++k)
            e = cudaMemcpy2DAsync(kd.p + k * nb, sizeof(double), K + k, 7 * sizeof(double), sizeof(double), nb,
                                  cudaMemcpyDeviceToDevice, s);
        int mi = (int)m;
        if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.p, &mi, sizeof(int), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dst.p, 0, sizeof(int), s);
        if (e != cudaSuccess) {
            set_error("%s", cudaGetErrorString(e));
            st = RELCP_ERR_CUDA;
            break;
        }
        if (fail(lcp_diag_launch(m, ia, ib, View<9, const double>::aos(geom, 9), View<7, const double>::aos(K, 7), c,
                                 diag.p, s)))
            break;
        LcpProblem pr{};
        pr.m_cap = m;
        pr.nrows_dev = cnt.p;
        pr.nbodies = nb;
        pr.ia = ia;
        pr.ib = ib;
        if (mixed) {
            if (fail(gf.ensure(9 * ma, s)) || fail(gamf.ensure(ma, s)) || fail(qf.ensure(ma, s)) ||
                fail(kf.ensure(7 * nba, s)))
                break;
            // one-time narrowing of the stateless call's inputs, on the device
            if (nb > 0 && fail(narrow_launch(kd.p, kf.p, 7 * nb, s))) break;
            if (m > 0 && (fail(narrow_launch(gd.p, gf.p, 9 * m, s)) || fail(narrow_launch(gamma, gamf.p, m, s)) ||
                          fail(narrow_launch(qv, qf.p, m, s))))
                break;
            if (e != cudaSuccess) {
                set_error("%s", cudaGetErrorString(e));
                st = RELCP_ERR_CUDA;
                break;
            }
            for (int k = 0; k < 9; ++k) pr.geom[k] = gf.p + k * m;
            pr.gamma = gamf.p;
            pr.qr = qf.p;
            for (int k = 0; k < 7; ++k) pr.Kr[k] = kf.p + k * nb;
        } else {
            if (fail(gam.ensure(ma, s))) break;
            if (m > 0) e = cudaMemcpyAsync(gam.p, gamma, m * sizeof(double), cudaMemcpyDeviceToDevice, s);
            for (int k = 0; k < 9; ++k) pr.geom[k] = gd.p + k * m;
            pr.gamma = gam.p;
            pr.qr = qv;
            for (int k = 0; k < 7; ++k) pr.Kr[k] = kd.p + k * nb;
        }
        pr.q = qv;
        pr.diag = diag.p;
        pr.invd = nullptr;
        for (int k = 0; k < 7; ++k) pr.K[k] = kd.p + k * nb;
        pr.c = c;
        pr.mixed = mixed;
        pr.tol = tol;
        pr.max_iter = max_iter;
        for (int k = 0; k < 6; ++k) pr.uc[k] = ucd.p + k * nb;
        pr.result = res.p;
        pr.status = dst.p;
        pr.ev_before = pr.ev_after = nullptr;
        sc.scan.status = dst.p;  // a prefix-sum timeout is reported like the solver's own
        int blocks = 0;
        float kms = 0.f;
        if (fail(lcp_solve(pr, sc, &blocks, &kms, s))) break;
        LcpDevResult hr{};
        int hst = 0;
        e = cudaMemcpyAsync(&hr, res.p, sizeof(hr), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, dst.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        for (int k = 0; k < 6 && e == cudaSuccess && nb > 0; ++k)
            e = cudaMemcpy2DAsync(uc + k, 6 * sizeof(double), ucd.p + k * nb, sizeof(double), sizeof(double), nb,
                                  cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && m > 0) {
            if (mixed) {
                if (fail(widen_launch(gamf.p, gamma, m, s))) break;
                e = cudaStreamSynchronize(s);
            } else {
                e = cudaMemcpyAsync(gamma, gam.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s);
            }
        }
        if (e != cudaSuccess) {
            set_error("%s", cudaGetErrorString(e));
            st = RELCP_ERR_CUDA;
            break;
        }
        info->iterations = (int)hr.iterations;
        info->residual = hr.residual;
        info->grid_blocks = blocks;
        info->status = status_from_device(hst);
        // the kernel's rule for one grid barrier per iteration (mixed path,
        // every row in a thread slot of its own)
        info->one_barrier = (mixed && m <= (int64_t)blocks * lcp_threads()) ? 1 : 0;
    } while (0);
    gd.release(s);
    kd.release(s);
    diag.release(s);
    ucd.release(s);
    gam.release(s);
    gf.release(s);
    gamf.release(s);
    qf.release(s);
    kf.release(s);
    cnt.release(s);
    res.release(s);
    dst.release(s);
    release(sc, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == RELCP_OK) st = RELCP_ERR_CUDA;
    if (st != RELCP_OK) {
        info->status = st;
        return st;
    }
    return (relcp_status)info->status;
}

}  // extern "C"
