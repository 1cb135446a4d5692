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
#include <cstdarg>
#include <cstring>
#include <string>
#include <vector>

#include "relcp_internal.cuh"
#include "step_kernels.cuh"
#include "mlp.cuh"

namespace relcp {

static thread_local char g_err[1024] = "";
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

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

}  // namespace relcp

using namespace relcp;

struct relcp_ctx {
    relcp_config cfg{};
    cudaStream_t s = nullptr;
    int64_t n = 0;
    bool has_bodies = false;
    double box[3] = {0, 0, 0};
    // body state and per-step body arrays (SoA)
    DBuf<double> x, q, axes, vel, fext, P, K, rb, ufree, uc, ustep, xt, qt, Pt;
    // pairs
    DBuf<int> pa, pb;
    int64_t npairs = 0;
    DBuf<double> s0, s1;  // SNSD outputs at C^k and at the trial (10 x npairs)
    DBuf<int> it0, it1, flags, fscan;
    DBuf<double> blockmax, scal;  // scal: [max overlap]
    DBuf<int> dstatus, imax;
    // rows (capacity rcap, SoA)
    int64_t nrows = 0, nrows0 = 0, rcap = 0;
    DBuf<int> r_ia, r_ib, r_rec, r_pair;
    DBuf<double> r_geom, r_q, r_diag, r_gamma;
    BroadphaseScratch bp;
    LcpScratch lcp;
    ScanScratch scan;
    MlpState mlp;
    relcp_step_stats stats{};
    int64_t steps_done = 0;
};

namespace {

relcp_status check_config(const relcp_config* c) {
    if (!c) return set_error("config is NULL"), RELCP_ERR_INVALID_ARG;
    if (c->dynamics != RELCP_INERTIAL && c->dynamics != RELCP_OVERDAMPED)
        return set_error("dynamics must be RELCP_INERTIAL or RELCP_OVERDAMPED"), RELCP_ERR_INVALID_ARG;
    if (c->precision != RELCP_FP64 && c->precision != RELCP_MIXED)
        return set_error("precision must be RELCP_FP64 or RELCP_MIXED"), RELCP_ERR_INVALID_ARG;
    if (c->guess != RELCP_GUESS_COLD && c->guess != RELCP_GUESS_MLP)
        return set_error("guess must be RELCP_GUESS_COLD or RELCP_GUESS_MLP"), RELCP_ERR_INVALID_ARG;
    if (!(c->dt > 0) || !(c->eps_ncp > 0) || !(c->skin >= 0) || !(c->lcp_tol > 0) || c->lcp_max_iter < 1 ||
        c->max_recursion < 0 || c->max_recursion > 4096)
        return set_error("dt, eps_ncp, lcp_tol > 0; skin >= 0; lcp_max_iter >= 1; 0 <= max_recursion <= 4096"),
               RELCP_ERR_INVALID_ARG;
    if (c->dynamics == RELCP_OVERDAMPED && !(c->drag_xi > 0))
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

relcp_status grow_rows(relcp_ctx* c, int64_t need) {
    if (need <= c->rcap) return RELCP_OK;
    int64_t nc = need + need / 2 + 64;
    cudaStream_t s = c->s;
    DBuf<int> ia, ib, rec, pair;
    DBuf<double> geom, q, diag, gamma;
    RELCP_TRY(ia.ensure(nc, s));
    RELCP_TRY(ib.ensure(nc, s));
    RELCP_TRY(rec.ensure(nc, s));
    RELCP_TRY(pair.ensure(nc, s));
    RELCP_TRY(geom.ensure(9 * nc, s));
    RELCP_TRY(q.ensure(nc, s));
    RELCP_TRY(diag.ensure(nc, s));
    RELCP_TRY(gamma.ensure(nc, s));
    // ensure() over-allocates; the logical capacity is nc
    if (c->nrows > 0) {
        int64_t m = c->nrows;
        RELCP_CUDA(cudaMemcpyAsync(ia.p, c->r_ia.p, m * sizeof(int), cudaMemcpyDeviceToDevice, s));
        RELCP_CUDA(cudaMemcpyAsync(ib.p, c->r_ib.p, m * sizeof(int), cudaMemcpyDeviceToDevice, s));
        RELCP_CUDA(cudaMemcpyAsync(rec.p, c->r_rec.p, m * sizeof(int), cudaMemcpyDeviceToDevice, s));
        RELCP_CUDA(cudaMemcpyAsync(pair.p, c->r_pair.p, m * sizeof(int), cudaMemcpyDeviceToDevice, s));
        for (int k = 0; k < 9; ++k)
            RELCP_CUDA(cudaMemcpyAsync(geom.p + k * nc, c->r_geom.p + k * c->rcap, m * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
        RELCP_CUDA(cudaMemcpyAsync(q.p, c->r_q.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
        RELCP_CUDA(cudaMemcpyAsync(diag.p, c->r_diag.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
        RELCP_CUDA(cudaMemcpyAsync(gamma.p, c->r_gamma.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    c->r_ia.release(s);
    c->r_ib.release(s);
    c->r_rec.release(s);
    c->r_pair.release(s);
    c->r_geom.release(s);
    c->r_q.release(s);
    c->r_diag.release(s);
    c->r_gamma.release(s);
    c->r_ia = ia;
    c->r_ib = ib;
    c->r_rec = rec;
    c->r_pair = pair;
    c->r_geom = geom;
    c->r_q = q;
    c->r_diag = diag;
    c->r_gamma = gamma;
    c->rcap = nc;
    return RELCP_OK;
}

struct PhaseTimer {
    static constexpr int kMaxEv = 512;
    bool on = false;
    cudaStream_t s{};
    cudaEvent_t ev[kMaxEv];
    int k = 0;
    relcp_status start(bool enable, cudaStream_t st) {
        on = enable;
        s = st;
        k = 0;
        if (!on) return RELCP_OK;
        for (int i = 0; i < kMaxEv; ++i) RELCP_CUDA(cudaEventCreate(&ev[i]));
        return RELCP_OK;
    }
    int mark() {
        if (!on || k >= kMaxEv) return -1;
        cudaEventRecord(ev[k], s);
        return k++;
    }
    float ms(int a, int b) {
        float t = 0.f;
        if (on && a >= 0 && b >= 0) cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
    void stop() {
        if (on)
            for (int i = 0; i < kMaxEv; ++i) cudaEventDestroy(ev[i]);
        on = false;
    }
};

relcp_status step_once(relcp_ctx* c) {
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
    RELCP_TRY(tm.start((cfg.flags & RELCP_FLAG_PHASE_TIMING) != 0, s));
    std::vector<std::pair<int, int>> snsd_marks;
    int t_begin = tm.mark();
    RELCP_CUDA(cudaMemsetAsync(c->dstatus.p, 0, sizeof(int), s));
    RELCP_CUDA(cudaMemsetAsync(c->imax.p, 0, sizeof(int), s));

    // bodies: normalised q, P, K, rb, U_free
    PrepArgs pa{};
    pa.n = n;
    pa.dynamics = cfg.dynamics;
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
    pa.rb = c->rb.p;
    pa.ufree = c->ufree.p;
    RELCP_TRY(prep_launch(pa, s));

    // broad phase
    View<3, const double> xv = View<3, const double>::soa(c->x.p, n);
    RELCP_TRY(broadphase(n, xv, c->rb.p, box0, cfg.skin, c->pa, c->pb, &c->npairs, c->bp, s));
    const int64_t np = c->npairs;
    st.n_pairs = np;
    int t_bp = tm.mark();
    const int64_t npa = np > 0 ? np : 1;
    RELCP_TRY(c->s0.ensure(10 * npa, s));
    RELCP_TRY(c->s1.ensure(10 * npa, s));
    RELCP_TRY(c->it0.ensure(npa, s));
    RELCP_TRY(c->it1.ensure(npa, s));
    RELCP_TRY(c->flags.ensure(npa, s));
    RELCP_TRY(c->fscan.ensure(npa + 1, s));
    RELCP_TRY(c->blockmax.ensure(npa / 64 + 8, s));

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

    // SNSD at C^k
    SnsdArgs sa{};
    sa.npairs = np;
    sa.pa = c->pa.p;
    sa.pb = c->pb.p;
    sa.pstride = 1;
    sa.x = xv;
    sa.P = View<6, const double>::soa(c->P.p, n);
    for (int k = 0; k < 3; ++k) sa.box[k] = box0[k];
    sa.guess.c[0] = sa.guess.c[1] = sa.guess.c[2] = nullptr;
    sa.guess.s = 1;
    st.guess_used = 0;
    if (cfg.guess == RELCP_GUESS_MLP && c->mlp.loaded && np > 0) {
        RELCP_TRY(mlp_guess(c->mlp, np, c->pa.p, c->pb.p, xv, View<4, const double>::soa(c->q.p, n),
                            View<3, const double>::soa(c->axes.p, n), box0, s));
        sa.guess = View<3, const double>::soa(c->mlp.guess.p, np);
        st.guess_used = 1;
    }
    sa.mixed = mixed ? 1 : 0;
    sa.out = snsd_out(c->s0, c->it0);
    sa.eps = 0.0;
    sa.viol = nullptr;
    sa.block_maxov = nullptr;
    sa.status = c->dstatus.p;
    {
        int e0 = tm.mark();
        RELCP_TRY(snsd_launch(sa, nullptr, s));
        int e1 = tm.mark();
        snsd_marks.push_back({e0, e1});
        st.snsd_evals += tm.on ? np : 0;
    }
    RELCP_TRY(iters_max_launch(np, c->it0.p, c->imax.p, s));
    int t_snsd0 = tm.mark();

    // A_0
    double phi_skin = cfg.phi_skin;
    RELCP_TRY(flag_le_launch(np, c->s0.p, phi_skin, c->flags.p, s));
    RELCP_TRY(exclusive_scan(c->flags.p, c->fscan.p, np, c->scan, s));
    int n0 = 0;
    RELCP_CUDA(cudaMemcpyAsync(&n0, c->fscan.p + np, sizeof(int), cudaMemcpyDeviceToHost, s));
    RELCP_CUDA(cudaStreamSynchronize(s));
    c->nrows = 0;
    if (cfg.fault_inject & RELCP_FAULT_ROW_CAPACITY) {
        set_error("row capacity exhausted (injected fault)");
        tm.stop();
        return RELCP_ERR_CAPACITY;
    }
    RELCP_TRY(grow_rows(c, n0 > 0 ? n0 : 1));
    RowsArgs ra{};
    ra.npairs = np;
    ra.nbodies = n;
    ra.pa = c->pa.p;
    ra.pb = c->pb.p;
    ra.flags = c->flags.p;
    ra.scan = c->fscan.p;
    ra.snsd = c->s0.p;
    ra.base = 0;
    ra.cap = c->rcap;
    ra.rec_index = 0;
    ra.c = dt;
    ra.strain_rate = cfg.strain_rate;
    for (int k = 0; k < 3; ++k) ra.box[k] = box0[k];
    ra.x = c->x.p;
    ra.ufree = c->ufree.p;
    ra.uc = c->uc.p;
    ra.K = c->K.p;
    ra.ia = c->r_ia.p;
    ra.ib = c->r_ib.p;
    ra.rec = c->r_rec.p;
    ra.pair = c->r_pair.p;
    ra.geom = c->r_geom.p;
    ra.q = c->r_q.p;
    ra.diag = c->r_diag.p;
    ra.gamma = c->r_gamma.p;
    ra.status = c->dstatus.p;
    RELCP_TRY(rows_launch(ra, s));
    c->nrows = n0;
    c->nrows0 = n0;
    st.n_rows0 = n0;

    int depth = 0;
    int lcp_iters_total = 0;
    float ms_lcp = 0, ms_aug = 0, ms_snsd = tm.ms(t_bp, t_snsd0);
    relcp_status step_status = RELCP_OK;
    LcpResult lr{};
    double maxov = 0.0;
    for (;;) {
        int t_l0 = tm.mark();
        LcpProblem pr{};
        pr.nrows = c->nrows;
        pr.nbodies = n;
        pr.ia = c->r_ia.p;
        pr.ib = c->r_ib.p;
        for (int k = 0; k < 9; ++k) pr.geom.c[k] = c->r_geom.p + k * c->rcap;
        pr.geom.s = 1;
        pr.q = c->r_q.p;
        pr.diag = c->r_diag.p;
        pr.K = View<7, const double>::soa(c->K.p, n);
        pr.c = dt;
        pr.mixed = mixed ? 1 : 0;
        pr.tol = cfg.lcp_tol;
        pr.max_iter = (cfg.fault_inject & RELCP_FAULT_LCP_ITERS) ? 1 : cfg.lcp_max_iter;
        pr.gamma = c->r_gamma.p;
        pr.uc = View<6, double>::soa(c->uc.p, n);
        pr.time_kernel = tm.on;
        RELCP_TRY(lcp_solve(pr, c->lcp, &lr, s));
        if (tm.on && c->nrows > 0) {
            st.ms_lcp_kernel += lr.kernel_ms;
            st.lcp_alg_bytes += lcp_bytes_per_iter(c->nrows, n, mixed) * (lr.iterations + 1);
            st.lcp_launches += 1;
        }
        if (depth < RELCP_MAX_DEPTH_STATS) {
            st.lcp_iters[depth] = lr.iterations;
            st.rows_per_rec[depth] = (int)c->nrows;
        }
        lcp_iters_total += lr.iterations;
        if (lr.dev_status) {
            relcp_status ls = status_from_device(lr.dev_status);
            if (ls == RELCP_ERR_TIMEOUT) {
                set_error("LCP grid barrier timed out");
                tm.stop();
                return ls;
            }
            if (step_status == RELCP_OK) step_status = ls;
        }
        int t_l1 = tm.mark();
        ms_lcp += tm.ms(t_l0, t_l1);

        // trial configuration and overlap test
        TrialArgs ta{};
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
        RELCP_TRY(trial_launch(ta, s));
        SnsdArgs sb = sa;
        sb.x = View<3, const double>::soa(c->xt.p, n);
        sb.P = View<6, const double>::soa(c->Pt.p, n);
        for (int k = 0; k < 3; ++k) sb.box[k] = box1[k];
        sb.guess = View<3, const double>::soa(c->s0.p + np, np);  // warm start: normals at C^k
        sb.out = snsd_out(c->s1, c->it1);
        sb.eps = cfg.eps_ncp;
        sb.viol = c->flags.p;
        sb.block_maxov = c->blockmax.p;
        int nblocks = 0;
        {
            int e0 = tm.mark();
            RELCP_TRY(snsd_launch(sb, &nblocks, s));
            int e1 = tm.mark();
            snsd_marks.push_back({e0, e1});
            st.snsd_evals += tm.on ? np : 0;
        }
        RELCP_TRY(iters_max_launch(np, c->it1.p, c->imax.p, s));
        RELCP_TRY(max_blocks_launch(np > 0 ? nblocks : 0, c->blockmax.p, c->scal.p, s));
        RELCP_TRY(exclusive_scan(c->flags.p, c->fscan.p, np, c->scan, s));
        int nv = 0;
        RELCP_CUDA(cudaMemcpyAsync(&nv, c->fscan.p + np, sizeof(int), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaMemcpyAsync(&maxov, c->scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaStreamSynchronize(s));
        int t_s1 = tm.mark();
        ms_snsd += tm.ms(t_l1, t_s1);
        if (nv == 0) break;
        if (depth >= cfg.max_recursion) {
            if (step_status == RELCP_OK) step_status = RELCP_ERR_RECURSION_LIMIT;
            break;
        }
        ++depth;
        RELCP_TRY(grow_rows(c, c->nrows + nv));
        RowsArgs rb2 = ra;
        rb2.snsd = c->s1.p;
        rb2.base = c->nrows;
        rb2.cap = c->rcap;
        rb2.rec_index = depth;
        rb2.ia = c->r_ia.p;
        rb2.ib = c->r_ib.p;
        rb2.rec = c->r_rec.p;
        rb2.pair = c->r_pair.p;
        rb2.geom = c->r_geom.p;
        rb2.q = c->r_q.p;
        rb2.diag = c->r_diag.p;
        rb2.gamma = c->r_gamma.p;
        RELCP_TRY(rows_launch(rb2, s));
        c->nrows += nv;
        int t_a = tm.mark();
        ms_aug += tm.ms(t_s1, t_a);
    }

    // accept
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
    RELCP_TRY(accept_launch(aa, s));
    int t_end = tm.mark();
    int dbits = 0, imax = 0;
    RELCP_CUDA(cudaMemcpyAsync(&dbits, c->dstatus.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    RELCP_CUDA(cudaMemcpyAsync(&imax, c->imax.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    RELCP_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < 3; ++k) c->box[k] = box1[k];
    relcp_status ds = status_from_device(dbits);
    if (step_status == RELCP_OK) step_status = ds;
    st.n_rows = c->nrows;
    st.depth = depth;
    st.status = step_status;
    st.lcp_iters_total = lcp_iters_total;
    st.newton_iters_max = imax;
    st.lcp_residual = lr.residual;
    st.max_overlap = maxov;
    for (int k = 0; k < 3; ++k) st.box[k] = c->box[k];
    st.ms_broadphase = tm.ms(t_begin, t_bp);
    st.ms_snsd = ms_snsd;
    st.ms_lcp = ms_lcp;
    st.ms_augment = ms_aug;
    st.ms_total = tm.ms(t_begin, t_end);
    for (auto& mk : snsd_marks) {
        if (mk.first >= 0 && mk.second >= 0) {
            st.ms_snsd_kernel += tm.ms(mk.first, mk.second);
            st.snsd_launches += 1;
        }
    }
    tm.stop();
    c->steps_done += 1;
    st.steps_done = c->steps_done;
    c->stats = st;
    return step_status;
}

relcp_status copy_in(const double* src, int64_t count, int32_t ptr_kind, std::vector<double>& out) {
    out.resize((size_t)count);
    if (count == 0) return RELCP_OK;
    if (ptr_kind == RELCP_PTR_DEVICE) {
        RELCP_CUDA(cudaMemcpy(out.data(), src, count * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(out.data(), src, count * sizeof(double));
    }
    return RELCP_OK;
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
    relcp_status st = c->dstatus.ensure(1, c->s);
    if (st == RELCP_OK) st = c->imax.ensure(1, c->s);
    if (st == RELCP_OK) st = c->scal.ensure(4, c->s);
    if (st != RELCP_OK) {
        delete c;
        return st;
    }
    *out = c;
    return RELCP_OK;
}

relcp_status relcp_set_config(relcp_ctx* c, const relcp_config* cfg) {
    if (!c) return set_error("ctx is NULL"), RELCP_ERR_INVALID_ARG;
    RELCP_TRY(check_config(cfg));
    c->cfg = *cfg;
    for (int k = 0; k < 3; ++k) c->box[k] = cfg->box[k];
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
    std::vector<double> hx, hq, ha, hv, hf;
    RELCP_TRY(copy_in(x, 3 * n, ptr_kind, hx));
    RELCP_TRY(copy_in(q, 4 * n, ptr_kind, hq));
    RELCP_TRY(copy_in(semi_axes, 3 * n, ptr_kind, ha));
    if (vel) RELCP_TRY(copy_in(vel, 6 * n, ptr_kind, hv));
    else hv.assign((size_t)(6 * n), 0.0);
    if (f_ext) RELCP_TRY(copy_in(f_ext, 6 * n, ptr_kind, hf));
    else hf.assign((size_t)(6 * n), 0.0);
    for (int64_t i = 0; i < n; ++i) {
        double qq = 0;
        for (int k = 0; k < 4; ++k) qq += hq[4 * i + k] * hq[4 * i + k];
        if (!(fabs(sqrt(qq) - 1.0) <= 1e-6))
            return set_error("body %lld: quaternion norm %.17g is not 1", (long long)i, sqrt(qq)),
                   RELCP_ERR_INVALID_ARG;
        for (int k = 0; k < 3; ++k) {
            if (!std::isfinite(hx[3 * i + k])) return set_error("body %lld: position not finite", (long long)i), RELCP_ERR_INVALID_ARG;
            if (!(ha[3 * i + k] > 0) || !std::isfinite(ha[3 * i + k]))
                return set_error("body %lld: semi-axes must be finite and > 0", (long long)i), RELCP_ERR_INVALID_ARG;
        }
        for (int k = 0; k < 6; ++k)
            if (!std::isfinite(hv[6 * i + k]) || !std::isfinite(hf[6 * i + k]))
                return set_error("body %lld: velocity / force not finite", (long long)i), RELCP_ERR_INVALID_ARG;
    }
    // transpose to SoA
    auto soa = [&](const std::vector<double>& a, int w) {
        std::vector<double> o((size_t)(w * n));
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < w; ++k) o[(size_t)(k * n + i)] = a[(size_t)(w * i + k)];
        return o;
    };
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
    if (n > 0) {
        std::vector<double> sx = soa(hx, 3), sq = soa(hq, 4), sa = soa(ha, 3), sv = soa(hv, 6), sf = soa(hf, 6);
        RELCP_CUDA(cudaMemcpyAsync(c->x.p, sx.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, s));
        RELCP_CUDA(cudaMemcpyAsync(c->q.p, sq.data(), 4 * n * sizeof(double), cudaMemcpyHostToDevice, s));
        RELCP_CUDA(cudaMemcpyAsync(c->axes.p, sa.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, s));
        RELCP_CUDA(cudaMemcpyAsync(c->vel.p, sv.data(), 6 * n * sizeof(double), cudaMemcpyHostToDevice, s));
        RELCP_CUDA(cudaMemcpyAsync(c->fext.p, sf.data(), 6 * n * sizeof(double), cudaMemcpyHostToDevice, s));
        RELCP_CUDA(cudaMemsetAsync(c->ustep.p, 0, 6 * n * sizeof(double), s));
        for (int k = 0; k < 3; ++k) c->box[k] = c->cfg.box[k];
        RELCP_TRY(wrap_launch(n, c->x.p, c->box, s));
        RELCP_CUDA(cudaStreamSynchronize(s));  // host staging buffers go out of scope
    }
    c->n = n;
    c->has_bodies = true;
    c->steps_done = 0;
    c->nrows = 0;
    c->npairs = 0;
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
    const int64_t n = c->n;
    if (n == 0) return RELCP_OK;
    cudaStream_t s = c->s;
    auto out = [&](const double* dsoa, int w, double* dst) -> relcp_status {
        if (!dst) return RELCP_OK;
        std::vector<double> hs((size_t)(w * n)), ha((size_t)(w * n));
        RELCP_CUDA(cudaMemcpyAsync(hs.data(), dsoa, w * n * sizeof(double), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < w; ++k) ha[(size_t)(w * i + k)] = hs[(size_t)(k * n + i)];
        if (ptr_kind == RELCP_PTR_DEVICE) {
            RELCP_CUDA(cudaMemcpyAsync(dst, ha.data(), w * n * sizeof(double), cudaMemcpyHostToDevice, s));
            RELCP_CUDA(cudaStreamSynchronize(s));
        } else {
            std::memcpy(dst, ha.data(), w * n * sizeof(double));
        }
        return RELCP_OK;
    };
    RELCP_TRY(out(c->x.p, 3, x));
    RELCP_TRY(out(c->q.p, 4, q));
    RELCP_TRY(out(c->steps_done > 0 ? c->ustep.p : c->vel.p, 6, vel));
    return RELCP_OK;
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
    if (gamma) RELCP_CUDA(cudaMemcpyAsync(gamma, c->r_gamma.p, m * sizeof(double), cudaMemcpyDefault, s));
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

void relcp_destroy(relcp_ctx* c) {
    if (!c) return;
    cudaStream_t s = c->s;
    DBuf<double>* dbs[] = {&c->x, &c->q, &c->axes, &c->vel, &c->fext, &c->P, &c->K, &c->rb, &c->ufree, &c->uc,
                           &c->ustep, &c->xt, &c->qt, &c->Pt, &c->s0, &c->s1, &c->blockmax, &c->scal,
                           &c->r_geom, &c->r_q, &c->r_diag, &c->r_gamma, &c->lcp.gamma2, &c->lcp.g2,
                           &c->lcp.partials, &c->lcp.result};
    for (auto* b : dbs) b->release(s);
    DBuf<int>* ibs[] = {&c->pa, &c->pb, &c->it0, &c->it1, &c->flags, &c->fscan, &c->dstatus, &c->imax, &c->r_ia,
                        &c->r_ib, &c->r_rec, &c->r_pair, &c->bp.cell_of, &c->bp.cell_count, &c->bp.cell_start,
                        &c->bp.cell_cursor, &c->bp.cell_body, &c->bp.pair_count, &c->bp.pair_off,
                        &c->bp.scan.partial, &c->lcp.inc_count, &c->lcp.inc_off, &c->lcp.inc_cursor, &c->lcp.inc,
                        &c->lcp.status, &c->lcp.scan.partial, &c->scan.partial};
    for (auto* b : ibs) b->release(s);
    DBuf<float>* fbs[] = {&c->lcp.gammaf, &c->lcp.gf, &c->lcp.ucf, &c->lcp.geomf};
    for (auto* b : fbs) b->release(s);
    c->lcp.barrier.release(s);
    mlp_release(c->mlp, s);
    cudaStreamSynchronize(s);
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
    relcp_status st = broadphase(n, View<3, const double>::aos(x, 3), rb, box3, skin, pa, pb, &np, sc, s);
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
                         &sc.pair_count, &sc.pair_off, &sc.scan.partial};
    for (auto* b : bufs) b->release(s);
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
    relcp_status st = snsd_launch(a, nullptr, s);
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
    cudaStream_t s = (cudaStream_t)stream;
    LcpScratch sc;
    LcpProblem pr{};
    pr.nrows = nrows;
    pr.nbodies = nbodies;
    pr.ia = ia;
    pr.ib = ib;
    pr.geom = View<9, const double>::aos(geom, 9);
    pr.q = qv;
    pr.diag = nullptr;
    pr.K = View<7, const double>::aos(K, 7);
    pr.c = c;
    pr.mixed = precision == RELCP_MIXED;
    pr.tol = tol;
    pr.max_iter = max_iter;
    pr.gamma = gamma;
    pr.uc = View<6, double>::aos(uc, 6);
    LcpResult lr{};
    relcp_status st = lcp_solve(pr, sc, &lr, s);
    DBuf<int>* ib_[] = {&sc.inc_count, &sc.inc_off, &sc.inc_cursor, &sc.inc, &sc.status, &sc.scan.partial};
    for (auto* b : ib_) b->release(s);
    DBuf<double>* db_[] = {&sc.gamma2, &sc.g2, &sc.partials, &sc.result};
    for (auto* b : db_) b->release(s);
    DBuf<float>* fb_[] = {&sc.gammaf, &sc.gf, &sc.ucf, &sc.geomf};
    for (auto* b : fb_) b->release(s);
    sc.barrier.release(s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == RELCP_OK) st = RELCP_ERR_CUDA;
    info->iterations = lr.iterations;
    info->residual = lr.residual;
    info->grid_blocks = lr.blocks;
    info->status = st != RELCP_OK ? st : status_from_device(lr.dev_status);
    info->pad = 0;
    if (st != RELCP_OK) return st;
    return (relcp_status)info->status;
}

}  // extern "C"
