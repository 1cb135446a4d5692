// Broad phase: candidate ("near-contacting", Algorithm 1 initialisation)
// pairs i < j whose bounding spheres grown by `skin` overlap under the
// periodic minimum image.
//
// Fully periodic boxes with at least three cells per axis use a cell list:
// cell side >= 2 max(rb) + skin, counting sort of bodies into cells (count,
// exclusive scan, fill), then one thread per body i scans the 27 neighbour
// cells for j > i.  Other cases (open axes, small scenes) test all j > i.
// Either way a first pass counts the pairs of each i, a scan gives each i
// its output segment, and a second pass writes the segment and sorts it by
// j, so the list is i-major with j ascending and independent of atomics.
//
// The distance test is a fixed sequence of separately rounded FP64
// operations (no contraction), so the decision is reproducible bit for bit.
// The cached list's per-step filter takes that decision through
// near_pair_fast: FP32 where a rounding-error bound certifies it, the FP64
// test for the pairs within the bound of the cutoff.
//
// The cached Verlet list's rebuild needs only a superset of the pairs within
// the grown cutoff (every step filters the list with the exact test), so with
// `superset` the cell-list passes test in FP32 (this part issues FP64 at a
// small fraction of the FP32 rate) against the cutoff plus a margin m that
// bounds the FP32 error: positions wrapped into [0, L) and rounded to FP32,
// differences, the minimum image and the sum of squares err by less than
// 8 2^-24 L in the distance, and m = 4e-6 (max L + 2 max rb + skin) is more than
// eight times that.  A pair the FP32 rounding could misjudge lies within m of
// the cutoff and is kept.
#include <utility>

#include "relcp_internal.cuh"
#include "scan_tile.cuh"

namespace relcp {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool near_pair(View<3, const double> x, const double* __restrict__ rb, int64_t i,
                                          int64_t j, double L0, double L1, double L2, double skin) {
    return near_pair_exact(x(0, i), x(1, i), x(2, i), x(0, j), x(1, j), x(2, j), rb[i], rb[j], L0, L1, L2, skin);
}

__global__ void brute_count(int64_t n, View<3, const double> x, const double* __restrict__ rb, double L0,
                            double L1, double L2, double skin, int* __restrict__ count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int64_t j = i + 1; j < n; ++j) c += near_pair(x, rb, i, j, L0, L1, L2, skin) ? 1 : 0;
    count[i] = c;
}

__global__ void brute_fill(int64_t n, View<3, const double> x, const double* __restrict__ rb, double L0,
                           double L1, double L2, double skin, const int* __restrict__ off, int* __restrict__ pa,
                           int* __restrict__ pb) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = off[i];
    for (int64_t j = i + 1; j < n; ++j)
        if (near_pair(x, rb, i, j, L0, L1, L2, skin)) {
            pa[o] = (int)i;
            pb[o] = (int)j;
            ++o;
        }
}

struct Grid {
    int nc[3];
    double inv_cs[3];
    double L[3];
};

__device__ __forceinline__ int cell_coord(double v, double L, double inv_cs, int nc) {
    double w = v - L * floor(v / L);  // wrap into [0, L)
    int c = (int)floor(w * inv_cs);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void cell_assign(int64_t n, View<3, const double> x, Grid g, int* __restrict__ cell_of,
                            int* __restrict__ cell_count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx = cell_coord(x(0, i), g.L[0], g.inv_cs[0], g.nc[0]);
    int cy = cell_coord(x(1, i), g.L[1], g.inv_cs[1], g.nc[1]);
    int cz = cell_coord(x(2, i), g.L[2], g.inv_cs[2], g.nc[2]);
    int cid = (cz * g.nc[1] + cy) * g.nc[0] + cx;
    cell_of[i] = cid;
    atomicAdd(&cell_count[cid], 1);
}

// a body's position wrapped into [0, L) per axis and rounded to FP32, with its
// bounding radius (the superset test's operands)
__device__ __forceinline__ float4 wrapped_f32(View<3, const double> x, const double* __restrict__ rb, const Grid& g,
                                              int64_t i) {
    float w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double v = x(k, i);
        w[k] = (float)(v - g.L[k] * floor(v / g.L[k]));
    }
    return make_float4(w[0], w[1], w[2], (float)rb[i]);
}

// xr (optional): the bodies' wrapped_f32 records in cell order, for the
// superset test's contiguous loads
__global__ void cell_fill(int64_t n, const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                          int* __restrict__ cursor, int* __restrict__ cell_body, View<3, const double> x,
                          const double* __restrict__ rb, Grid g, float4* __restrict__ xr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cid = cell_of[i];
    int slot = atomicAdd(&cursor[cid], 1);
    cell_body[cell_start[cid] + slot] = (int)i;
    if (xr) xr[cell_start[cid] + slot] = wrapped_f32(x, rb, g, i);
}

__device__ __forceinline__ float min_image_f32(float d, float L, float invL) { return d - L * rintf(d * invL); }

// SUPERSET: the FP32 test against (rb_i + rb_j + skin + margin) on the cell-
// ordered records xr; otherwise the exact FP64 test
template <bool FILL, bool SUPERSET>
__global__ void cell_pairs(int64_t n, View<3, const double> x, const double* __restrict__ rb, Grid g, double skin,
                           const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                           const int* __restrict__ cell_body, int* __restrict__ count, const int* __restrict__ off,
                           int* __restrict__ pa, int* __restrict__ pb, const float4* __restrict__ xr,
                           float margin) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    float Lf[3] = {0.f, 0.f, 0.f}, iLf[3] = {0.f, 0.f, 0.f}, sk = 0.f;
    if (SUPERSET) {
        xi = wrapped_f32(x, rb, g, i);
        for (int k = 0; k < 3; ++k) {
            Lf[k] = (float)g.L[k];
            iLf[k] = (float)(1.0 / g.L[k]);
        }
        sk = (float)skin + margin;
    }
    int cid = cell_of[i];
    int cx = cid % g.nc[0];
    int cy = (cid / g.nc[0]) % g.nc[1];
    int cz = cid / (g.nc[0] * g.nc[1]);
    int c = 0;
    int o = FILL ? off[i] : 0;
    for (int dz = -1; dz <= 1; ++dz) {
        int z = cz + dz;
        z = z < 0 ? z + g.nc[2] : (z >= g.nc[2] ? z - g.nc[2] : z);
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            y = y < 0 ? y + g.nc[1] : (y >= g.nc[1] ? y - g.nc[1] : y);
            for (int dx = -1; dx <= 1; ++dx) {
                int xx = cx + dx;
                xx = xx < 0 ? xx + g.nc[0] : (xx >= g.nc[0] ? xx - g.nc[0] : xx);
                int nb = (z * g.nc[1] + y) * g.nc[0] + xx;
                int e = cell_start[nb + 1];
                for (int k = cell_start[nb]; k < e; ++k) {
                    int j = cell_body[k];
                    if (j <= i) continue;
                    bool near;
                    if (SUPERSET) {
                        const float4 xj = xr[k];
                        const float dx = min_image_f32(xj.x - xi.x, Lf[0], iLf[0]);
                        const float dy = min_image_f32(xj.y - xi.y, Lf[1], iLf[1]);
                        const float dz = min_image_f32(xj.z - xi.z, Lf[2], iLf[2]);
                        const float r = xi.w + xj.w + sk;
                        near = dx * dx + dy * dy + dz * dz <= r * r;
                    } else {
                        near = near_pair(x, rb, i, j, g.L[0], g.L[1], g.L[2], skin);
                    }
                    if (near) {
                        if (FILL) {
                            pa[o + c] = (int)i;
                            pb[o + c] = j;
                        }
                        ++c;
                    }
                }
            }
        }
    }
    if (!FILL) {
        count[i] = c;
    } else {
        // insertion sort of this body's segment by j
        for (int a = 1; a < c; ++a) {
            int v = pb[o + a];
            int b = a - 1;
            while (b >= 0 && pb[o + b] > v) {
                pb[o + b + 1] = pb[o + b];
                --b;
            }
            pb[o + b + 1] = v;
        }
    }
}

__global__ void max_reduce(int64_t n, const double* __restrict__ v, double* __restrict__ out) {
    __shared__ double sh[32];
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) *out = m;
    }
}

// largest displacement of a body since the Verlet build, the affine box
// scaling s = L / Lb (per periodic axis) taken out: |min_image(x - s xb)|
__global__ void disp_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ xb, double s0,
                            double s1, double s2, double L0, double L1, double L2, unsigned long long* dmax) {
    pdl_wait();
    pdl_trigger();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0;
    if (i < n) {
        const double sc[3] = {s0, s1, s2}, L[3] = {L0, L1, L2};
        for (int k = 0; k < 3; ++k) {
            double d = min_image(x[k * n + i] - sc[k] * xb[k * n + i], L[k]);
            d2 += d * d;
        }
    }
    double d = sqrt(d2);
    for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dmax, (unsigned long long)__double_as_longlong(d));
}

// exact candidate test on the cached list (same operations as near_pair)
__global__ void filter_kernel(int64_t nv, const int* __restrict__ vpa, const int* __restrict__ vpb,
                              View<3, const double> x, const double* __restrict__ rb, double L0, double L1,
                              double L2, const double* __restrict__ Ldev, double skin, int* __restrict__ flag) {
    pdl_wait();
    pdl_trigger();
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nv) return;
    if (Ldev) {
        L0 = Ldev[0];
        L1 = Ldev[1];
        L2 = Ldev[2];
    }
    const float Lf[3] = {trunc_f32(L0), trunc_f32(L1), trunc_f32(L2)};
    const float iLf[3] = {Lf[0] > 0.f ? 1.f / Lf[0] : 0.f, Lf[1] > 0.f ? 1.f / Lf[1] : 0.f,
                          Lf[2] > 0.f ? 1.f / Lf[2] : 0.f};
    const int i = vpa[p], j = vpb[p];
    flag[p] = near_pair_fast(x(0, i), x(1, i), x(2, i), x(0, j), x(1, j), x(2, j), rb[i], rb[j], L0, L1, L2, skin, Lf,
                             iLf, fmaxf(Lf[0], fmaxf(Lf[1], Lf[2])), trunc_f32(skin))
                  ? 1
                  : 0;
}

// The cached list's exact filter, the prefix sum of its flags and the
// compaction in one pass: each block takes a tile of kFcThreads x kFcItems
// entries (entry e of the tile's k-th round at tile base + k kFcThreads +
// thread, so the loads coalesce), tests them, scans the flags across the
// device by look-back (scan_tile.cuh) and writes the surviving entries in
// list order, exactly as the filter, scan and compaction kernels do apart.
// The last tile writes the count to *count_out (and *count_copy).
constexpr int kFcThreads = 512, kFcItems = 2, kFcTile = kFcThreads * kFcItems;
__global__ void __launch_bounds__(kFcThreads)
    filter_compact_kernel(int64_t nv, const int* __restrict__ vpa, const int* __restrict__ vpb,
                          View<3, const double> x, const double* __restrict__ rb, const double* __restrict__ Ldev,
                          double L0, double L1, double L2, double skin, int* __restrict__ pa, int* __restrict__ pb,
                          int* __restrict__ pv, int* count_out, int* count_copy, unsigned long long* tiles, int* ctr,
                          int* status) {
    pdl_wait();
    pdl_trigger();
    __shared__ int fl[kFcTile];
    const int t = tile_scan::take_ticket(ctr);
    const int64_t base = (int64_t)t * kFcTile;
    if (Ldev) {
        L0 = Ldev[0];
        L1 = Ldev[1];
        L2 = Ldev[2];
    }
    int ia[kFcItems], ib[kFcItems];
    bool f[kFcItems];
#pragma unroll
    for (int k = 0; k < kFcItems; ++k) {
        const int64_t e = base + k * kFcThreads + threadIdx.x;
        ia[k] = ib[k] = 0;
        if (e < nv) {
            ia[k] = vpa[e];
            ib[k] = vpb[e];
        }
    }
    const float Lf[3] = {trunc_f32(L0), trunc_f32(L1), trunc_f32(L2)};
    const float iLf[3] = {Lf[0] > 0.f ? 1.f / Lf[0] : 0.f, Lf[1] > 0.f ? 1.f / Lf[1] : 0.f,
                          Lf[2] > 0.f ? 1.f / Lf[2] : 0.f};
    const float Lmaxf = fmaxf(Lf[0], fmaxf(Lf[1], Lf[2])), skinf = trunc_f32(skin);
#pragma unroll
    for (int k = 0; k < kFcItems; ++k) {
        const int64_t e = base + k * kFcThreads + threadIdx.x;
        f[k] = e < nv && near_pair_fast(x(0, ia[k]), x(1, ia[k]), x(2, ia[k]), x(0, ib[k]), x(1, ib[k]), x(2, ib[k]),
                                        rb[ia[k]], rb[ib[k]], L0, L1, L2, skin, Lf, iLf, Lmaxf, skinf);
        fl[k * kFcThreads + threadIdx.x] = f[k] ? 1 : 0;
    }
    __syncthreads();
    // thread r scans the tile's entries r kFcItems .. r kFcItems + kFcItems - 1
    int my[kFcItems], c = 0;
#pragma unroll
    for (int k = 0; k < kFcItems; ++k) {
        my[k] = fl[threadIdx.x * kFcItems + k];
        c += my[k];
    }
    int tot;
    const int inc = tile_scan::block_inclusive_scan(c, &tot);
    const int excl = tile_scan::tile_prefix(t, tot, tiles, status);
    int run = excl + inc - c;
#pragma unroll
    for (int k = 0; k < kFcItems; ++k) {
        fl[threadIdx.x * kFcItems + k] = run;  // each thread rewrites only the words it read
        run += my[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kFcItems; ++k) {
        const int64_t e = base + k * kFcThreads + threadIdx.x;
        if (f[k]) {
            const int p = fl[k * kFcThreads + threadIdx.x];
            pa[p] = ia[k];
            pb[p] = ib[k];
            pv[p] = (int)e;
        }
    }
    if (t == (int)gridDim.x - 1 && threadIdx.x == 0) {
        *count_out = excl + tot;
        if (count_copy) *count_copy = excl + tot;
    }
    tile_scan::tile_finish(tiles, ctr);
}

__global__ void compact_kernel(int64_t nv, const int* __restrict__ vpa, const int* __restrict__ vpb,
                               const int* __restrict__ flag, const int* __restrict__ pos, int* __restrict__ pa,
                               int* __restrict__ pb, int* __restrict__ pv) {
    pdl_wait();
    pdl_trigger();
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv || !flag[v]) return;
    pa[pos[v]] = vpa[v];
    pb[pos[v]] = vpb[v];
    pv[pos[v]] = (int)v;
}

// carry the memo of every pair that is in both the old and the new cached
// list (both sorted by (i, j)) to its new entry; new pairs get stamp -1
__global__ void memo_remap_kernel(int64_t nv, const int* __restrict__ vpa, const int* __restrict__ vpb,
                                  int64_t nold, const int* __restrict__ opa, const int* __restrict__ opb,
                                  const PairMemo* __restrict__ omemo, PairMemo* __restrict__ memo) {
    pdl_wait();
    pdl_trigger();
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const long long key = ((long long)vpa[v] << 32) | (long long)(unsigned)vpb[v];
    int64_t lo = 0, hi = nold;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const long long km = ((long long)opa[mid] << 32) | (long long)(unsigned)opb[mid];
        if (km < key) lo = mid + 1;
        else hi = mid;
    }
    PairMemo m;
    m.stamp = -1;
    m.pidx = -1;
    m.gamma = 0.0;
    if (lo < nold && opa[lo] == vpa[v] && opb[lo] == vpb[v]) m = omemo[lo];
    memo[v] = m;
}

}  // namespace

relcp_status broadphase(int64_t n, View<3, const double> x, const double* rb, double rbmax_hint, const double box[3],
                        double skin, DBuf<int>& pa, DBuf<int>& pb, int64_t* npairs, BroadphaseScratch& sc,
                        cudaStream_t s, bool superset) {
    *npairs = 0;
    if (n < 2) return RELCP_OK;
    unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    RELCP_TRY(sc.pair_count.ensure((size_t)n, s));
    RELCP_TRY(sc.pair_off.ensure((size_t)n + 1, s));

    bool periodic = box[0] > 0 && box[1] > 0 && box[2] > 0;
    Grid g{};
    bool use_cells = false;
    float margin = 0.f;  // the superset test's margin (cell path only)
    if (periodic && n > 2048) {
        // largest bounding radius decides the cell side
        double rbmax = rbmax_hint;
        if (!(rbmax > 0.0)) {
            DBuf<double> mx;
            RELCP_TRY(mx.ensure(1, s));
            note_launch();
            max_reduce<<<1, 1024, 0, s>>>(n, rb, mx.p);
            RELCP_CUDA(cudaGetLastError());
            RELCP_CUDA(cudaMemcpyAsync(&rbmax, mx.p, sizeof(double), cudaMemcpyDeviceToHost, s));
            RELCP_CUDA(cudaStreamSynchronize(s));
            mx.release(s);
        }
        double cut = (2.0 * rbmax + skin) * (1.0 + 1e-9);
        use_cells = true;
        int64_t ncells = 1;
        for (int k = 0; k < 3; ++k) {
            int nc = (int)floor(box[k] / cut);
            if (nc < 3) use_cells = false;
            nc = nc > 1024 ? 1024 : nc;
            g.nc[k] = nc;
            g.L[k] = box[k];
            g.inv_cs[k] = nc / box[k];
            ncells *= nc > 0 ? nc : 1;
        }
        if (use_cells) {
            RELCP_TRY(sc.cell_of.ensure((size_t)n, s));
            RELCP_TRY(sc.cell_count.ensure((size_t)ncells, s));
            RELCP_TRY(sc.cell_cursor.ensure((size_t)ncells, s));
            RELCP_TRY(sc.cell_start.ensure((size_t)ncells + 1, s));
            RELCP_TRY(sc.cell_body.ensure((size_t)n, s));
            RELCP_CUDA(cudaMemsetAsync(sc.cell_count.p, 0, ncells * sizeof(int), s));
            RELCP_CUDA(cudaMemsetAsync(sc.cell_cursor.p, 0, ncells * sizeof(int), s));
            note_launch();
            cell_assign<<<nb, kThreads, 0, s>>>(n, x, g, sc.cell_of.p, sc.cell_count.p);
            RELCP_CUDA(cudaGetLastError());
            RELCP_TRY(exclusive_scan(sc.cell_count.p, sc.cell_start.p, ncells, sc.scan, s));
            if (superset) {
                RELCP_TRY(sc.cell_xr.ensure((size_t)n, s));
                margin = (float)(4e-6 * (fmax(box[0], fmax(box[1], box[2])) + 2.0 * rbmax + skin));
            }
            note_launch();
            cell_fill<<<nb, kThreads, 0, s>>>(n, sc.cell_of.p, sc.cell_start.p, sc.cell_cursor.p, sc.cell_body.p, x, rb,
                                              g, superset ? sc.cell_xr.p : nullptr);
            RELCP_CUDA(cudaGetLastError());
            note_launch();
            if (superset)
                cell_pairs<false, true><<<nb, kThreads, 0, s>>>(n, x, rb, g, skin, sc.cell_of.p, sc.cell_start.p,
                                                                sc.cell_body.p, sc.pair_count.p, nullptr, nullptr,
                                                                nullptr, sc.cell_xr.p, margin);
            else
                cell_pairs<false, false><<<nb, kThreads, 0, s>>>(n, x, rb, g, skin, sc.cell_of.p, sc.cell_start.p,
                                                                 sc.cell_body.p, sc.pair_count.p, nullptr, nullptr,
                                                                 nullptr, nullptr, 0.f);
            RELCP_CUDA(cudaGetLastError());
        }
    }
    if (!use_cells) {
        note_launch();
        brute_count<<<nb, kThreads, 0, s>>>(n, x, rb, box[0], box[1], box[2], skin, sc.pair_count.p);
        RELCP_CUDA(cudaGetLastError());
    }
    RELCP_TRY(exclusive_scan(sc.pair_count.p, sc.pair_off.p, n, sc.scan, s));
    int total = 0;
    RELCP_CUDA(cudaMemcpyAsync(&total, sc.pair_off.p + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    RELCP_CUDA(cudaStreamSynchronize(s));
    if (total < 0 || (int64_t)total > n * (n - 1) / 2) {
        set_error("broad phase: inconsistent pair count %d", total);
        return RELCP_ERR_TIMEOUT;
    }
    *npairs = total;
    if (total == 0) return RELCP_OK;
    RELCP_TRY(pa.ensure((size_t)total, s));
    RELCP_TRY(pb.ensure((size_t)total, s));
    if (use_cells) {
        note_launch();
        if (superset)
            cell_pairs<true, true><<<nb, kThreads, 0, s>>>(n, x, rb, g, skin, sc.cell_of.p, sc.cell_start.p,
                                                           sc.cell_body.p, nullptr, sc.pair_off.p, pa.p, pb.p,
                                                           sc.cell_xr.p, margin);
        else
            cell_pairs<true, false><<<nb, kThreads, 0, s>>>(n, x, rb, g, skin, sc.cell_of.p, sc.cell_start.p,
                                                            sc.cell_body.p, nullptr, sc.pair_off.p, pa.p, pb.p,
                                                            nullptr, 0.f);
    } else {
        note_launch();
        brute_fill<<<nb, kThreads, 0, s>>>(n, x, rb, box[0], box[1], box[2], skin, sc.pair_off.p, pa.p, pb.p);
    }
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

}  // namespace relcp

namespace relcp {

relcp_status broadphase_cached(int64_t n, const double* x_soa, const double* rb, double rbmax, const double box[3],
                               double skin, DBuf<int>& pa, DBuf<int>& pb, int64_t* npairs, BroadphaseScratch& sc,
                               cudaStream_t s) {
    *npairs = 0;
    if (n < 2) return RELCP_OK;
    const unsigned nbk = (unsigned)((n + kThreads - 1) / kThreads);
    View<3, const double> xv = View<3, const double>::soa(x_soa, n);
    const double cutmax = 2.0 * rbmax + skin;
    if (sc.vn_bodies != n || sc.skin_b != skin) sc.valid = false;
    for (int attempt = 0; attempt < 2; ++attempt) {
        double sfac[3] = {1.0, 1.0, 1.0};
        bool geom_ok = sc.valid;
        for (int k = 0; k < 3 && geom_ok; ++k) {
            if ((box[k] > 0) != (sc.Lb[k] > 0)) geom_ok = false;
            else if (box[k] > 0) sfac[k] = box[k] / sc.Lb[k];
        }
        if (!geom_ok) {
            // rebuild: candidates within R_i + R_j + skin + delta at the current
            // positions; the memo follows the pairs that stay in the list
            const int64_t nold = (sc.vn_bodies == n) ? sc.vn : 0;
            std::swap(sc.vpa, sc.vpa_old);
            std::swap(sc.vpb, sc.vpb_old);
            std::swap(sc.memo, sc.memo_old);
            sc.delta = 0.15 * cutmax;
            int64_t nv = 0;
            RELCP_TRY(broadphase(n, xv, rb, rbmax, box, skin + sc.delta, sc.vpa, sc.vpb, &nv, sc, s, true));
            sc.vn = nv;
            RELCP_TRY(sc.memo.ensure((size_t)(nv > 0 ? nv : 1), s));
            if (nv > 0) {
                note_launch();
                launch_pdl(memo_remap_kernel, dim3((unsigned)((nv + kThreads - 1) / kThreads)), dim3(kThreads), 0,
                           s, nv, sc.vpa.p, sc.vpb.p, nold, sc.vpa_old.p, sc.vpb_old.p, sc.memo_old.p, sc.memo.p);
                RELCP_CUDA(cudaGetLastError());
            }
            RELCP_TRY(sc.xb.ensure((size_t)(3 * n), s));
            RELCP_CUDA(cudaMemcpyAsync(sc.xb.p, x_soa, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            for (int k = 0; k < 3; ++k) sc.Lb[k] = box[k];
            sc.vn_bodies = n;
            sc.skin_b = skin;
            sc.valid = true;
            sc.rebuilds += 1;
            for (int k = 0; k < 3; ++k) sfac[k] = 1.0;
        }
        const int64_t nv = sc.vn;
        const int64_t nva = nv > 0 ? nv : 1;
        RELCP_TRY(sc.vflag.ensure((size_t)nva, s));
        RELCP_TRY(sc.vscan.ensure((size_t)nva + 1, s));
        RELCP_TRY(sc.dmax.ensure(1, s));
        RELCP_CUDA(cudaMemsetAsync(sc.dmax.p, 0, sizeof(unsigned long long), s));
        note_launch();
        launch_pdl(disp_kernel, dim3(nbk), dim3(kThreads), 0, s, n, x_soa, sc.xb.p, sfac[0], sfac[1], sfac[2],
                   box[0], box[1], box[2], sc.dmax.p);
        RELCP_CUDA(cudaGetLastError());
        if (nv > 0) {
            note_launch();
            launch_pdl(filter_kernel, dim3((unsigned)((nv + kThreads - 1) / kThreads)), dim3(kThreads), 0, s, nv,
                       sc.vpa.p, sc.vpb.p, xv, rb, box[0], box[1], box[2], nullptr, skin, sc.vflag.p);
            RELCP_CUDA(cudaGetLastError());
        }
        RELCP_TRY(exclusive_scan(sc.vflag.p, sc.vscan.p, nv, sc.scan, s));
        int total = 0;
        unsigned long long dbits = 0;
        RELCP_CUDA(cudaMemcpyAsync(&total, sc.vscan.p + nv, sizeof(int), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaMemcpyAsync(&dbits, sc.dmax.p, sizeof(dbits), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaStreamSynchronize(s));
        double dmax = __builtin_bit_cast(double, dbits);
        // the cached list holds every pair with |d_b| <= cut + delta; a pair in
        // range now has |d_b| <= (cut + 2 dmax) / s, so the list is complete if
        // cut |1/s - 1| + 2 dmax / s <= delta (with a 10% margin)
        double smin = 1.0, grow = 0.0;
        for (int k = 0; k < 3; ++k) {
            smin = fmin(smin, sfac[k]);
            grow = fmax(grow, fabs(1.0 / sfac[k] - 1.0));
        }
        bool ok = cutmax * grow + 2.0 * dmax / smin <= 0.9 * sc.delta;
        if (!ok) {
            sc.valid = false;
            continue;
        }
        *npairs = total;
        // pair buffers hold the whole cached list, so that later steps can
        // compact into them without learning the count on the host
        RELCP_TRY(pa.ensure((size_t)nva, s));
        RELCP_TRY(pb.ensure((size_t)nva, s));
        RELCP_TRY(sc.pv.ensure((size_t)nva, s));
        if (total > 0) {
            note_launch();
            launch_pdl(compact_kernel, dim3((unsigned)((nv + kThreads - 1) / kThreads)), dim3(kThreads), 0, s, nv,
                       sc.vpa.p, sc.vpb.p, sc.vflag.p, sc.vscan.p, pa.p, pb.p, sc.pv.p);
            RELCP_CUDA(cudaGetLastError());
        }
        return RELCP_OK;
    }
    set_error("Verlet list rebuilt but the displacement bound still fails");
    return RELCP_ERR_CUDA;
}

}  // namespace relcp

namespace relcp {

bool verlet_bound_holds(const BroadphaseScratch& sc, int64_t n, const double box[3], double rbmax, double skin,
                        double dmax) {
    if (!sc.valid || sc.vn_bodies != n || sc.skin_b != skin) return false;
    double smin = 1.0, grow = 0.0;
    for (int k = 0; k < 3; ++k) {
        if ((box[k] > 0) != (sc.Lb[k] > 0)) return false;
        const double f = box[k] > 0 ? box[k] / sc.Lb[k] : 1.0;
        smin = fmin(smin, f);
        grow = fmax(grow, fabs(1.0 / f - 1.0));
    }
    const double cutmax = 2.0 * rbmax + skin;
    return cutmax * grow + 2.0 * dmax / smin <= 0.9 * sc.delta;
}

bool broadphase_lookahead_params(const BroadphaseScratch& sc, int64_t n, const double box[3], double sfac[3]) {
    if (!sc.valid || sc.vn_bodies != n || n < 2) return false;
    for (int k = 0; k < 3; ++k) sfac[k] = (box[k] > 0 && sc.Lb[k] > 0) ? box[k] / sc.Lb[k] : 1.0;
    return true;
}

int64_t broadphase_filter_tiles(int64_t nv) { return (nv + kFcTile - 1) / kFcTile; }

relcp_status broadphase_filter_async(int64_t n, const double* x_soa, const double* rb, const double box[3],
                                     const double* box_dev, double skin, DBuf<int>& pa, DBuf<int>& pb,
                                     BroadphaseScratch& sc, cudaStream_t s, int* np_copy) {
    const int64_t nv = sc.vn;
    if (n < 2 || nv == 0) return RELCP_OK;
    View<3, const double> xv = View<3, const double>::soa(x_soa, n);
    const int64_t ntiles = (nv + kFcTile - 1) / kFcTile;
    if (ntiles > (int64_t)1 << 30) return RELCP_ERR_INVALID_ARG;
    RELCP_TRY(scan_reserve_tiles(sc.scan, ntiles, s));
    int* status = sc.scan.status ? sc.scan.status : sc.scan.ctr.p + 2;
    note_launch();
    launch_pdl(filter_compact_kernel, dim3((unsigned)ntiles), dim3(kFcThreads), 0, s, nv, sc.vpa.p, sc.vpb.p, xv,
               rb, box_dev, box[0], box[1], box[2], skin, pa.p, pb.p, sc.pv.p, sc.vscan.p + nv, np_copy,
               sc.scan.tiles.p, sc.scan.ctr.p, status);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

}  // namespace relcp
