// pz_api.cu -- the C ABI of include/pz.h: validation, one-time window
// preparation (sorting, per-tile line ranges, device tables) and the
// orchestration of the kernels in pz_line.cu and pz_rt.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "pz_internal.h"

namespace pz {

// An NVTX range around each entry point (a profiler's timeline shows the pz_* calls and
// the kernels they enqueue; without a profiler attached a push and a pop cost a few ns).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define PZ_RANGE(name) ::pz::NvtxRange pz_nvtx_range_(name)

static thread_local std::string g_err;

pz_status fail(pz_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

pz_status cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return PZ_OK;
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PZ_ENOMEM : PZ_ECUDA;
}

static cudaEvent_t prof_event(pz_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static void prof_fold(pz_ctx *c) {
    for (auto &m : c->marks) {
        float ms = 0.0f;
        if (cudaEventSynchronize(m.b) == cudaSuccess && cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            c->k_ms[m.kid] += ms;
            c->k_count[m.kid] += 1;
        }
        c->ev_pool.push_back(m.a);
        c->ev_pool.push_back(m.b);
    }
    c->marks.clear();
}

// During a capture the events become event-record nodes of the graph (external
// records), so that every replay times its kernels where they run.
cudaEvent_t prof_begin(pz_ctx *c, cudaStream_t s) {
    if (!c->profiling) return nullptr;
    cudaEvent_t a = prof_event(c);
    if (c->capturing)
        cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
    else
        cudaEventRecord(a, s);
    return a;
}

void prof_end(pz_ctx *c, cudaStream_t s, int kid, cudaEvent_t a) {
    if (!a) return;
    cudaEvent_t b = prof_event(c);
    if (c->capturing) {
        cudaEventRecordWithFlags(b, s, cudaEventRecordExternal);
        c->cap_marks.push_back({a, b, kid});
        return;
    }
    cudaEventRecord(b, s);
    c->marks.push_back({a, b, kid});
    if (c->marks.size() > 8192) prof_fold(c);
}

// Events recorded by a graph are read after each replay (the host waits for the
// replay's last event) and are destroyed with the graph.
static void fold_graph_marks(pz_ctx *c, const StepGraph &G) {
    if (G.marks.empty() || cudaEventSynchronize(G.marks.back().b) != cudaSuccess) return;
    for (const auto &m : G.marks) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            c->k_ms[m.kid] += ms;
            c->k_count[m.kid] += 1;
        }
    }
}

static void destroy_marks(std::vector<ProfMark> &marks) {
    for (auto &m : marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    marks.clear();
}

template <class Fn>
static cudaError_t timed(pz_ctx *c, cudaStream_t s, int kid, Fn &&fn) {
    cudaEvent_t a = prof_begin(c, s);
    cudaError_t e = fn();
    prof_end(c, s, kid, a);
    return e;
}

#define PZ_TRY(expr)                         \
    do {                                     \
        pz_status _st = (expr);              \
        if (_st != PZ_OK) return _st;        \
    } while (0)
#define PZ_CUDA(expr, what) PZ_TRY(cuda_check((expr), what))

// Device memory of the library: cudaMalloc / cudaFree, or the caller's allocator
// (pz_set_allocator).  The allocator may change only while no context exists, so that
// every buffer is freed by the allocator that made it.
static std::mutex g_alloc_mu;
static pz_alloc_fn g_alloc = nullptr;
static pz_free_fn g_free = nullptr;
static void *g_alloc_user = nullptr;
static std::atomic<int> g_live_ctx{0};
constexpr size_t kAllocAlign = 256;   // alignment a caller's allocator must give (as cudaMalloc)

static cudaError_t dev_alloc(void **p, size_t bytes) {
    pz_alloc_fn a;
    pz_free_fn f;
    void *u;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        f = g_free;
        u = g_alloc_user;
    }
    if (!a) return cudaMalloc(p, bytes);
    *p = a(bytes, u);
    if (*p && ((uintptr_t)*p % kAllocAlign) != 0) {   // misaligned memory is refused
        f(*p, u);
        *p = nullptr;
    }
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

static void dev_free(void *p) {
    if (!p) return;
    pz_free_fn f;
    void *u;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        f = g_free;
        u = g_alloc_user;
    }
    if (f)
        f(p, u);
    else
        cudaFree(p);
}

template <typename T>
static pz_status dalloc(T **p, size_t n, const char *what) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cuda_check(dev_alloc((void **)p, n * sizeof(T)), what);
}

template <typename T>
static pz_status upload(T **p, const std::vector<T> &h, const char *what) {
    PZ_TRY(dalloc(p, h.size(), what));
    if (!h.empty()) PZ_CUDA(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), what);
    return PZ_OK;
}

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

static bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void dfree(void *p) { dev_free(p); }

// Work items of the persistent line kernels: (star, tile * groups + group, lo, hi) with
// [lo, hi) the star's lines that the item must visit, ordered by estimated cost,
// longest first, so that the queue balances uneven stars and tiles.
//   far:  lines whose window |i - i_l| <= W touches the tile; one item per depth
//         group of DS x GW layers, every (star, tile, group) present (the far
//         forward writes every cell of kappa_line).  An item that costs much more
//         than 1/kPiecesPerCta of a resident CTA's share is cut into P pieces of
//         its line range (a single spectrum has fewer (tile, group) items than
//         twice the resident CTAs, and whole items left a long tail of idle SMs).
//         Backward pieces add their per-line sums atomically like whole items;
//         forward pieces store compensated partial sums, and the piece that
//         finishes an item last combines them in piece order (deterministic);
//         near-core backward items are cut the same way;
//   near: lines whose centre lies within 20 Doppler widths (the widest of the star)
//         of the tile plus a margin; forward items for every (star, tile, group of
//         kNearDepthsFwd layers) (they write the near-core buffer), backward items of
//         kNearDepthsBwd layers only where the range is not empty.
constexpr double kPiecesPerCta = 8.0;       // target far pieces per resident CTA
constexpr int kMaxPieces = 32;              // pieces of one far item at most
constexpr int kMinPieceLines = 256;         // lines of a far piece at least
constexpr size_t kMaxPartBytes = (size_t)512 << 20;   // partial-sum buffer of the split forward items
constexpr double kNearCtasPerSm = 6.0;      // resident near-core CTAs per SM (estimate for the split)
constexpr int kMinNearPieceLines = 64;      // lines of a near-core backward piece at least

static pz_status build_items(pz_ctx *c) {
    const int T = c->tiling.lambda_per_tile();
    const int nt = (int)((c->nlam + T - 1) / T);
    const int DC = c->tiling.depth_per_cta();
    const int ngf = (c->nd + DC - 1) / DC;
    const int nnf = (c->nd + kNearDepthsFwd - 1) / kNearDepthsFwd, nnb = (c->nd + kNearDepthsBwd - 1) / kNearDepthsBwd;
    struct Item {
        int4 v;
        double cost;
    };
    std::vector<Item> fi, nf, nb;
    fi.reserve((size_t)c->S * nt * ngf);
    nf.reserve((size_t)c->S * nt * nnf);
    for (int st = 0; st < c->S; ++st) {
        auto b0 = c->h_il.begin() + c->h_line_off[st], b1 = c->h_il.begin() + c->h_line_off[st + 1];
        double kmin = 1e300;
        for (int k = 0; k < c->ns * c->nd; ++k)
            kmin = std::min(kmin, kC * (double)c->h_invdv[(size_t)st * c->ns * c->nd + k]);
        const double hw = 20.0 / (kmin * c->lnr) * 1.02 + 4.0;
        for (int t = 0; t < nt; ++t) {
            const int64_t a = (int64_t)t * T - c->W, b = (int64_t)t * T + T - 1 + c->W;
            const int lo = (int)(std::lower_bound(b0, b1, (int32_t)std::max<int64_t>(a, INT32_MIN)) - c->h_il.begin());
            const int hi = (int)(std::upper_bound(b0, b1, (int32_t)std::min<int64_t>(b, INT32_MAX)) - c->h_il.begin());
            for (int g = 0; g < ngf; ++g)
                fi.push_back({make_int4(st, t * ngf + g, lo, hi), (double)(hi - lo) * std::min(DC, c->nd - g * DC)});
            double na = (double)t * T - hw, nb_ = (double)t * T + T - 1 + hw;
            na = std::max(na, (double)INT32_MIN / 2);
            nb_ = std::min(nb_, (double)INT32_MAX / 2);
            const int nlo = (int)(std::lower_bound(b0, b1, (int32_t)std::floor(na)) - c->h_il.begin());
            const int nhi = (int)(std::upper_bound(b0, b1, (int32_t)std::ceil(nb_)) - c->h_il.begin());
            for (int g = 0; g < nnf; ++g)
                nf.push_back({make_int4(st, t * nnf + g, nlo, nhi),
                              (double)(nhi - nlo) * std::min(kNearDepthsFwd, c->nd - g * kNearDepthsFwd)});
            if (nhi > nlo)
                for (int g = 0; g < nnb; ++g)
                    nb.push_back({make_int4(st, t * nnb + g, nlo, nhi),
                                  (double)(nhi - nlo) * std::min(kNearDepthsBwd, c->nd - g * kNearDepthsBwd)});
        }
    }
    auto order = [](std::vector<Item> &v) {
        std::stable_sort(v.begin(), v.end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });
        std::vector<int4> out(v.size());
        for (size_t k = 0; k < v.size(); ++k) out[k] = v[k].v;
        return out;
    };
    // far pieces: P = round(cost / piece cost), the piece cost a 1/kPiecesPerCta share of
    // what each resident CTA (n_sm x minb of them) would take
    double tot = 0.0;
    for (const Item &it : fi) tot += it.cost;
    const double workers = (double)std::max(c->n_sm, 1) * std::max(c->tiling.minb, 1);
    const double piece = std::max(tot / (workers * kPiecesPerCta), 1.0);
    const size_t slot_bytes = (size_t)DC * 32 * 2 * sizeof(float4);   // DS x threads x (hi, lo) quads
    struct FItem {
        int4 v, ext;
        double cost;
    };
    std::vector<FItem> fp;
    std::vector<Item> bp;
    fp.reserve(fi.size());
    int nslot = 0, nsplit = 0;
    for (const Item &it : fi) {
        const int n = it.v.w - it.v.z;
        int P = (int)std::lround(it.cost / piece);
        P = std::max(1, std::min({P, kMaxPieces, n / kMinPieceLines}));
        if ((size_t)(nslot + P) * slot_bytes > kMaxPartBytes) P = 1;
        for (int q = 0; q < P; ++q) {
            const int lo = it.v.z + (int)((int64_t)n * q / P), hi = it.v.z + (int)((int64_t)n * (q + 1) / P);
            const int4 v = make_int4(it.v.x, it.v.y, lo, hi);
            const int4 ext = P > 1 ? make_int4(nslot, P, nsplit, q) : make_int4(-1, 1, -1, 0);
            fp.push_back({v, ext, it.cost / P});
            if (hi > lo) bp.push_back({v, it.cost / P});
        }
        if (P > 1) {
            nslot += P;
            ++nsplit;
        }
    }
    std::stable_sort(fp.begin(), fp.end(), [](const FItem &x, const FItem &y) { return x.cost > y.cost; });
    std::vector<int4> hf(fp.size()), hx(fp.size());
    for (size_t k = 0; k < fp.size(); ++k) {
        hf[k] = fp[k].v;
        hx[k] = fp[k].ext;
    }
    // near-core backward pieces (per-line sums added atomically, as whole items do); the
    // near kernels hold about kNearCtasPerSm CTAs per SM
    double totn = 0.0;
    for (const Item &it : nb) totn += it.cost;
    const double npiece = std::max(totn / ((double)std::max(c->n_sm, 1) * kNearCtasPerSm * kPiecesPerCta), 1.0);
    std::vector<Item> nbp;
    nbp.reserve(nb.size());
    for (const Item &it : nb) {
        const int n = it.v.w - it.v.z;
        int P = (int)std::lround(it.cost / npiece);
        P = std::max(1, std::min({P, kMaxPieces, n / kMinNearPieceLines}));
        for (int q = 0; q < P; ++q) {
            const int lo = it.v.z + (int)((int64_t)n * q / P), hi = it.v.z + (int)((int64_t)n * (q + 1) / P);
            if (hi > lo) nbp.push_back({make_int4(it.v.x, it.v.y, lo, hi), it.cost / P});
        }
    }
    std::vector<int4> hbf = order(bp), hn = order(nf), hb = order(nbp);
    dfree(c->d_fitems);
    dfree(c->d_fext);
    dfree(c->d_bitems);
    dfree(c->d_nitems_f);
    dfree(c->d_nitems_b);
    dfree(c->d_fcnt);
    c->d_fitems = c->d_fext = c->d_bitems = c->d_nitems_f = c->d_nitems_b = nullptr;
    c->d_fcnt = nullptr;
    PZ_TRY(upload(&c->d_fitems, hf, "work items"));
    PZ_TRY(upload(&c->d_fext, hx, "work items"));
    PZ_TRY(upload(&c->d_bitems, hbf, "work items"));
    PZ_TRY(upload(&c->d_nitems_f, hn, "work items"));
    PZ_TRY(upload(&c->d_nitems_b, hb, "work items"));
    PZ_TRY(dalloc(&c->d_fcnt, (size_t)nsplit, "work items"));
    PZ_CUDA(cudaMemset(c->d_fcnt, 0, sizeof(int) * std::max(nsplit, 1)), "work items");
    const size_t part = (size_t)nslot * slot_bytes;
    if (c->fpart_cap < part) {
        dfree(c->d_fpart);
        c->d_fpart = nullptr;
        c->fpart_cap = 0;
        PZ_TRY(dalloc(&c->d_fpart, part / sizeof(float4), "far-wing partial sums"));
        c->fpart_cap = part;
    }
    c->n_fitems = (int)hf.size();
    c->n_bitems = (int)hbf.size();
    c->n_fsplit = nsplit;
    c->n_nitems_f = (int)hn.size();
    c->n_nitems_b = (int)hb.size();
    c->ntiles = nt;
    c->tileT = T;
    return PZ_OK;
}

// Fast-path threshold per (star, species, depth slab of DS layers): a line whose
// distance from every point of the tile is >= thr (grid units) has |v| >= 20 at every
// depth of the slab, because |v| = |expm1(Delta ln r)| c/dv_D >= |Delta| ln r (1 - |Delta| ln r / 2) c/dv_D.
// Slabs past the last layer (grid padding) get 0.
static pz_status build_thresholds(pz_ctx *c) {
    const int DS = c->tiling.DS, DC = c->tiling.depth_per_cta();
    const int nslab = ((c->nd + DC - 1) / DC) * c->tiling.GW;
    double shrink = 1.0 - 0.5 * (c->W + 1024.0) * c->lnr;
    if (shrink < 0.5) shrink = 0.5;
    std::vector<float> thr((size_t)c->S * c->ns * nslab, 0.0f);
    for (int st = 0; st < c->S; ++st)
        for (int s = 0; s < c->ns; ++s)
            for (int b = 0; b < nslab; ++b) {
                double mn = 1e300;
                for (int d = b * DS; d < std::min(c->nd, (b + 1) * DS); ++d)
                    mn = std::min(mn, (double)c->h_invdv[((size_t)st * c->ns + s) * c->nd + d]);
                if (mn < 1e300)
                    thr[((size_t)st * c->ns + s) * nslab + b] =
                        (float)(20.0 / (kC * mn * c->lnr * shrink) * (1.0 + 1e-4) + 1e-3);
            }
    dfree(c->d_thr);
    c->d_thr = nullptr;
    PZ_TRY(upload(&c->d_thr, thr, "thresholds"));
    c->nslab = nslab;
    return PZ_OK;
}

static void drop_graph(pz_ctx *c) {
    if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
    destroy_marks(c->graph.marks);
    c->graph = StepGraph();
    if (c->ggraph.exec) cudaGraphExecDestroy(c->ggraph.exec);
    destroy_marks(c->ggraph.marks);
    c->ggraph = StepGraph();
}

static void destroy_ctx(pz_ctx *c) {
    if (!c) return;
    drop_graph(c);
    void *ptrs[] = {c->d_m, c->d_T, c->d_beta_hi, c->d_beta_lo, c->d_ne, c->d_npert, c->d_c2T, c->d_ne64,
                    c->d_npert64, c->d_rho64, c->d_R, c->d_Rbase, c->d_invdv, c->d_Ksd, c->d_pop64, c->d_mass64, c->d_xi64,
                    c->d_thr, c->d_kc, c->d_B, c->d_stim, c->d_dab, c->d_mdgf, c->d_mdg6, c->d_eos, c->L.orig, c->L.star, c->L.ilf,
                    c->L.il32, c->L.frac, c->L.sp, c->L.E, c->L.lamcm, c->L.grad, c->L.g4, c->L.g6base, c->L.g6,
                    c->L.Q, c->L.Qbase, c->L.x64, c->L.lg_gf, c->L.lg_rad, c->L.lg_4, c->L.lg_6, c->L.dgf, c->L.dg6,
                    c->d_line_off, c->d_fitems, c->d_fext, c->d_bitems, c->d_fpart, c->d_fcnt, c->d_nitems_f,
                    c->d_nitems_b, c->d_ctr, c->d_knear, c->d_kline,
                    c->d_F, c->d_Fc, c->d_g, c->d_gc, c->d_tap0, c->d_ntap, c->d_tapw, c->d_dFbar, c->d_Gt,
                    c->d_Gt64, c->d_gacc, c->d_gline, c->d_gab, c->d_dLdf, c->d_finfo, c->d_status,
                    c->d_keep, c->L.gradbase, c->L.g4base, c->L.dgrad, c->L.dg4, c->d_mdgrad, c->d_mdg4,
                    c->d_grp_of, c->d_grp_off, c->d_grp_mem, c->d_sigma};
    for (void *p : ptrs) dfree(p);
    destroy_marks(c->marks);
    destroy_marks(c->cap_marks);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    --g_live_ctx;
}

// Validation of one atmosphere; shared fields are checked against ref (star 0).
static pz_status check_atmos(const pz_atmos *at, const pz_atmos *ref, const char *who) {
    const std::string w(who);
    if (!at) return fail(PZ_EINVAL, w + ": atmos is NULL");
    const int nd = at->n_depth, ns = at->n_species;
    if (nd < 2 || nd > kMaxDepth) return fail(PZ_EINVAL, w + ": n_depth must be in [2, 128]");
    if (ns < 1) return fail(PZ_EINVAL, w + ": n_species must be >= 1");
    if (at->n_lambda < 1 || at->n_lambda > 16000000) return fail(PZ_EINVAL, w + ": n_lambda must be in [1, 1.6e7]");
    if (!at->m || !at->T || !at->rho || !at->n_e || !at->n_pert || !at->pop || !at->mass_amu || !at->kappa_c)
        return fail(PZ_EINVAL, w + ": an atmosphere array is NULL");
    if (!finite_pos(at->lambda0_nm) || !finite_pos(at->R_grid)) return fail(PZ_EINVAL, w + ": lambda0 and R_grid must be > 0");
    if (!(std::isfinite(at->xi_cms) && at->xi_cms >= 0)) return fail(PZ_EINVAL, w + ": xi must be finite and >= 0");
    if (ref && (at->n_depth != ref->n_depth || at->n_species != ref->n_species || at->n_lambda != ref->n_lambda ||
                at->lambda0_nm != ref->lambda0_nm || at->R_grid != ref->R_grid))
        return fail(PZ_EINVAL, w + ": every star must share n_depth, n_species and the wavelength grid");
    for (int d = 0; d < nd; ++d) {
        if (!finite_pos(at->m[d]) || !finite_pos(at->T[d]) || !finite_pos(at->rho[d]))
            return fail(PZ_EINVAL, w + ": m, T, rho must be finite and > 0");
        if (!(std::isfinite(at->n_e[d]) && at->n_e[d] >= 0) || !(std::isfinite(at->n_pert[d]) && at->n_pert[d] >= 0))
            return fail(PZ_EINVAL, w + ": n_e and n_pert must be finite and >= 0");
        if (d > 0 && !(at->m[d] > at->m[d - 1])) return fail(PZ_EINVAL, w + ": m must be strictly increasing");
    }
    for (int s = 0; s < ns; ++s) {
        if (!finite_pos(at->mass_amu[s])) return fail(PZ_EINVAL, w + ": mass_amu must be > 0");
        for (int d = 0; d < nd; ++d) {
            double p = at->pop[(size_t)s * nd + d];
            if (!(std::isfinite(p) && p >= 0)) return fail(PZ_EINVAL, w + ": pop must be finite and >= 0");
        }
    }
    for (int64_t k = 0; k < (int64_t)nd * at->n_lambda; ++k)
        if (!finite_pos(at->kappa_c[k])) return fail(PZ_EINVAL, w + ": kappa_c must be finite and > 0");
    return PZ_OK;
}

static pz_status ensure_far_tables(pz_ctx *c);

static pz_status create_impl(int S, const pz_atmos *atv, const pz_linelist *ll, const int64_t *sub_off,
                             const int32_t *sub_idx, pz_precision prec, pz_ctx **out, const char *who) {
    const std::string w(who);
    if (!out) return fail(PZ_EINVAL, w + ": out is NULL");
    *out = nullptr;
    if (!atv || !ll) return fail(PZ_EINVAL, w + ": atmos or lines is NULL");
    if (S < 1 || S > 512) return fail(PZ_EINVAL, w + ": n_stars must be in [1, 512]");
    if (prec != PZ_FP64 && prec != PZ_MIXED) return fail(PZ_EINVAL, w + ": unknown precision");
    for (int st = 0; st < S; ++st) PZ_TRY(check_atmos(atv + st, st ? atv : nullptr, who));
    const pz_atmos *at0 = atv;
    const int nd = at0->n_depth, ns = at0->n_species;
    const int64_t nlam = at0->n_lambda;
    if (ll->n_lines < 0 || ll->n_lines > 2000000000) return fail(PZ_EINVAL, w + ": n_lines out of range");
    if (ll->half_window < 0 || ll->half_window > 500000) return fail(PZ_EINVAL, w + ": half_window must be in [0, 5e5]");
    const int64_t nl = ll->n_lines;
    if (nl > 0 && (!ll->lambda_nm || !ll->log_gf || !ll->E_low_eV || !ll->log_gamma_rad || !ll->log_gamma4 ||
                   !ll->log_gamma6 || !ll->species))
        return fail(PZ_EINVAL, w + ": a line array is NULL");
    for (int64_t l = 0; l < nl; ++l) {
        if (!finite_pos(ll->lambda_nm[l])) return fail(PZ_EINVAL, w + ": lambda_nm must be finite and > 0");
        if (!std::isfinite(ll->log_gf[l]) || !std::isfinite(ll->E_low_eV[l]) || !std::isfinite(ll->log_gamma_rad[l]) ||
            !std::isfinite(ll->log_gamma4[l]) || !std::isfinite(ll->log_gamma6[l]))
            return fail(PZ_EINVAL, w + ": non-finite line parameter");
        if (ll->species[l] < 0 || ll->species[l] >= ns) return fail(PZ_EINVAL, w + ": species out of range");
    }
    if (sub_off) {
        if (sub_off[0] != 0) return fail(PZ_EINVAL, w + ": subset_offsets[0] must be 0");
        for (int st = 0; st < S; ++st)
            if (sub_off[st + 1] < sub_off[st]) return fail(PZ_EINVAL, w + ": subset_offsets must be non-decreasing");
        if (sub_off[S] > 0 && !sub_idx) return fail(PZ_EINVAL, w + ": subset_index is NULL");
        if (sub_off[S] > 2000000000) return fail(PZ_EINVAL, w + ": too many subset entries");
        for (int64_t k = 0; k < sub_off[S]; ++k)
            if (sub_idx[k] < 0 || sub_idx[k] >= nl) return fail(PZ_EINVAL, w + ": subset_index out of range");
    } else if ((int64_t)S * nl > 2000000000) {
        return fail(PZ_EINVAL, w + ": n_stars x n_lines too large");
    }

    int dev = 0;
    PZ_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(PZ_EINVAL, w + ": device ordinal beyond the supported 64");
    pz_ctx *c = new pz_ctx();
    ++g_live_ctx;
    c->device = dev;
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev);
    c->prec = prec;
    c->S = S;
    c->nd = nd;
    c->ns = ns;
    c->nlam = nlam;
    c->ld = ((nlam + 511) / 512) * 512;
    c->lambda0_nm = at0->lambda0_nm;
    c->R = at0->R_grid;
    c->lnr = std::log1p(1.0 / at0->R_grid);
    c->W = ll->half_window;
    c->nl_caller = nl;

    auto bail = [&](pz_status st) {
        destroy_ctx(c);
        return st;
    };
    if (ensure_device_tables() != PZ_OK || ensure_expn_table() != PZ_OK) return bail(PZ_ECUDA);
    if (cuda_check(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "stream")) return bail(PZ_ECUDA);

    // ---- lines: centre placement, drop, sort within each star ----
    const double W = c->W;
    std::vector<double> x(nl);
    std::vector<char> inwin(nl);
    for (int64_t l = 0; l < nl; ++l) {
        x[l] = std::log(ll->lambda_nm[l] / at0->lambda0_nm) / c->lnr;
        double il = std::floor(x[l] + 0.5);
        inwin[l] = il >= -W && il <= (double)(nlam - 1) + W;
    }
    std::vector<int64_t> keep;
    std::vector<int32_t> kstar;
    c->h_line_off.assign(S + 1, 0);
    for (int st = 0; st < S; ++st) {
        const size_t first = keep.size();
        const int64_t a = sub_off ? sub_off[st] : 0, b = sub_off ? sub_off[st + 1] : nl;
        for (int64_t k = a; k < b; ++k) {
            const int64_t l = sub_off ? (int64_t)sub_idx[k] : k;
            if (inwin[l]) keep.push_back(l);
        }
        std::stable_sort(keep.begin() + first, keep.end(), [&](int64_t p, int64_t q) { return x[p] < x[q]; });
        kstar.resize(keep.size(), st);
        c->h_line_off[st + 1] = (int64_t)keep.size();
    }
    const int64_t n = (int64_t)keep.size();
    c->L.n = n;
    std::vector<int32_t> orig(n), il32(n), sp(n);
    std::vector<float> ilf(n), frac(n), E(n), lamcm(n), grad(n), g4(n), g6(n), Qf(n), lg_gf(n), lg_rad(n), lg_4(n),
        lg_6(n), zeros(n, 0.0f);
    std::vector<double> Qb(n), x64(n);
    const double C0 = kPI * kE * kE / (kME * kC) / kSQRTPI;
    int64_t evals = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t l = keep[k];
        double il = std::floor(x[l] + 0.5);
        orig[k] = (int32_t)l;
        il32[k] = (int32_t)il;
        ilf[k] = (float)il;
        frac[k] = (float)(x[l] - il);
        sp[k] = ll->species[l];
        E[k] = ll->E_low_eV[l];
        double lc = ll->lambda_nm[l] * 1e-7;
        lamcm[k] = (float)lc;
        grad[k] = (float)std::pow(10.0, (double)ll->log_gamma_rad[l]);
        g4[k] = (float)std::pow(10.0, (double)ll->log_gamma4[l]);
        g6[k] = (float)std::pow(10.0, (double)ll->log_gamma6[l]);
        Qb[k] = C0 * lc * std::pow(10.0, (double)ll->log_gf[l]);
        Qf[k] = (float)Qb[k];
        x64[k] = x[l];
        lg_gf[k] = ll->log_gf[l];
        lg_rad[k] = ll->log_gamma_rad[l];
        lg_4[k] = ll->log_gamma4[l];
        lg_6[k] = ll->log_gamma6[l];
        int64_t i0 = std::max<int64_t>(0, (int64_t)il - c->W), i1 = std::min<int64_t>(nlam - 1, (int64_t)il + c->W);
        evals += (i1 - i0 + 1);
    }
    c->n_evals = evals * nd;
    c->h_il = il32;
    std::vector<float> mzeros(std::max<int64_t>(nl, 1), 0.0f);
    if (upload(&c->L.orig, orig, "lines") || upload(&c->L.star, kstar, "lines") || upload(&c->L.il32, il32, "lines") ||
        upload(&c->L.ilf, ilf, "lines") || upload(&c->L.frac, frac, "lines") || upload(&c->L.sp, sp, "lines") ||
        upload(&c->L.E, E, "lines") || upload(&c->L.lamcm, lamcm, "lines") || upload(&c->L.grad, grad, "lines") ||
        upload(&c->L.g4, g4, "lines") || upload(&c->L.g6base, g6, "lines") || upload(&c->L.g6, g6, "lines") ||
        upload(&c->L.gradbase, grad, "lines") || upload(&c->L.g4base, g4, "lines") ||
        upload(&c->L.dgrad, zeros, "lines") || upload(&c->L.dg4, zeros, "lines") ||
        upload(&c->d_mdgrad, mzeros, "corrections") || upload(&c->d_mdg4, mzeros, "corrections") ||
        upload(&c->L.Q, Qf, "lines") || upload(&c->L.Qbase, Qb, "lines") || upload(&c->L.x64, x64, "lines") ||
        upload(&c->L.lg_gf, lg_gf, "lines") || upload(&c->L.lg_rad, lg_rad, "lines") ||
        upload(&c->L.lg_4, lg_4, "lines") || upload(&c->L.lg_6, lg_6, "lines") || upload(&c->L.dgf, zeros, "lines") ||
        upload(&c->L.dg6, zeros, "lines") || upload(&c->d_mdgf, mzeros, "corrections") ||
        upload(&c->d_mdg6, mzeros, "corrections") || upload(&c->d_line_off, c->h_line_off, "lines"))
        return bail(PZ_ENOMEM);

    // ---- depth and species tables, [S][...] ----
    const size_t SD = (size_t)S * nd, SSD = (size_t)S * ns * nd;
    c->h_m.resize(SD);
    c->h_T.resize(SD);
    std::vector<float> bh(SD), bl(SD), ne(SD), npert(SD), c2T(SD), invdv(SSD), Ksd(SSD), Rf(SSD);
    std::vector<double> ne64(SD), np64(SD), rho64(SD), Rb(SSD), pop64(SSD), mass64((size_t)S * ns), xi64(S);
    for (int st = 0; st < S; ++st) {
        const pz_atmos *at = atv + st;
        xi64[st] = at->xi_cms;
        for (int d = 0; d < nd; ++d) {
            const size_t o = (size_t)st * nd + d;
            c->h_m[o] = at->m[d];
            c->h_T[o] = at->T[d];
            double beta = kEV / (kKB * at->T[d]);
            bh[o] = (float)beta;
            bl[o] = (float)(beta - (double)bh[o]);
            ne[o] = (float)at->n_e[d];
            npert[o] = (float)at->n_pert[d];
            c2T[o] = (float)(kC2 / at->T[d]);
            ne64[o] = at->n_e[d];
            np64[o] = at->n_pert[d];
            rho64[o] = at->rho[d];
        }
        for (int s = 0; s < ns; ++s) {
            mass64[(size_t)st * ns + s] = at->mass_amu[s];
            for (int d = 0; d < nd; ++d) {
                double dv = std::sqrt(2.0 * kKB * at->T[d] / (at->mass_amu[s] * kAMU) + at->xi_cms * at->xi_cms);
                const size_t id = (size_t)s * nd + d, o = (size_t)st * ns * nd + id;
                invdv[o] = (float)(1.0 / dv);
                // K = 2^36/k^2 of the far-wing prefactors, k = c/dv_D rounded as the kernels form it
                const float kf = (float)kC * invdv[o];
                Ksd[o] = kKScale / (kf * kf);
                pop64[o] = at->pop[id];
                Rb[o] = (1.0 / dv) * at->pop[id] / at->rho[d];
                Rf[o] = (float)Rb[o];
            }
        }
    }
    c->h_invdv = invdv;
    std::vector<double> dab(1, 0.0);
    std::vector<int32_t> eos(ns, -1);
    if (upload(&c->d_m, c->h_m, "depth") || upload(&c->d_T, c->h_T, "depth") || upload(&c->d_beta_hi, bh, "depth") ||
        upload(&c->d_beta_lo, bl, "depth") || upload(&c->d_ne, ne, "depth") || upload(&c->d_npert, npert, "depth") ||
        upload(&c->d_c2T, c2T, "depth") || upload(&c->d_ne64, ne64, "depth") || upload(&c->d_npert64, np64, "depth") ||
        upload(&c->d_rho64, rho64, "depth") || upload(&c->d_invdv, invdv, "species") || upload(&c->d_Ksd, Ksd, "species") ||
        upload(&c->d_R, Rf, "species") ||
        upload(&c->d_Rbase, Rb, "species") || upload(&c->d_pop64, pop64, "species") ||
        upload(&c->d_mass64, mass64, "species") || upload(&c->d_xi64, xi64, "species") || build_thresholds(c) ||
        upload(&c->d_dab, dab, "abund") || upload(&c->d_eos, eos, "abund"))
        return bail(PZ_ENOMEM);

    // ---- continuum opacity [S][nd][ld] ----
    if (dalloc(&c->d_kc, SD * c->ld, "kappa_c")) return bail(PZ_ENOMEM);
    if (cuda_check(cudaMemset(c->d_kc, 0, sizeof(double) * SD * c->ld), "kappa_c")) return bail(PZ_ECUDA);
    for (int st = 0; st < S; ++st)
        if (cuda_check(cudaMemcpy2D(c->d_kc + (size_t)st * nd * c->ld, c->ld * sizeof(double), atv[st].kappa_c,
                                    nlam * sizeof(double), nlam * sizeof(double), nd, cudaMemcpyHostToDevice),
                       "kappa_c"))
            return bail(PZ_ECUDA);
    // ---- Planck function and stimulated-emission factor [S][nd][ld], from T and lambda ----
    if (dalloc(&c->d_B, SD * c->ld, "Planck table") || dalloc(&c->d_stim, SD * c->ld, "Planck table"))
        return bail(PZ_ENOMEM);
    if (cuda_check(launch_planck_tables(c, 0), "Planck table")) return bail(PZ_ECUDA);

    // ---- resident buffers ----
    size_t ksz = (prec == PZ_MIXED) ? sizeof(float) : sizeof(double);
    if (cuda_check(dev_alloc(&c->d_kline, ksz * SD * c->ld), "kappa_line buffer") ||
        (prec == PZ_MIXED && dalloc(&c->d_knear, SD * c->ld, "kappa_line buffer")) ||
        dalloc(&c->d_F, (size_t)S * nlam, "flux") || dalloc(&c->d_Fc, (size_t)S * nlam, "flux") ||
        dalloc(&c->d_ctr, 4, "work counters") || dalloc(&c->d_status, 1, "status word"))
        return bail(PZ_ENOMEM);
    if (cuda_check(cudaMemset(c->d_status, 0, sizeof(int32_t)), "status word")) return bail(PZ_ECUDA);
    if (prec == PZ_MIXED && cuda_check(cudaMemset(c->d_knear, 0, sizeof(float) * SD * c->ld), "kappa_line buffer"))
        return bail(PZ_ECUDA);
    if (build_items(c) != PZ_OK) return bail(PZ_ENOMEM);
    if (prec == PZ_MIXED && ensure_far_tables(c) != PZ_OK) return bail(PZ_ENOMEM);
    if (cuda_check(cudaDeviceSynchronize(), who)) return bail(PZ_ECUDA);
    *out = c;
    return PZ_OK;
}

// instrument outputs [S][n]
static pz_status ensure_out_buffers(pz_ctx *c, int64_t n) {
    if (c->d_g && c->pix_cap >= n) return PZ_OK;
    drop_graph(c);
    dfree(c->d_g);
    dfree(c->d_gc);
    dfree(c->d_dLdf);
    c->d_g = c->d_gc = nullptr;
    c->d_dLdf = nullptr;
    PZ_TRY(dalloc(&c->d_g, (size_t)c->S * n, "instrument output"));
    PZ_TRY(dalloc(&c->d_gc, (size_t)c->S * n, "instrument output"));
    c->pix_cap = n;
    return PZ_OK;
}

static pz_status ensure_backward_buffers(pz_ctx *c) {
    const size_t SD = (size_t)c->S * c->nd;
    if (!c->d_dFbar) PZ_TRY(dalloc(&c->d_dFbar, (size_t)c->S * c->nlam, "backward scratch"));
    if (c->prec == PZ_MIXED && !c->d_Gt) PZ_TRY(dalloc(&c->d_Gt, SD * c->ld, "backward scratch"));
    if (c->prec == PZ_FP64 && !c->d_Gt64) PZ_TRY(dalloc(&c->d_Gt64, SD * c->ld, "backward scratch"));
    // room for the four-family reverse pass (pz_backward4): six rows per line, four per caller line
    if (!c->d_gacc) PZ_TRY(dalloc(&c->d_gacc, 6 * std::max<int64_t>(c->L.n, 1), "backward scratch"));
    if (!c->d_gline) PZ_TRY(dalloc(&c->d_gline, 4 * std::max<int64_t>(c->nl_caller, 1), "backward scratch"));
    if (c->n_elem > 0 && !c->d_gab) PZ_TRY(dalloc(&c->d_gab, c->n_elem, "backward scratch"));
    return PZ_OK;
}

// Far-wing line records for the current tiling (mixed form), one per depth group and line.
// Allocated here, outside any stream capture, and grown only when a tiling needs more.
static pz_status ensure_far_tables(pz_ctx *c) {
    const size_t ib = far_info_bytes(c);
    if (c->finfo_cap < ib) {
        dfree(c->d_finfo);
        c->d_finfo = nullptr;
        c->finfo_cap = 0;
        if (dev_alloc(&c->d_finfo, ib) != cudaSuccess) {
            cudaGetLastError();
            return fail(PZ_ENOMEM, "far-wing line records: allocation failed");
        }
        c->finfo_cap = ib;
    }
    return PZ_OK;
}

// Validate a tiling and make it current: thresholds and work items are rebuilt and
// the captured calibration graph is dropped.
static pz_status apply_tiling(pz_ctx *c, const Tiling &t, const char *who) {
    const std::string w(who);
    if (!tiling_supported(t.J, t.DS, t.minb))
        return fail(PZ_EINVAL, w + ": unsupported (lambda_per_thread, depth_per_warp, ctas_per_sm)");
    if (t.GW < 1 || t.GW > 4) return fail(PZ_EINVAL, w + ": warps_per_cta must be in [1, 4]");
    if (t.LC < 1 || t.LC > 512) return fail(PZ_EINVAL, w + ": lines_per_chunk must be in [1, 512]");
    if (!tiling_fits(t)) return fail(PZ_EINVAL, w + ": shared-memory chunk too large");
    drop_graph(c);
    c->tiling = t;
    PZ_TRY(build_thresholds(c));
    PZ_TRY(build_items(c));
    if (c->prec == PZ_MIXED) PZ_TRY(ensure_far_tables(c));
    return PZ_OK;
}

// The backward stages after the objective's seed dL/df: instrument adjoint, transfer
// adjoint, line gradients, finalisation into caller order.
static pz_status enqueue_backward(pz_ctx *c, const float *dLdf, float *g_gf, float *g_g6, float *g_ab,
                                  cudaStream_t s, bool four = false, float *g_rad = nullptr, float *g_g4 = nullptr) {
    PZ_CUDA(timed(c, s, PZ_K_INST_ADJOINT, [&] { return launch_inst_adjoint(c, dLdf, s); }), "instrument adjoint");
    PZ_CUDA(timed(c, s, PZ_K_RT_ADJOINT, [&] { return launch_rt_adjoint(c, s); }), "transfer adjoint");
    c->have_gt = true;
    const int64_t nl1 = std::max<int64_t>(c->L.n, 1);
    PZ_CUDA(cudaMemsetAsync(c->d_gacc, 0, sizeof(double) * (four ? 6 : 2) * nl1, s), "backward");
    if (c->L.n > 0) {
        // one line pass per damping family: the first gives the gf and van der Waals sums,
        // the radiative and Stark passes their second sums (rows 3 and 5)
        const int passes = four ? 3 : 1;
        for (int p = 0; p < passes; ++p) {
            c->bwd_dsel = p;
            c->gacc_off = 2 * p * c->L.n;
            cudaError_t e = timed(c, s, PZ_K_LINE_BWD, [&] {
                return c->prec == PZ_MIXED ? launch_line_bwd_mixed(c, s) : launch_line_bwd_fp64(c, s);
            });
            c->bwd_dsel = 0;
            c->gacc_off = 0;
            PZ_CUDA(e, "line gradient kernel");
        }
    }
    PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] { return launch_grad_finalize(c, g_gf, g_g6, g_ab, s, four, g_rad, g_g4); }),
            "gradient finalize");
    return PZ_OK;
}

__global__ void k_f32_to_f64(int n, const float *a, double *b) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) b[k] = (double)a[k];
}

// rows of [rows][ld] FP64 -> [rows][nlam] FP32; row = blockIdx.y
__global__ void k_d2f_2d(int64_t nlam, int64_t ld, const double *a, float *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t r = blockIdx.y;
    if (i < nlam) b[r * nlam + i] = (float)a[r * ld + i];
}

}  // namespace pz

using namespace pz;

extern "C" {

pz_status pz_create(const pz_atmos *atmos, const pz_linelist *lines, pz_precision precision, pz_ctx **out) {
    PZ_RANGE("pz_create");
    return create_impl(1, atmos, lines, nullptr, nullptr, precision, out, "pz_create");
}

pz_status pz_create_batch(int32_t n_stars, const pz_atmos *atmos, const pz_linelist *lines,
                          const int64_t *subset_offsets, const int32_t *subset_index, pz_precision precision,
                          pz_ctx **out) {
    PZ_RANGE("pz_create_batch");
    return create_impl(n_stars, atmos, lines, subset_offsets, subset_index, precision, out, "pz_create_batch");
}

pz_status pz_destroy(pz_ctx *ctx) {
    PZ_RANGE("pz_destroy");
    if (!ctx) return PZ_OK;
    cudaDeviceSynchronize();
    destroy_ctx(ctx);
    return PZ_OK;
}

const char *pz_last_error(void) { return g_err.c_str(); }

pz_status pz_set_allocator(pz_alloc_fn alloc, pz_free_fn free_fn, void *user) {
    PZ_RANGE("pz_set_allocator");
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(PZ_EINVAL, "pz_set_allocator: give both functions or neither");
    if (g_live_ctx.load() != 0)
        return fail(PZ_ESTATE, "pz_set_allocator: contexts exist; destroy them before changing the allocator");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_user = alloc ? user : nullptr;
    return PZ_OK;
}

int64_t pz_eval_count(const pz_ctx *ctx) { return ctx ? ctx->n_evals : 0; }

int32_t pz_last_launch_count(const pz_ctx *ctx) { return ctx ? ctx->launches : 0; }

int32_t pz_n_stars(const pz_ctx *ctx) { return ctx ? ctx->S : 0; }

int64_t pz_star_lines(const pz_ctx *ctx, int32_t star) {
    if (!ctx || star < 0 || star >= ctx->S) return -1;
    return ctx->h_line_off[star + 1] - ctx->h_line_off[star];
}

pz_status pz_set_tiling(pz_ctx *c, int32_t J, int32_t DS, int32_t GW, int32_t LC, int32_t MINB) {
    PZ_RANGE("pz_set_tiling");
    if (!c) return fail(PZ_EINVAL, "pz_set_tiling: ctx is NULL");
    Tiling t = c->tiling;
    if (J > 0) t.J = J;
    if (DS > 0) t.DS = DS;
    if (GW > 0) t.GW = GW;
    if (LC > 0) t.LC = LC;
    if (MINB > 0) t.minb = MINB;
    if (LC > 0) t.LCB = t.LC;
    return apply_tiling(c, t, "pz_set_tiling");
}

pz_status pz_autotune(pz_ctx *c, int32_t with_backward, int32_t reps, int32_t *best, double *best_ms, void *stream) {
    PZ_RANGE("pz_autotune");
    if (!c) return fail(PZ_EINVAL, "pz_autotune: ctx is NULL");
    if (c->prec != PZ_MIXED) return fail(PZ_EINVAL, "pz_autotune: only the mixed-precision form has tilings");
    if (reps < 1 || reps > 100) return fail(PZ_EINVAL, "pz_autotune: reps must be in [1, 100]");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    if (with_backward) {
        PZ_TRY(ensure_backward_buffers(c));
        // G of the last reverse pass, or zeros: the kernels' cost does not depend on G
        if (!c->have_gt)
            PZ_CUDA(cudaMemsetAsync(c->d_Gt, 0, sizeof(float) * (size_t)c->S * c->nd * c->ld, s), "pz_autotune");
    }
    cudaEvent_t ev[4];
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return cuda_check(cudaGetLastError(), "pz_autotune: events");
    const size_t gbytes = sizeof(double) * 2 * std::max<int64_t>(c->L.n, 1);
    // time one tiling: one untimed pass, then reps forward launches and reps backward launches
    auto measure = [&](const Tiling &t, double &fwd_ms, double &bwd_ms) -> pz_status {
        PZ_TRY(apply_tiling(c, t, "pz_autotune"));
        auto bwd = [&]() -> cudaError_t {
            cudaError_t e = cudaMemsetAsync(c->d_gacc, 0, gbytes, s);
            return e != cudaSuccess ? e : launch_line_bwd_mixed(c, s);
        };
        PZ_CUDA(launch_line_fwd_mixed(c, s), "pz_autotune: forward");
        if (with_backward) PZ_CUDA(bwd(), "pz_autotune: backward");
        PZ_CUDA(cudaEventRecord(ev[0], s), "pz_autotune");
        for (int r = 0; r < reps; ++r) PZ_CUDA(launch_line_fwd_mixed(c, s), "pz_autotune: forward");
        PZ_CUDA(cudaEventRecord(ev[1], s), "pz_autotune");
        for (int r = 0; r < reps && with_backward; ++r) PZ_CUDA(bwd(), "pz_autotune: backward");
        PZ_CUDA(cudaEventRecord(ev[2], s), "pz_autotune");
        PZ_CUDA(cudaEventSynchronize(ev[2]), "pz_autotune");
        float a = 0.0f, b = 0.0f;
        PZ_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]), "pz_autotune");
        PZ_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]), "pz_autotune");
        fwd_ms = a / reps;
        bwd_ms = with_backward ? b / reps : 0.0;
        return PZ_OK;
    };
    // coordinate search from the current tiling: (lambda points, depths, CTAs per SM)
    // over the compiled list, then warps per CTA, then lines per chunk
    Tiling cur = c->tiling;
    double cf = 0, cb = 0;
    pz_status st = measure(cur, cf, cb);
    int tried = 1;
    auto consider = [&](Tiling t) -> pz_status {
        if (!tiling_supported(t.J, t.DS, t.minb) || t.GW < 1 || t.GW > 4 || !tiling_fits(t)) return PZ_OK;
        double f = 0, b = 0;
        PZ_TRY(measure(t, f, b));
        ++tried;
        if (f + b < cf + cb) {
            cur = t;
            cf = f;
            cb = b;
        }
        return PZ_OK;
    };
    static const int kJDM[][3] = {{4, 6, 1}, {4, 6, 2}, {4, 6, 3}, {4, 6, 4}, {4, 6, 5}, {4, 6, 6},  {4, 8, 1},
                                  {4, 8, 2}, {4, 8, 3}, {4, 12, 1}, {4, 12, 2}, {2, 6, 4}, {2, 6, 6},  {2, 8, 2},
                                  {2, 8, 3}, {2, 8, 4}, {2, 8, 5}, {2, 12, 1}, {2, 12, 2}, {2, 12, 3}};
    // two rounds of the three phases: a tiling that needs both a different register budget and
    // a different chunk (or CTA width) is reachable only after the others have moved
    for (int round = 0; round < 2 && st == PZ_OK; ++round) {
        {
            const Tiling base = cur;
            for (const auto &q : kJDM) {
                Tiling t = base;
                t.J = q[0];
                t.DS = q[1];
                t.minb = q[2];
                if (t.J == base.J && t.DS == base.DS && t.minb == base.minb) continue;
                if ((st = consider(t)) != PZ_OK) break;
            }
        }
        if (st == PZ_OK) {
            const Tiling base = cur;
            for (int gw = 1; gw <= 4 && st == PZ_OK; ++gw)
                if (gw != base.GW) {
                    Tiling t = base;
                    t.GW = gw;
                    st = consider(t);
                }
        }
        if (st == PZ_OK) {
            const Tiling base = cur;
            for (int lc : {16, 32, 64, 128})
                if (lc != base.LC && st == PZ_OK) {
                    Tiling t = base;
                    t.LC = lc;
                    t.LCB = lc;
                    st = consider(t);
                }
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st != PZ_OK) return st;
    PZ_TRY(apply_tiling(c, cur, "pz_autotune"));
    // the buffers hold the last candidate's results: the forward must run again
    c->have_kline = c->have_flux = c->have_inst = false;
    if (best) {
        best[0] = cur.J;
        best[1] = cur.DS;
        best[2] = cur.GW;
        best[3] = cur.LC;
        best[4] = cur.minb;
        best[5] = tried;
    }
    if (best_ms) {
        best_ms[0] = cf;
        best_ms[1] = cb;
    }
    return PZ_OK;
}

pz_status pz_set_centre_test(pz_ctx *c, double eta, int64_t *kept_pairs, void *stream) {
    PZ_RANGE("pz_set_centre_test");
    if (!c) return fail(PZ_EINVAL, "pz_set_centre_test: ctx is NULL");
    if (!(std::isfinite(eta) && eta >= 0.0)) return fail(PZ_EINVAL, "pz_set_centre_test: eta must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    drop_graph(c);
    c->have_kline = c->have_flux = c->have_inst = false;
    if (eta == 0.0) {
        PZ_CUDA(cudaStreamSynchronize(s), "pz_set_centre_test");
        dfree(c->d_keep);
        c->d_keep = nullptr;
        c->centre_eta = 0.0;
        if (kept_pairs) *kept_pairs = c->L.n * (int64_t)c->nd;
        return PZ_OK;
    }
    const size_t words = (size_t)std::max<int64_t>(c->L.n, 1) * kKeepWords;
    if (!c->d_keep) PZ_TRY(dalloc(&c->d_keep, words, "centre-test mask"));
    PZ_CUDA(cudaMemsetAsync(c->d_keep, 0, sizeof(uint32_t) * words, s), "pz_set_centre_test");
    unsigned long long *d_cnt = nullptr;
    if (kept_pairs) {
        PZ_TRY(dalloc(&d_cnt, 1, "pz_set_centre_test"));
        PZ_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), s), "pz_set_centre_test");
    }
    pz_status st = cuda_check(launch_centre_mask(c, eta, d_cnt, s), "pz_set_centre_test");
    c->launches = 1;
    if (st == PZ_OK && kept_pairs) {
        unsigned long long h = 0;
        if ((st = cuda_check(cudaMemcpyAsync(&h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, s), "pz_set_centre_test")) ==
            PZ_OK)
            st = cuda_check(cudaStreamSynchronize(s), "pz_set_centre_test");
        *kept_pairs = (int64_t)h;
    }
    dfree(d_cnt);
    if (st != PZ_OK) return st;
    c->centre_eta = eta;
    return PZ_OK;
}

pz_status pz_set_corrections(pz_ctx *c, const float *dgf, const float *dg6, const float *dab,
                             const int32_t *eos, int32_t n_elem, void *stream) {
    PZ_RANGE("pz_set_corrections");
    if (!c) return fail(PZ_EINVAL, "pz_set_corrections: ctx is NULL");
    if (n_elem < 0) return fail(PZ_EINVAL, "pz_set_corrections: n_elem < 0");
    if (dab && (n_elem == 0 || !eos)) return fail(PZ_EINVAL, "pz_set_corrections: dabund needs n_elem > 0 and elem_of_species");
    if (dab) {
        for (int s = 0; s < c->ns; ++s)
            if (eos[s] < -1 || eos[s] >= n_elem) return fail(PZ_EINVAL, "pz_set_corrections: elem_of_species out of range");
    }
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    const int64_t n = c->nl_caller;
    auto set_master = [&](const float *src, float *dst, const char *what) -> pz_status {
        if (!src) return cuda_check(cudaMemsetAsync(dst, 0, sizeof(float) * std::max<int64_t>(n, 1), s), what);
        if (n == 0) return PZ_OK;
        if (is_device_ptr(src))
            return cuda_check(cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyDeviceToDevice, s), what);
        PZ_CUDA(cudaStreamSynchronize(s), what);
        return cuda_check(cudaMemcpy(dst, src, sizeof(float) * n, cudaMemcpyHostToDevice), what);
    };
    PZ_TRY(set_master(dgf, c->d_mdgf, "dlog_gf"));
    PZ_TRY(set_master(dg6, c->d_mdg6, "dlog_gamma6"));
    if (dab) {
        if (n_elem != c->n_elem) {
            drop_graph(c);
            PZ_CUDA(cudaStreamSynchronize(s), "dabund");
            dfree(c->d_dab);
            dfree(c->d_gab);
            c->d_dab = nullptr;
            c->d_gab = nullptr;
            PZ_TRY(dalloc(&c->d_dab, n_elem, "dabund"));
        }
        std::vector<int32_t> heos(eos, eos + c->ns);
        PZ_CUDA(cudaStreamSynchronize(s), "elem_of_species");
        PZ_CUDA(cudaMemcpy(c->d_eos, heos.data(), sizeof(int32_t) * c->ns, cudaMemcpyHostToDevice), "elem_of_species");
        if (is_device_ptr(dab)) {
            PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] {
                        k_f32_to_f64<<<(n_elem + 255) / 256, 256, 0, s>>>(n_elem, dab, c->d_dab);
                        return cudaGetLastError();
                    }),
                    "dabund");
            c->launches++;
        } else {
            std::vector<double> h(dab, dab + n_elem);
            PZ_CUDA(cudaMemcpy(c->d_dab, h.data(), sizeof(double) * n_elem, cudaMemcpyHostToDevice), "dabund");
        }
        c->n_elem = n_elem;
    } else {
        if (c->n_elem != 0) drop_graph(c);
        c->n_elem = 0;
        std::vector<int32_t> heos(c->ns, -1);
        PZ_CUDA(cudaStreamSynchronize(s), "elem_of_species");
        PZ_CUDA(cudaMemcpy(c->d_eos, heos.data(), sizeof(int32_t) * c->ns, cudaMemcpyHostToDevice), "elem_of_species");
    }
    PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] { return launch_apply_corrections(c, s); }), "apply corrections");
    c->have_kline = c->have_flux = c->have_inst = false;
    return PZ_OK;
}

pz_status pz_get_corrections(pz_ctx *c, float *dgf, float *dg6, float *dab, void *stream) {
    PZ_RANGE("pz_get_corrections");
    if (!c) return fail(PZ_EINVAL, "pz_get_corrections: ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = c->nl_caller;
    if (dgf && n > 0) PZ_CUDA(cudaMemcpyAsync(dgf, c->d_mdgf, sizeof(float) * n, cudaMemcpyDefault, s), "dlog_gf");
    if (dg6 && n > 0) PZ_CUDA(cudaMemcpyAsync(dg6, c->d_mdg6, sizeof(float) * n, cudaMemcpyDefault, s), "dlog_gamma6");
    if (dab && c->n_elem > 0) {
        std::vector<double> h(c->n_elem);
        PZ_CUDA(cudaMemcpyAsync(h.data(), c->d_dab, sizeof(double) * c->n_elem, cudaMemcpyDeviceToHost, s), "dabund");
        PZ_CUDA(cudaStreamSynchronize(s), "dabund");
        std::vector<float> f(h.begin(), h.end());
        PZ_CUDA(cudaMemcpy(dab, f.data(), sizeof(float) * c->n_elem, cudaMemcpyDefault), "dabund");
    }
    PZ_CUDA(cudaStreamSynchronize(s), "pz_get_corrections");
    return PZ_OK;
}

pz_status pz_line_opacity(pz_ctx *c, float *kappa, void *stream) {
    PZ_RANGE("pz_line_opacity");
    if (!c) return fail(PZ_EINVAL, "pz_line_opacity: ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    PZ_CUDA(timed(c, s, PZ_K_LINE_FWD,
                  [&] { return c->prec == PZ_MIXED ? launch_line_fwd_mixed(c, s) : launch_line_fwd_fp64(c, s); }),
            "line opacity kernel");
    if (kappa) {
        const size_t rows = (size_t)c->S * c->nd;
        if (c->prec == PZ_MIXED) {
            PZ_CUDA(cudaMemcpy2DAsync(kappa, c->nlam * sizeof(float), c->d_kline, c->ld * sizeof(float),
                                      c->nlam * sizeof(float), rows, cudaMemcpyDeviceToDevice, s),
                    "copy kappa_line");
        } else {
            dim3 grid((unsigned)((c->nlam + 255) / 256), (unsigned)rows);
            PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] {
                        k_d2f_2d<<<grid, 256, 0, s>>>(c->nlam, c->ld, (const double *)c->d_kline, kappa);
                        return cudaGetLastError();
                    }),
                    "copy kappa_line");
            c->launches++;
        }
    }
    c->have_kline = true;
    c->have_flux = c->have_inst = false;
    return PZ_OK;
}

pz_status pz_flux(pz_ctx *c, double *F, double *Fc, void *stream) {
    PZ_RANGE("pz_flux");
    if (!c) return fail(PZ_EINVAL, "pz_flux: ctx is NULL");
    if (!c->have_kline) return fail(PZ_ESTATE, "pz_flux: call pz_line_opacity first");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    PZ_CUDA(timed(c, s, PZ_K_FLUX, [&] { return launch_flux(c, s); }), "flux kernel");
    const size_t nb = sizeof(double) * c->S * c->nlam;
    if (F) PZ_CUDA(cudaMemcpyAsync(F, c->d_F, nb, cudaMemcpyDeviceToDevice, s), "copy F");
    if (Fc) PZ_CUDA(cudaMemcpyAsync(Fc, c->d_Fc, nb, cudaMemcpyDeviceToDevice, s), "copy Fc");
    c->have_flux = true;
    c->have_inst = false;
    return PZ_OK;
}

pz_status pz_instrument(pz_ctx *c, double v_r, double v_b, double R_lsf, const double *pix, int64_t n_pix, float *f,
                        void *stream) {
    PZ_RANGE("pz_instrument");
    if (!c) return fail(PZ_EINVAL, "pz_instrument: ctx is NULL");
    if (!c->have_flux) return fail(PZ_ESTATE, "pz_instrument: call pz_flux first");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    if (n_pix < 0) return fail(PZ_EINVAL, "pz_instrument: n_pix < 0");
    if (n_pix == 0) {
        if (!c->identity_inst) drop_graph(c);
        PZ_TRY(ensure_out_buffers(c, c->nlam));
        c->identity_inst = true;
        c->n_out = c->nlam;
    } else {
        if (!pix) return fail(PZ_EINVAL, "pz_instrument: pix_lambda_nm is NULL");
        if (!finite_pos(R_lsf)) return fail(PZ_EINVAL, "pz_instrument: R_lsf must be > 0");
        if (!(std::isfinite(v_b) && v_b >= 0) || !std::isfinite(v_r) || std::fabs(v_r) > 1e5)
            return fail(PZ_EINVAL, "pz_instrument: v_r, v_b out of range");
        for (int64_t p = 0; p < n_pix; ++p) {
            if (!finite_pos(pix[p])) return fail(PZ_EINVAL, "pz_instrument: pixel wavelengths must be > 0");
            if (p > 0 && !(pix[p] > pix[p - 1])) return fail(PZ_EINVAL, "pz_instrument: pixels must be increasing");
        }
        double sig_lsf = 1.0 / (2.0 * std::sqrt(2.0 * std::log(2.0)) * R_lsf);
        double sig_b = v_b * 1e5 / kC;
        double sig = std::sqrt(sig_lsf * sig_lsf + sig_b * sig_b) / c->lnr;
        int64_t mt = 2 * (int64_t)std::ceil(5.0 * sig) + 2;
        if (mt > kMaxTaps) return fail(PZ_EINVAL, "pz_instrument: instrument kernel wider than 4096 grid points");
        bool same = !c->identity_inst && c->inst_key[0] == v_r && c->inst_key[1] == v_b && c->inst_key[2] == R_lsf &&
                    (int64_t)c->pix_key.size() == n_pix && std::equal(pix, pix + n_pix, c->pix_key.begin());
        if (!same) {
            drop_graph(c);
            if (c->n_pix < n_pix || c->max_taps < mt) {
                PZ_CUDA(cudaStreamSynchronize(s), "instrument");
                dfree(c->d_tap0);
                dfree(c->d_ntap);
                dfree(c->d_tapw);
                c->d_tap0 = c->d_ntap = nullptr;
                c->d_tapw = nullptr;
                PZ_TRY(dalloc(&c->d_tap0, n_pix, "instrument"));
                PZ_TRY(dalloc(&c->d_ntap, n_pix, "instrument"));
                PZ_TRY(dalloc(&c->d_tapw, (size_t)n_pix * mt, "instrument"));
            }
            c->n_pix = n_pix;
            c->max_taps = (int32_t)mt;
            double *d_pix = nullptr;
            int32_t *d_err = nullptr;
            PZ_TRY(dalloc(&d_pix, n_pix, "instrument"));
            PZ_TRY(dalloc(&d_err, 1, "instrument"));
            pz_status st = PZ_OK;
            int32_t herr = 0;
            if ((st = cuda_check(cudaMemcpyAsync(d_pix, pix, sizeof(double) * n_pix, cudaMemcpyHostToDevice, s), "pixels")) ==
                    PZ_OK &&
                (st = cuda_check(cudaMemsetAsync(d_err, 0, sizeof(int32_t), s), "pixels")) == PZ_OK &&
                (st = cuda_check(timed(c, s, PZ_K_INSTRUMENT,
                                       [&] { return launch_inst_build(c, d_pix, v_r, v_b, R_lsf, d_err, s); }),
                                 "instrument build")) == PZ_OK &&
                (st = cuda_check(cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "instrument build")) ==
                    PZ_OK)
                st = cuda_check(cudaStreamSynchronize(s), "instrument build");
            dfree(d_pix);
            dfree(d_err);
            if (st != PZ_OK) return st;
            if (herr) {
                c->identity_inst = true;
                c->n_out = 0;
                c->pix_key.clear();
                return fail(PZ_EINVAL, "pz_instrument: a pixel has no tap inside the synthesis grid");
            }
            c->inst_key[0] = v_r;
            c->inst_key[1] = v_b;
            c->inst_key[2] = R_lsf;
            c->pix_key.assign(pix, pix + n_pix);
        }
        PZ_TRY(ensure_out_buffers(c, n_pix));
        c->identity_inst = false;
        c->n_out = n_pix;
    }
    PZ_CUDA(timed(c, s, PZ_K_INSTRUMENT, [&] { return launch_inst_apply(c, f, s); }), "instrument apply");
    c->have_inst = true;
    return PZ_OK;
}

pz_status pz_loss_chi2(pz_ctx *c, const float *y, const float *w, int64_t n, double *loss, float *dLdf, void *stream) {
    PZ_RANGE("pz_loss_chi2");
    if (!c) return fail(PZ_EINVAL, "pz_loss_chi2: ctx is NULL");
    if (!c->have_inst) return fail(PZ_ESTATE, "pz_loss_chi2: call pz_instrument first");
    if (!y) return fail(PZ_EINVAL, "pz_loss_chi2: y is NULL");
    if (n != c->n_out) return fail(PZ_EINVAL, "pz_loss_chi2: n differs from the instrument output size");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    if (loss) PZ_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s), "loss");
    PZ_CUDA(timed(c, s, PZ_K_LOSS, [&] { return launch_loss(c, y, w, (int64_t)c->S * n, loss, dLdf, s); }),
            "loss kernel");
    return PZ_OK;
}

pz_status pz_backward(pz_ctx *c, const float *dLdf, float *g_gf, float *g_g6, float *g_ab, void *stream) {
    PZ_RANGE("pz_backward");
    if (!c) return fail(PZ_EINVAL, "pz_backward: ctx is NULL");
    if (!c->have_inst) return fail(PZ_ESTATE, "pz_backward: call pz_instrument first");
    if (!dLdf) return fail(PZ_EINVAL, "pz_backward: dL_df is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    PZ_TRY(ensure_backward_buffers(c));
    return enqueue_backward(c, dLdf, g_gf, g_g6, g_ab, s);
}

pz_status pz_backward4(pz_ctx *c, const float *dLdf, float *g_gf, float *g_rad, float *g_g4, float *g_g6,
                       float *g_ab, void *stream) {
    PZ_RANGE("pz_backward4");
    if (!c) return fail(PZ_EINVAL, "pz_backward4: ctx is NULL");
    if (!c->have_inst) return fail(PZ_ESTATE, "pz_backward4: call pz_instrument first");
    if (!dLdf) return fail(PZ_EINVAL, "pz_backward4: dL_df is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    PZ_TRY(ensure_backward_buffers(c));
    return enqueue_backward(c, dLdf, g_gf, g_g6, g_ab, s, true, g_rad, g_g4);
}

// One calibration step: corrections -> line opacity -> flux -> instrument -> chi^2 ->
// adjoint -> gradients -> delta -= lr * gradient, enqueued on the capture stream.
static pz_status enqueue_step(pz_ctx *c, const float *y, const float *w, double *loss, float *g_gf, float *g_g6,
                              float *g_ab, float lr_gf, float lr_g6, float lr_ab, cudaStream_t s) {
    PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] { return launch_apply_corrections(c, s); }), "apply corrections");
    PZ_CUDA(timed(c, s, PZ_K_LINE_FWD,
                  [&] { return c->prec == PZ_MIXED ? launch_line_fwd_mixed(c, s) : launch_line_fwd_fp64(c, s); }),
            "line opacity kernel");
    PZ_CUDA(timed(c, s, PZ_K_FLUX, [&] { return launch_flux(c, s); }), "flux kernel");
    PZ_CUDA(timed(c, s, PZ_K_INSTRUMENT, [&] { return launch_inst_apply(c, nullptr, s); }), "instrument apply");
    if (loss) PZ_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s), "loss");
    PZ_CUDA(timed(c, s, PZ_K_LOSS, [&] { return launch_loss(c, y, w, (int64_t)c->S * c->n_out, loss, c->d_dLdf, s); }),
            "loss kernel");
    PZ_TRY(enqueue_backward(c, c->d_dLdf, g_gf, g_g6, g_ab, s));
    PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] { return launch_update(c, lr_gf, lr_g6, lr_ab, s); }), "update");
    return PZ_OK;
}

pz_status pz_calib_step(pz_ctx *c, const float *y, const float *w, int64_t n, float lr_gf, float lr_g6, float lr_ab,
                        double *loss, float *g_gf, float *g_g6, float *g_ab, void *stream) {
    PZ_RANGE("pz_calib_step");
    if (!c) return fail(PZ_EINVAL, "pz_calib_step: ctx is NULL");
    if (c->n_out <= 0) return fail(PZ_ESTATE, "pz_calib_step: call pz_instrument once first");
    if (!y) return fail(PZ_EINVAL, "pz_calib_step: y is NULL");
    if (n != c->n_out) return fail(PZ_EINVAL, "pz_calib_step: n differs from the instrument output size");
    if (!std::isfinite(lr_gf) || !std::isfinite(lr_g6) || !std::isfinite(lr_ab))
        return fail(PZ_EINVAL, "pz_calib_step: learning rates must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    PZ_TRY(ensure_backward_buffers(c));
    if (!c->d_dLdf) PZ_TRY(dalloc(&c->d_dLdf, (size_t)c->S * c->pix_cap, "step seed"));
    StepGraph &G = c->graph;
    const void *key[6] = {y, w, loss, g_gf, g_g6, g_ab};
    bool same = G.exec && G.n == n && G.lr[0] == lr_gf && G.lr[1] == lr_g6 && G.lr[2] == lr_ab &&
                G.prof == c->profiling;
    for (int k = 0; k < 6 && same; ++k) same = G.key[k] == key[k];
    if (!same) {
        drop_graph(c);
        PZ_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "pz_calib_step: capture");
        c->capturing = true;
        c->launches = 0;
        c->cap_marks.clear();
        pz_status st = enqueue_step(c, y, w, loss, g_gf, g_g6, g_ab, lr_gf, lr_g6, lr_ab, c->cap_stream);
        c->capturing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
        if (st != PZ_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            destroy_marks(c->cap_marks);
            return st != PZ_OK ? st : cuda_check(e, "pz_calib_step: end capture");
        }
        e = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            G.exec = nullptr;
            destroy_marks(c->cap_marks);
            return cuda_check(e, "pz_calib_step: instantiate");
        }
        for (int k = 0; k < 6; ++k) G.key[k] = key[k];
        G.lr[0] = lr_gf;
        G.lr[1] = lr_g6;
        G.lr[2] = lr_ab;
        G.n = n;
        G.launches = c->launches;
        G.prof = c->profiling;
        G.marks.swap(c->cap_marks);
    }
    cudaEvent_t ev = prof_begin(c, s);
    cudaError_t e = cudaGraphLaunch(G.exec, s);
    prof_end(c, s, PZ_K_STEP, ev);
    PZ_CUDA(e, "pz_calib_step: graph launch");
    if (c->profiling) fold_graph_marks(c, G);
    c->launches = G.launches;
    c->have_kline = c->have_flux = c->have_inst = true;
    return PZ_OK;
}

// Caller-order master correction from host or device memory (NULL: zero).
static pz_status set_master_corr(pz_ctx *c, const float *src, float *dst, cudaStream_t s, const char *what) {
    const int64_t n = c->nl_caller;
    if (!src) return cuda_check(cudaMemsetAsync(dst, 0, sizeof(float) * std::max<int64_t>(n, 1), s), what);
    if (n == 0) return PZ_OK;
    if (is_device_ptr(src))
        return cuda_check(cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyDeviceToDevice, s), what);
    PZ_CUDA(cudaStreamSynchronize(s), what);
    return cuda_check(cudaMemcpy(dst, src, sizeof(float) * n, cudaMemcpyHostToDevice), what);
}

pz_status pz_set_damping_corrections(pz_ctx *c, const float *dgrad, const float *dg4, void *stream) {
    PZ_RANGE("pz_set_damping_corrections");
    if (!c) return fail(PZ_EINVAL, "pz_set_damping_corrections: ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    PZ_TRY(set_master_corr(c, dgrad, c->d_mdgrad, s, "dlog_gamma_rad"));
    PZ_TRY(set_master_corr(c, dg4, c->d_mdg4, s, "dlog_gamma4"));
    PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] { return launch_apply_corrections(c, s); }), "apply corrections");
    c->have_kline = c->have_flux = c->have_inst = false;
    return PZ_OK;
}

pz_status pz_get_damping_corrections(pz_ctx *c, float *dgrad, float *dg4, void *stream) {
    PZ_RANGE("pz_get_damping_corrections");
    if (!c) return fail(PZ_EINVAL, "pz_get_damping_corrections: ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = c->nl_caller;
    if (dgrad && n > 0)
        PZ_CUDA(cudaMemcpyAsync(dgrad, c->d_mdgrad, sizeof(float) * n, cudaMemcpyDefault, s), "dlog_gamma_rad");
    if (dg4 && n > 0) PZ_CUDA(cudaMemcpyAsync(dg4, c->d_mdg4, sizeof(float) * n, cudaMemcpyDefault, s), "dlog_gamma4");
    PZ_CUDA(cudaStreamSynchronize(s), "pz_get_damping_corrections");
    return PZ_OK;
}

pz_status pz_set_line_groups(pz_ctx *c, const int32_t *group_of_line, int64_t n_groups) {
    PZ_RANGE("pz_set_line_groups");
    if (!c) return fail(PZ_EINVAL, "pz_set_line_groups: ctx is NULL");
    if (n_groups < 0 || n_groups > std::max<int64_t>(c->nl_caller, 1))
        return fail(PZ_EINVAL, "pz_set_line_groups: n_groups must be in [0, n_lines]");
    if (n_groups > 0 && !group_of_line) return fail(PZ_EINVAL, "pz_set_line_groups: group_of_line is NULL");
    const int64_t n = c->nl_caller;
    std::vector<int32_t> q(std::max<int64_t>(n, 1), -1);
    std::vector<int64_t> off(n_groups + 1, 0);
    if (n_groups > 0) {
        for (int64_t k = 0; k < n; ++k) {
            const int32_t g = group_of_line[k];
            if (g < -1 || g >= n_groups) return fail(PZ_EINVAL, "pz_set_line_groups: group id out of range");
            q[k] = g;
            if (g >= 0) off[g + 1]++;
        }
    }
    for (int64_t g = 0; g < n_groups; ++g) off[g + 1] += off[g];
    std::vector<int32_t> mem(std::max<int64_t>(off[n_groups], 1), 0);
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    for (int64_t k = 0; k < n && n_groups > 0; ++k)
        if (q[k] >= 0) mem[fill[q[k]]++] = (int32_t)k;
    drop_graph(c);
    PZ_CUDA(cudaDeviceSynchronize(), "pz_set_line_groups");
    dfree(c->d_grp_of);
    dfree(c->d_grp_off);
    dfree(c->d_grp_mem);
    c->d_grp_of = nullptr;
    c->d_grp_off = nullptr;
    c->d_grp_mem = nullptr;
    c->n_groups = 0;
    if (n_groups == 0) return PZ_OK;
    PZ_TRY(upload(&c->d_grp_of, q, "line groups"));
    PZ_TRY(upload(&c->d_grp_off, off, "line groups"));
    PZ_TRY(upload(&c->d_grp_mem, mem, "line groups"));
    c->n_groups = n_groups;
    return PZ_OK;
}

// Group evaluation: group corrections -> line opacity -> flux -> instrument -> chi^2 ->
// four-family reverse pass -> group sums, enqueued on the capture stream.
static pz_status enqueue_group_eval(pz_ctx *c, const float *y, const float *w, const float *x, double *loss, float *g,
                                    cudaStream_t s) {
    PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] { return launch_group_gather(c, x, s); }), "group corrections");
    PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] { return launch_apply_corrections(c, s); }), "apply corrections");
    PZ_CUDA(timed(c, s, PZ_K_LINE_FWD,
                  [&] { return c->prec == PZ_MIXED ? launch_line_fwd_mixed(c, s) : launch_line_fwd_fp64(c, s); }),
            "line opacity kernel");
    PZ_CUDA(timed(c, s, PZ_K_FLUX, [&] { return launch_flux(c, s); }), "flux kernel");
    PZ_CUDA(timed(c, s, PZ_K_INSTRUMENT, [&] { return launch_inst_apply(c, nullptr, s); }), "instrument apply");
    if (loss) PZ_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s), "loss");
    PZ_CUDA(timed(c, s, PZ_K_LOSS, [&] { return launch_loss(c, y, w, (int64_t)c->S * c->n_out, loss, c->d_dLdf, s); }),
            "loss kernel");
    PZ_TRY(enqueue_backward(c, c->d_dLdf, nullptr, nullptr, nullptr, s, true, nullptr, nullptr));
    if (g) PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] { return launch_group_reduce(c, g, s); }), "group gradients");
    return PZ_OK;
}

pz_status pz_group_eval(pz_ctx *c, const float *y, const float *w, int64_t n, const float *x, double *loss, float *g,
                        void *stream) {
    PZ_RANGE("pz_group_eval");
    if (!c) return fail(PZ_EINVAL, "pz_group_eval: ctx is NULL");
    if (c->n_groups <= 0) return fail(PZ_ESTATE, "pz_group_eval: call pz_set_line_groups first");
    if (c->n_out <= 0) return fail(PZ_ESTATE, "pz_group_eval: call pz_instrument once first");
    if (!y || !x) return fail(PZ_EINVAL, "pz_group_eval: y and x are required");
    if (n != c->n_out) return fail(PZ_EINVAL, "pz_group_eval: n differs from the instrument output size");
    cudaStream_t s = (cudaStream_t)stream;
    PZ_TRY(ensure_backward_buffers(c));
    if (!c->d_dLdf) PZ_TRY(dalloc(&c->d_dLdf, (size_t)c->S * c->pix_cap, "step seed"));
    StepGraph &G = c->ggraph;
    const void *key[6] = {y, w, x, loss, g, nullptr};
    bool same = G.exec && G.n == n && G.prof == c->profiling;
    for (int k = 0; k < 6 && same; ++k) same = G.key[k] == key[k];
    if (!same) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        destroy_marks(G.marks);
        G = StepGraph();
        PZ_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "pz_group_eval: capture");
        c->capturing = true;
        c->launches = 0;
        c->cap_marks.clear();
        pz_status st = enqueue_group_eval(c, y, w, x, loss, g, c->cap_stream);
        c->capturing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
        if (st != PZ_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            destroy_marks(c->cap_marks);
            return st != PZ_OK ? st : cuda_check(e, "pz_group_eval: end capture");
        }
        e = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            G.exec = nullptr;
            destroy_marks(c->cap_marks);
            return cuda_check(e, "pz_group_eval: instantiate");
        }
        for (int k = 0; k < 6; ++k) G.key[k] = key[k];
        G.n = n;
        G.launches = c->launches;
        G.prof = c->profiling;
        G.marks.swap(c->cap_marks);
    }
    cudaEvent_t ev = prof_begin(c, s);
    cudaError_t e = cudaGraphLaunch(G.exec, s);
    prof_end(c, s, PZ_K_STEP, ev);
    PZ_CUDA(e, "pz_group_eval: graph launch");
    if (c->profiling) fold_graph_marks(c, G);
    c->launches = G.launches;
    c->have_kline = c->have_flux = c->have_inst = true;
    return PZ_OK;
}

pz_status pz_build_line_groups(int64_t n, const double *lambda_nm, const float *E_low_eV, const int32_t *species,
                               const float *strength, double dE_eV, double dlam_nm, int32_t *group_of_line,
                               int64_t *n_groups) {
    PZ_RANGE("pz_build_line_groups");
    if (n < 0 || (n > 0 && (!lambda_nm || !E_low_eV || !species || !strength || !group_of_line)) || !n_groups)
        return fail(PZ_EINVAL, "pz_build_line_groups: bad arguments");
    if (!(dE_eV >= 0.0) || !(dlam_nm >= 0.0) || !std::isfinite(dE_eV) || !std::isfinite(dlam_nm))
        return fail(PZ_EINVAL, "pz_build_line_groups: tolerances must be finite and >= 0");
    for (int64_t k = 0; k < n; ++k)
        if (!std::isfinite(strength[k]) || !std::isfinite(lambda_nm[k]) || !std::isfinite(E_low_eV[k]))
            return fail(PZ_EINVAL, "pz_build_line_groups: non-finite line data");
    // seeds from the strongest down (equal strengths by index)
    std::vector<int64_t> order(n);
    std::iota(order.begin(), order.end(), (int64_t)0);
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return strength[a] > strength[b] || (strength[a] == strength[b] && a < b);
    });
    // candidates: lines by (species, wavelength); a seed scans its species' wavelength
    // window, widened slightly so that the exact test below decides every boundary case
    std::vector<int64_t> by(n);
    std::iota(by.begin(), by.end(), (int64_t)0);
    std::sort(by.begin(), by.end(), [&](int64_t a, int64_t b) {
        if (species[a] != species[b]) return species[a] < species[b];
        if (lambda_nm[a] != lambda_nm[b]) return lambda_nm[a] < lambda_nm[b];
        return a < b;
    });
    std::vector<int32_t> q(n, -1);
    const double pad = dlam_nm * 1e-9 + 1e-9;
    int64_t G = 0;
    for (int64_t s : order) {
        if (q[s] >= 0) continue;
        if (G >= INT32_MAX) return fail(PZ_EINVAL, "pz_build_line_groups: too many groups");
        q[s] = (int32_t)G;
        const int32_t sp = species[s];
        const double ls = lambda_nm[s], es = (double)E_low_eV[s];
        auto lo = std::lower_bound(by.begin(), by.end(), s, [&](int64_t m, int64_t) {
            return species[m] < sp || (species[m] == sp && lambda_nm[m] < ls - dlam_nm - pad);
        });
        for (auto it = lo; it != by.end(); ++it) {
            const int64_t m = *it;
            if (species[m] != sp || lambda_nm[m] > ls + dlam_nm + pad) break;
            if (q[m] >= 0) continue;
            if (std::fabs((double)E_low_eV[m] - es) <= dE_eV && std::fabs(lambda_nm[m] - ls) <= dlam_nm)
                q[m] = (int32_t)G;
        }
        ++G;
    }
    for (int64_t k = 0; k < n; ++k) group_of_line[k] = q[k];
    *n_groups = G;
    return PZ_OK;
}

pz_status pz_set_scattering(pz_ctx *c, const double *sigma_c, void *stream) {
    PZ_RANGE("pz_set_scattering");
    if (!c) return fail(PZ_EINVAL, "pz_set_scattering: ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (!sigma_c) {
        if (c->d_sigma) {
            PZ_CUDA(cudaStreamSynchronize(s), "pz_set_scattering");
            dfree(c->d_sigma);
            c->d_sigma = nullptr;
        }
        c->have_flux = c->have_inst = false;
        return PZ_OK;
    }
    if (c->nd < 2) return fail(PZ_EINVAL, "pz_set_scattering: needs at least two layers");
    const size_t n = (size_t)c->S * c->nd * c->nlam;
    for (size_t k = 0; k < n; ++k)
        if (!(sigma_c[k] >= 0.0) || !std::isfinite(sigma_c[k]))
            return fail(PZ_EINVAL, "pz_set_scattering: sigma_c must be finite and >= 0");
    drop_graph(c);
    PZ_CUDA(cudaStreamSynchronize(s), "pz_set_scattering");
    if (!c->d_sigma) {
        PZ_TRY(dalloc(&c->d_sigma, (size_t)c->S * c->nd * c->ld, "sigma_c"));
        PZ_CUDA(cudaMemset(c->d_sigma, 0, sizeof(double) * (size_t)c->S * c->nd * c->ld), "sigma_c");
    }
    for (int st = 0; st < c->S; ++st)
        PZ_CUDA(cudaMemcpy2D(c->d_sigma + (size_t)st * c->nd * c->ld, c->ld * sizeof(double),
                             sigma_c + (size_t)st * c->nd * c->nlam, c->nlam * sizeof(double),
                             c->nlam * sizeof(double), c->nd, cudaMemcpyHostToDevice),
                "sigma_c");
    c->have_flux = c->have_inst = false;
    return PZ_OK;
}

pz_status pz_set_profiling(pz_ctx *c, int32_t enable) {
    PZ_RANGE("pz_set_profiling");
    if (!c) return fail(PZ_EINVAL, "pz_set_profiling: ctx is NULL");
    prof_fold(c);
    for (int k = 0; k < PZ_NK; ++k) {
        c->k_ms[k] = 0.0;
        c->k_count[k] = 0;
    }
    c->profiling = enable != 0;
    return PZ_OK;
}

pz_status pz_kernel_times(pz_ctx *c, double *ms, int64_t *counts, int32_t nk) {
    PZ_RANGE("pz_kernel_times");
    if (!c || nk < 0 || (nk > 0 && (!ms || !counts))) return fail(PZ_EINVAL, "pz_kernel_times: bad arguments");
    prof_fold(c);
    for (int k = 0; k < nk && k < PZ_NK; ++k) {
        ms[k] = c->k_ms[k];
        counts[k] = c->k_count[k];
    }
    for (int k = PZ_NK; k < nk; ++k) {
        ms[k] = 0.0;
        counts[k] = 0;
    }
    return PZ_OK;
}

pz_status pz_probe_voigt(const float *a, const float *v, int64_t n, float *H, float *dH, void *stream) {
    PZ_RANGE("pz_probe_voigt");
    if (n < 0 || (n > 0 && (!a || !v || !H))) return fail(PZ_EINVAL, "pz_probe_voigt: bad arguments");
    PZ_TRY(ensure_device_tables());
    PZ_CUDA(launch_probe_voigt(a, v, n, H, dH, (cudaStream_t)stream), "probe voigt");
    return PZ_OK;
}

pz_status pz_sync_status(pz_ctx *c, void *stream, int32_t *flags) {
    PZ_RANGE("pz_sync_status");
    if (!c) return fail(PZ_EINVAL, "pz_sync_status: ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int32_t h = 0;
    PZ_CUDA(cudaMemcpyAsync(&h, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "pz_sync_status");
    PZ_CUDA(cudaStreamSynchronize(s), "pz_sync_status");
    if (flags) *flags = h;
    if (h != 0) {
        PZ_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), s), "pz_sync_status");
        PZ_CUDA(cudaStreamSynchronize(s), "pz_sync_status");
        if (h & kStatusWaitGaveUp)
            return fail(PZ_ETIMEOUT, "pz_sync_status: a bounded device-side wait gave up (outputs incomplete)");
        return fail(PZ_ENUMERIC, "pz_sync_status: the scattering-source refinement did not converge for some "
                                 "wavelength (flux or gradients unreliable there)");
    }
    return PZ_OK;
}

pz_status pz_probe_wait(int64_t limit_ns, int32_t *flags, void *stream) {
    PZ_RANGE("pz_probe_wait");
    if (limit_ns < 1 || limit_ns > 1000000000) return fail(PZ_EINVAL, "pz_probe_wait: limit_ns must be in [1, 1e9]");
    if (!flags) return fail(PZ_EINVAL, "pz_probe_wait: flags is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *d = nullptr;
    PZ_TRY(dalloc(&d, 1, "pz_probe_wait"));
    pz_status st = PZ_OK;
    int32_t h = 0;
    if ((st = cuda_check(cudaMemsetAsync(d, 0, sizeof(int32_t), s), "pz_probe_wait")) == PZ_OK &&
        (st = cuda_check(launch_probe_wait((uint64_t)limit_ns, d, s), "pz_probe_wait")) == PZ_OK &&
        (st = cuda_check(cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "pz_probe_wait")) == PZ_OK)
        st = cuda_check(cudaStreamSynchronize(s), "pz_probe_wait");
    dfree(d);
    if (st != PZ_OK) return st;
    *flags = h;
    return PZ_OK;
}

pz_status pz_probe_pipe(int32_t pipe, int32_t iters, double *ops_per_s, void *stream) {
    PZ_RANGE("pz_probe_pipe");
    if (pipe < 0 || pipe > 2)
        return fail(PZ_EINVAL, "pz_probe_pipe: pipe must be 0 (FP32 FMA), 1 (MUFU) or 2 (FP64 FMA)");
    if (iters < 1 || iters > (1 << 20)) return fail(PZ_EINVAL, "pz_probe_pipe: iters must be in [1, 2^20]");
    if (!ops_per_s) return fail(PZ_EINVAL, "pz_probe_pipe: ops_per_s is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    PZ_CUDA(cudaGetDevice(&dev), "pz_probe_pipe");
    PZ_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "pz_probe_pipe");
    const int blocks = 8 * nsm;
    float *out = nullptr;
    PZ_TRY(dalloc(&out, (size_t)blocks * kProbeThreads, "pz_probe_pipe"));
    cudaEvent_t a = nullptr, b = nullptr;
    pz_status st = PZ_OK;
    float ms = 0.0f;
    if ((st = cuda_check(cudaEventCreate(&a), "pz_probe_pipe")) == PZ_OK &&
        (st = cuda_check(cudaEventCreate(&b), "pz_probe_pipe")) == PZ_OK &&
        (st = cuda_check(launch_probe_pipe(pipe, iters, blocks, out, s), "pz_probe_pipe")) == PZ_OK &&   // warm-up
        (st = cuda_check(cudaEventRecord(a, s), "pz_probe_pipe")) == PZ_OK &&
        (st = cuda_check(launch_probe_pipe(pipe, iters, blocks, out, s), "pz_probe_pipe")) == PZ_OK &&
        (st = cuda_check(cudaEventRecord(b, s), "pz_probe_pipe")) == PZ_OK &&
        (st = cuda_check(cudaEventSynchronize(b), "pz_probe_pipe")) == PZ_OK)
        st = cuda_check(cudaEventElapsedTime(&ms, a, b), "pz_probe_pipe");
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    dfree(out);
    if (st != PZ_OK) return st;
    const double per_thread = pipe == 0 ? 16.0 : 8.0;
    *ops_per_s = (double)blocks * kProbeThreads * per_thread * (double)iters / (ms * 1e-3);
    return PZ_OK;
}

pz_status pz_probe_expn(const double *x, int64_t n, double *out, void *stream) {
    PZ_RANGE("pz_probe_expn");
    if (n < 0 || (n > 0 && (!x || !out))) return fail(PZ_EINVAL, "pz_probe_expn: bad arguments");
    PZ_CUDA(launch_probe_expn(x, n, out, (cudaStream_t)stream), "probe expn");
    return PZ_OK;
}

}  // extern "C"
