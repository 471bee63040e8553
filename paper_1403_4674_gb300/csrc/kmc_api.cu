// kmc_api.cu -- host side of the C ABI declared in include/kmc.h.
//
// Owns the library's device scratch (bit tiles, edges, per-domain counters,
// launch plan, rate tables, error word), validates
// arguments, builds the fixed-point rate table on the host, plans which CTA
// (and which thread-block cluster) owns which domain, and enqueues the
// kernels of kmc_kernels.cuh on the caller's stream.
#include "kmc.h"
#include "kmc_kernels.cuh"
#include "kmc_ring.cuh"
#include "kmc_part.cuh"
#include "kmc_tpd.cuh"
#include "kmc_tpdr.cuh"
#include "kmc_tpdr64.cuh"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

using namespace kmcdev;

namespace {

// Host copy of a launch plan (see RunParams for the device arrays).
struct Plan {
    int mode = 0;     // KMC_LAUNCH_CLUSTER, KMC_LAUNCH_GRID or KMC_LAUNCH_THREADS (then cta_col_off holds the
                      // five offsets of the colour-sorted domain list slot_g; the other lists are empty)
    int cluster = 0;  // CTAs per cluster (CLUSTER mode)
    int n_cta = 0;
    int wpb = 0;
    int max_rt = 0;
    int max_slots = 0;
    size_t smem = 0;
    std::vector<uint32_t> cta_slot_off, cta_col_off, cta_rt_off, rt_rep, slot_g, slot_rt, slot_nb;
};

} // namespace

struct kmc_ctx {
    int dev = 0;
    int n_rep = 0;
    int LD = 0;
    int log2nd = 0;
    int k = 1;                       // default steps per visit
    std::vector<int32_t> L, Dx;
    std::vector<int32_t> kr, init_r; // per-replica steps per visit and start mode
    std::vector<uint64_t> seed;
    std::vector<uint32_t> dom_off;   // n_rep + 1
    std::vector<uint64_t> site_off;  // n_rep
    std::vector<uint64_t> blk_off;   // n_rep + 1
    std::vector<uint32_t> dom_rep;   // n_dom
    int n_dom = 0;
    int8_t *spins = nullptr;
    cudaStream_t stream = nullptr;

    int32_t *d_L = nullptr, *d_Dx = nullptr, *d_k = nullptr, *d_init = nullptr;
    uint32_t *d_dom_off = nullptr, *d_dom_rep = nullptr;
    uint64_t *d_site_off = nullptr, *d_blk_off = nullptr, *d_seed = nullptr;
    uint64_t *d_A = nullptr;
    int64_t *d_gfix = nullptr; // [n_rep][GFIX_WORDS] fixed-point score products
    double *d_grad = nullptr, *d_h = nullptr;
    uint8_t *d_tiles = nullptr;
    uint64_t *d_edges = nullptr, *d_dctr = nullptr;
    int *d_err = nullptr;
    unsigned long long *d_polls = nullptr; // halo-poll iterations (profiling)
    uint64_t *d_obs_dom = nullptr;         // thread plans: open observation record per domain
    unsigned long long *d_obs_acc = nullptr;
    size_t obs_acc_words = 0;
    void *d_tmp = nullptr; // n_dom * 32 + n_rep * 64 bytes, host-facing staging
    // device copy of the launch plan
    uint32_t *d_plan = nullptr;
    size_t plan_words = 0;

    double J = 1.0, nu = 1.0;
    std::vector<double> beta, h, a, gb, gh;
    std::vector<uint64_t> A;
    int law = KMC_RATE_METROPOLIS;

    int64_t sched_done = 0;
    int64_t visits_done = 0;
    int last_time_mode = KMC_TIME_EXPONENTIAL;
    bool clocks_exponential = true; // every run since the last reset drew exponential clock variates
    double dtau = 0.0;          // fixed-time visits (KMC_TIME_HORIZON): domain time per visit
    int hkmax = 0;
    uint64_t *d_htab = nullptr; // Poisson CDF thresholds, HORIZON_MAX_STEPS words
    int obs_unit = KMC_OBS_SCHEDULE;
    bool grad = false;

    int sm_count = 0, smem_optin = 0;
    Plan plan;
    int req_mode = KMC_LAUNCH_AUTO, req_size = 0, req_wpb = 16; // last requested plan
    int64_t launches = 0;
    int debug_extra = 0;
    uint64_t bar_limit_ns = 2000000000ull;
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
    std::string err;
};

// Working memory of kmc_run_schedule_noalloc: every GPU that loads this
// library holds these bytes until the process exits.  Host code must not use
// the symbol as an address; it resolves the device address per device with
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[KMC_NOALLOC_MAX_BYTES];

namespace {

const uint64_t DEFAULT_BAR_LIMIT_NS = 2000000000ull;
const int MAX_WPB = 16;

kmc_status fail(kmc_ctx *c, kmc_status s, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CUDA_TRY(ctx, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), KMC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

// Calls that copy from pageable host memory or synchronise cannot be part of
// a CUDA graph: refuse them while the context's stream is capturing.
bool capturing(const kmc_ctx *c)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st != cudaStreamCaptureStatusNone;
}

kmc_status refuse_capture(kmc_ctx *c, const char *what)
{
    if (capturing(c)) return fail(c, KMC_EINVAL, "%s cannot run while the stream is capturing a graph", what);
    return KMC_OK;
}

int ld_index(int LD) { return LD == 8 ? 0 : LD == 16 ? 1 : LD == 32 ? 2 : LD == 64 ? 3 : -1; }

int slot_bytes_for(int LD)
{
    return LD == 8 ? slot_bytes<8>() : LD == 16 ? slot_bytes<16>() : LD == 32 ? slot_bytes<32>() : slot_bytes<64>();
}

// Acceptance table (App. A, Eq. Glauber_TM): FP64 a_c, fixed point A_c =
// round(a_c 2^P), P = 63 - log2(n_d), reciprocal floor((2^64-1)/A_c) and the
// score derivatives d log a_c / d beta, d log a_c / d h.
void build_table(double J, double beta, double h, int law, int log2nd, double *a, uint64_t *A,
                 double *gb, double *gh)
{
    const int P = 63 - log2nd;
    for (int c = 0; c < 10; ++c) {
        const int up = c / 5, q = c % 5;
        const double sigma = up ? 1.0 : -1.0;
        const double dE = 2.0 * sigma * (J * (double)(2 * q - 4) + h);
        double ac, dlb, dlh;
        if (law == KMC_RATE_METROPOLIS) {
            if (dE <= 0.0) {
                ac = 1.0;
                dlb = 0.0;
                dlh = 0.0;
            } else {
                ac = std::exp(-beta * dE);
                dlb = -dE;
                dlh = -beta * 2.0 * sigma;
            }
        } else {
            ac = 1.0 / (1.0 + std::exp(beta * dE));
            dlb = -dE * (1.0 - ac);
            dlh = -beta * 2.0 * sigma * (1.0 - ac);
        }
        a[c] = ac;
        A[c] = (uint64_t)std::nearbyint(std::ldexp(ac, P));
        gb[c] = dlb;
        gh[c] = dlh;
    }
}

// First class whose fixed-point acceptance A_c rounded to 0 (n entries), or
// -1.  Every a_c of either law is positive for finite beta, so A_c = 0 would
// give the quantised chain a one-way rate: the flip out of class c never
// happens while its reverse does, and detailed balance (Eq. 4) fails.
int zero_rate_class(const uint64_t *A, int n)
{
    for (int c = 0; c < n; ++c)
        if (A[c] == 0) return c;
    return -1;
}

// NVTX range for the host span of one entry point that enqueues device work
// (visible in Nsight Systems, and usable as an Nsight Compute filter with
// --nvtx-include "kmc_run_schedule/"); the calls do nothing unless a tool
// is attached.
struct NvtxRange {
    explicit NvtxRange(const char *fmt, ...)
    {
        char buf[160];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Status of a failed cudaMalloc: out of device memory, or any other CUDA
// failure (no device, driver too old, a sticky error of the context).
kmc_status alloc_status(cudaError_t e)
{
    return (e == cudaErrorMemoryAllocation) ? KMC_ENOMEM : KMC_ECUDA;
}

template <typename T>
kmc_status dev_alloc(kmc_ctx *c, T **p, size_t n)
{
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, alloc_status(e), "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
    }
    return KMC_OK;
}

using RunKernel = void (*)(const RunParams);

RunKernel run_kernel_for(int LD, bool expo, bool grad, bool cluster)
{
#define KMC_PICK2(LDV, E, G)                                                   \
    if (LD == LDV && expo == E && grad == G)                                   \
        return cluster ? run_kernel<LDV, E, G, true> : run_kernel<LDV, E, G, false>;
#define KMC_PICK(LDV)                                                          \
    KMC_PICK2(LDV, true, true) KMC_PICK2(LDV, true, false) KMC_PICK2(LDV, false, true) KMC_PICK2(LDV, false, false)
    KMC_PICK(8)
    KMC_PICK(16)
    KMC_PICK(32)
    KMC_PICK(64)
#undef KMC_PICK
#undef KMC_PICK2
    return nullptr;
}

LayoutParams layout_params(kmc_ctx *c)
{
    LayoutParams P;
    P.n_rep = c->n_rep;
    P.n_dom = c->n_dom;
    P.rep_L = c->d_L;
    P.rep_Dx = c->d_Dx;
    P.rep_dom_off = c->d_dom_off;
    P.rep_site_off = c->d_site_off;
    P.rep_blk_off = c->d_blk_off;
    P.rep_seed = c->d_seed;
    P.rep_init = c->d_init;
    P.dom_rep = c->d_dom_rep;
    P.spins = c->spins;
    P.tiles = c->d_tiles;
    P.edges = c->d_edges;
    P.dctr = c->d_dctr;
    P.err = c->d_err;
    return P;
}

RunParams run_params(kmc_ctx *c)
{
    RunParams P;
    std::memset(&P, 0, sizeof P);
    P.n_rep = c->n_rep;
    P.rep_Dx = c->d_Dx;
    P.rep_k = c->d_k;
    P.rep_dom_off = c->d_dom_off;
    P.rep_seed = c->d_seed;
    P.rep_A = c->d_A;
    P.rep_gfix = c->d_gfix;
    P.rep_grad = c->d_grad;
    const Plan &pl = c->plan;
    uint32_t *base = c->d_plan;
    size_t off = 0;
    auto take = [&](size_t n) { uint32_t *p = base + off; off += n; return p; };
    P.cta_slot_off = take(pl.cta_slot_off.size());
    P.cta_col_off = take(pl.cta_col_off.size());
    P.cta_rt_off = take(pl.cta_rt_off.size());
    P.rt_rep = take(pl.rt_rep.size());
    P.slot_g = take(pl.slot_g.size());
    P.slot_rt = take(pl.slot_rt.size());
    P.slot_nb = take(pl.slot_nb.size());
    P.max_rt = pl.max_rt;
    P.cluster = pl.mode == KMC_LAUNCH_CLUSTER ? pl.cluster : 0;
    P.tiles = c->d_tiles;
    P.dctr = c->d_dctr;
    P.edges = c->d_edges;
    P.err = c->d_err;
    P.bar_limit_ns = c->bar_limit_ns;
    P.debug_extra = c->debug_extra;
    P.lambda = (double)(c->LD * c->LD) * c->nu;
    P.dom_rep = c->d_dom_rep;
    P.obs_dom = c->d_obs_dom;
    return P;
}

int grid_for(int n_items, int per_block)
{
    int g = (n_items + per_block - 1) / per_block;
    return std::max(1, std::min(g, 65535));
}

int domain_colour(const kmc_ctx *c, uint32_t g)
{
    const uint32_t r = c->dom_rep[g];
    const uint32_t d = g - c->dom_off[r];
    const int D = c->Dx[r];
    return (int)((d % D) & 1u) | (int)(((d / D) & 1u) << 1);
}

uint32_t neighbour(const kmc_ctx *c, uint32_t g, int side)
{
    const uint32_t r = c->dom_rep[g];
    const uint32_t d = g - c->dom_off[r];
    const int D = c->Dx[r];
    const int bx = (int)(d % D), by = (int)(d / D);
    int nx = bx, ny = by;
    if (side == EDGE_N) ny = (by + D - 1) % D;
    else if (side == EDGE_S) ny = (by + 1) % D;
    else if (side == EDGE_W) nx = (bx + D - 1) % D;
    else nx = (bx + 1) % D;
    return c->dom_off[r] + (uint32_t)(ny * D + nx);
}

// Fill per-CTA slot lists (colour-sorted), replica tables and neighbour refs
// from an assignment domain -> CTA.
void finish_plan(const kmc_ctx *c, Plan &pl, const std::vector<std::vector<uint32_t>> &cta_doms)
{
    const int slot_b = slot_bytes_for(c->LD);
    pl.n_cta = (int)cta_doms.size();
    pl.cta_slot_off.assign(1, 0);
    pl.cta_col_off.clear();
    pl.cta_rt_off.assign(1, 0);
    pl.rt_rep.clear();
    pl.slot_g.clear();
    pl.slot_rt.clear();
    pl.max_rt = 1;
    pl.max_slots = 1;
    std::vector<uint32_t> where_cta(c->n_dom, 0), where_slot(c->n_dom, 0);
    for (int b = 0; b < pl.n_cta; ++b) {
        std::vector<uint32_t> doms = cta_doms[b];
        std::stable_sort(doms.begin(), doms.end(), [&](uint32_t x, uint32_t y) {
            const int cx = domain_colour(c, x), cy = domain_colour(c, y);
            return cx != cy ? cx < cy : x < y;
        });
        std::vector<uint32_t> reps;
        for (uint32_t g : doms) reps.push_back(c->dom_rep[g]);
        std::sort(reps.begin(), reps.end());
        reps.erase(std::unique(reps.begin(), reps.end()), reps.end());
        uint32_t colc[5] = {0, 0, 0, 0, 0};
        for (size_t i = 0; i < doms.size(); ++i) {
            const uint32_t g = doms[i];
            colc[domain_colour(c, g) + 1]++;
            const uint32_t rt = (uint32_t)(std::lower_bound(reps.begin(), reps.end(), c->dom_rep[g]) - reps.begin());
            where_cta[g] = (uint32_t)b;
            where_slot[g] = (uint32_t)i;
            pl.slot_g.push_back(g);
            pl.slot_rt.push_back(rt);
        }
        for (int q = 1; q < 5; ++q) colc[q] += colc[q - 1];
        for (int q = 0; q < 5; ++q) pl.cta_col_off.push_back(colc[q]);
        pl.cta_slot_off.push_back((uint32_t)pl.slot_g.size());
        for (uint32_t r : reps) pl.rt_rep.push_back(r);
        pl.cta_rt_off.push_back((uint32_t)pl.rt_rep.size());
        pl.max_rt = std::max(pl.max_rt, (int)reps.size());
        pl.max_slots = std::max(pl.max_slots, (int)doms.size());
    }
    pl.slot_nb.resize(pl.slot_g.size() * 4);
    for (size_t s = 0; s < pl.slot_g.size(); ++s) {
        const uint32_t g = pl.slot_g[s];
        for (int side = 0; side < 4; ++side) {
            const uint32_t gn = neighbour(c, g, side);
            if (pl.mode == KMC_LAUNCH_CLUSTER) {
                const uint32_t cta = where_cta[gn];
                const uint32_t rank = cta % (uint32_t)pl.cluster;
                pl.slot_nb[s * 4 + side] = (rank << 24) | where_slot[gn];
            } else if (where_cta[gn] == where_cta[g]) {
                // same CTA: the halo is polled in shared memory (bit 31 flags it)
                pl.slot_nb[s * 4 + side] = 0x80000000u | where_slot[gn];
            } else {
                pl.slot_nb[s * 4 + side] = gn;
            }
        }
    }
    pl.smem = (size_t)pl.max_rt * RT_BYTES + (size_t)pl.max_slots * slot_b;
}

// CLUSTER plan: every replica inside one cluster of `C` CTAs; a replica with
// n domains spreads over m = ceil(n/4 / (wpb*load)) CTAs (one visit per warp
// and phase when load = 1); replicas that need one CTA share CTAs.  Replicas
// are packed in order of decreasing k, so that the CTAs of a cluster (which
// all wait for its slowest at the end of the launch) carry replicas of about
// equal cost per visit.
kmc_status plan_cluster(kmc_ctx *c, int C, int wpb, int load, Plan &pl)
{
    pl = Plan();
    pl.mode = KMC_LAUNCH_CLUSTER;
    pl.cluster = C;
    pl.wpb = wpb;
    const int slot_b = slot_bytes_for(c->LD);
    const int cap_per_colour = wpb * load;               // domains of one colour per CTA
    std::vector<std::vector<uint32_t>> cta_doms;
    std::vector<int> cta_fill;                           // per-colour domains in the CTA
    std::vector<int> cta_nrep;
    int cluster_base = -1;                               // first CTA of the open cluster
    auto open_cluster = [&]() {
        cluster_base = (int)cta_doms.size();
        for (int q = 0; q < C; ++q) {
            cta_doms.emplace_back();
            cta_fill.push_back(0);
            cta_nrep.push_back(0);
        }
    };
    std::vector<int> order(c->n_rep);
    for (int r = 0; r < c->n_rep; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return c->kr[x] > c->kr[y]; });
    for (int r : order) {
        const int n = c->Dx[r] * c->Dx[r];
        const int per_colour = n / 4;
        const int m = (per_colour + cap_per_colour - 1) / cap_per_colour;
        if (m > C) return fail(c, KMC_EINVAL, "replica %d (%d domains) needs %d CTAs, more than a cluster of %d", r, n, m, C);
        if ((size_t)RT_BYTES + (size_t)((n + m - 1) / m) * slot_b > (size_t)c->smem_optin)
            return fail(c, KMC_EINVAL, "replica %d does not fit in the shared memory of %d CTAs", r, m);
        std::vector<uint32_t> ctas;
        if (m == 1) {
            // first CTA of the open cluster with room (domains of all colours scale together)
            int pick = -1;
            if (cluster_base >= 0) {
                for (int q = cluster_base; q < cluster_base + C; ++q) {
                    const size_t smem_after = (size_t)(cta_nrep[q] + 1) * RT_BYTES +
                                              (cta_doms[q].size() + (size_t)n) * slot_b;
                    if (cta_fill[q] + per_colour <= cap_per_colour && smem_after <= (size_t)c->smem_optin) {
                        pick = q;
                        break;
                    }
                }
            }
            if (pick < 0) {
                open_cluster();
                pick = cluster_base;
            }
            ctas.push_back((uint32_t)pick);
        } else {
            // m empty CTAs at the end of the open cluster, else a new cluster
            int start = -1;
            if (cluster_base >= 0) {
                int q = cluster_base + C;
                while (q > cluster_base && cta_doms[q - 1].empty()) --q;
                if (cluster_base + C - q >= m) start = q;
            }
            if (start < 0) {
                open_cluster();
                start = cluster_base;
            }
            for (int q = 0; q < m; ++q) ctas.push_back((uint32_t)(start + q));
        }
        // colour-balanced round robin over the replica's CTAs
        int rr[4] = {0, 0, 0, 0};
        for (int d = 0; d < n; ++d) {
            const uint32_t g = c->dom_off[r] + (uint32_t)d;
            const int col = domain_colour(c, g);
            const uint32_t q = ctas[rr[col]++ % ctas.size()];
            cta_doms[q].push_back(g);
        }
        for (uint32_t q : ctas) {
            cta_fill[q] += (per_colour + (int)ctas.size() - 1) / (int)ctas.size();
            cta_nrep[q] += 1;
        }
    }
    finish_plan(c, pl, cta_doms);
    if (pl.smem > (size_t)c->smem_optin)
        return fail(c, KMC_EINVAL, "cluster plan needs %zu bytes of shared memory per CTA (%d available)", pl.smem,
                    c->smem_optin);
    return KMC_OK;
}

// GRID plan: each colour list (all replicas, ascending g) cut into n_cta
// contiguous chunks of equal estimated cost; a visit costs about k + 8
// step-equivalents (the fixed part is halo, class build and publication).
kmc_status plan_grid(kmc_ctx *c, int n_cta, int wpb, Plan &pl)
{
    pl = Plan();
    pl.mode = KMC_LAUNCH_GRID;
    pl.cluster = 0;
    pl.wpb = wpb;
    std::vector<std::vector<uint32_t>> lists(4);
    for (uint32_t g = 0; g < (uint32_t)c->n_dom; ++g) lists[domain_colour(c, g)].push_back(g);
    std::vector<std::vector<uint32_t>> cta_doms(n_cta);
    for (int q = 0; q < 4; ++q) {
        const std::vector<uint32_t> &lq = lists[q];
        uint64_t total = 0;
        for (uint32_t g : lq) total += (uint64_t)c->kr[c->dom_rep[g]] + 8;
        uint64_t acc = 0;
        int b = 0;
        for (uint32_t g : lq) {
            const uint64_t w = (uint64_t)c->kr[c->dom_rep[g]] + 8;
            // the chunk whose cost interval holds this domain's midpoint
            const uint64_t mid2 = 2 * acc + w; // twice the midpoint
            while (b + 1 < n_cta && mid2 * (uint64_t)n_cta >= 2 * total * (uint64_t)(b + 1)) ++b;
            cta_doms[b].push_back(g);
            acc += w;
        }
    }
    finish_plan(c, pl, cta_doms);
    if (pl.smem > (size_t)c->smem_optin)
        return fail(c, KMC_EINVAL, "grid plan needs %zu bytes of shared memory per CTA (%d available)", pl.smem,
                    c->smem_optin);
    return KMC_OK;
}

// THREADS plan (L_d = 8): the domains sorted by colour, then by id, so that
// consecutive threads hold neighbouring domains of one replica.
kmc_status plan_threads(kmc_ctx *c, int n_cta, int wpb, Plan &pl)
{
    if (c->LD != 8) return fail(c, KMC_EINVAL, "the thread-per-domain plan needs L_d = 8 (L_d = %d)", c->LD);
    if (n_cta < 1) return fail(c, KMC_EINVAL, "thread plan needs >= 1 CTA");
    pl = Plan();
    pl.mode = KMC_LAUNCH_THREADS;
    pl.n_cta = n_cta;
    pl.wpb = wpb;
    std::vector<std::vector<uint32_t>> lists(4);
    for (uint32_t g = 0; g < (uint32_t)c->n_dom; ++g) lists[domain_colour(c, g)].push_back(g);
    pl.cta_col_off.assign(5, 0);
    for (int q = 0; q < 4; ++q) {
        pl.slot_g.insert(pl.slot_g.end(), lists[q].begin(), lists[q].end());
        pl.cta_col_off[q + 1] = (uint32_t)pl.slot_g.size();
    }
    pl.smem = 0;
    return KMC_OK;
}

using TpdKernel = void (*)(const RunParams);
// the thread-per-domain kernel of the context's domain side (scores: the
// shared-memory kernel of 16x16 and 32x32 domains only)
TpdKernel tpd_kernel_for(int LD, bool expo, bool grad)
{
    if (LD == 64) return expo ? tpdr64_kernel<true> : tpdr64_kernel<false>;
    if (LD == 16)
        return grad ? (expo ? tpdr_kernel<16, true, true> : tpdr_kernel<16, false, true>)
                    : (expo ? tpdr_kernel<16, true, false> : tpdr_kernel<16, false, false>);
    if (LD == 32)
        return grad ? (expo ? tpdr_kernel<32, true, true> : tpdr_kernel<32, false, true>)
                    : (expo ? tpdr_kernel<32, true, false> : tpdr_kernel<32, false, false>);
    return expo ? tpd_kernel<true> : tpd_kernel<false>;
}
size_t tpdr_warp_bytes_for(int LD)
{
    return LD == 16 ? tpdr_warp_bytes<16>() : LD == 32 ? tpdr_warp_bytes<32>() : tpdr64_warp_bytes();
}

// THREADS plan for L_d = 16, 32: warps of 32 domains of one colour, one per
// thread and consecutive in the colour list (a colour's last warp may be
// partly empty), the colours' warps interleaved so that a CTA holds
// neighbouring groups of every colour; slot_g holds 32 entries per warp of
// the grid, 0xFFFFFFFF for an empty lane or warp.  The domains stay in the
// CTA's shared memory for the whole launch.  The colour list holds the
// replicas one after another, or with `interleave` their domains dealt
// round-robin (the first of each replica, then the second, ...), so that a
// warp's 32 domains come from many replicas: a warp's visit lasts as long as
// its busiest lane, and a replica's chain of visits then waits on fewer of
// its own busiest domains at a time.  That pays when the replicas differ in
// cost (steps per visit, temperature): 1024^2 x 18 workload 661 -> 598 ms;
// on a batch of alike replicas it couples the replicas' dataflow for
// nothing (256 x 256^2 with scores: 278 -> 322 ms).
kmc_status plan_thread_rows(kmc_ctx *c, int wpb, Plan &pl, bool interleave)
{
    if (c->LD != 16 && c->LD != 32 && c->LD != 64) return fail(c, KMC_EINVAL, "no thread-row kernel for L_d = %d", c->LD);
    if (wpb < 1 || wpb > 4) return fail(c, KMC_EINVAL, "thread plans take 1..4 warps per CTA");
    pl = Plan();
    pl.mode = KMC_LAUNCH_THREADS;
    pl.wpb = wpb;
    std::vector<std::vector<uint32_t>> lists(4);
    if (!interleave) {
        for (uint32_t g = 0; g < (uint32_t)c->n_dom; ++g) lists[domain_colour(c, g)].push_back(g);
    } else {
        std::vector<std::vector<std::vector<uint32_t>>> per(4, std::vector<std::vector<uint32_t>>(c->n_rep));
        for (uint32_t g = 0; g < (uint32_t)c->n_dom; ++g) per[domain_colour(c, g)][c->dom_rep[g]].push_back(g);
        for (int q = 0; q < 4; ++q) {
            size_t longest = 0;
            for (const auto &v : per[q]) longest = std::max(longest, v.size());
            for (size_t j = 0; j < longest; ++j)
                for (const auto &v : per[q])
                    if (j < v.size()) lists[q].push_back(v[j]);
        }
    }
    size_t most = 0;
    for (const auto &lq : lists) most = std::max(most, (lq.size() + 31) / 32);
    for (size_t i = 0; i < most; ++i) {
        for (int q = 0; q < 4; ++q) {
            const std::vector<uint32_t> &lq = lists[q];
            if (i * 32 >= lq.size()) continue;
            for (size_t l = 0; l < 32; ++l) pl.slot_g.push_back(i * 32 + l < lq.size() ? lq[i * 32 + l] : 0xFFFFFFFFu);
        }
    }
    const int n_warps = (int)(pl.slot_g.size() / 32);
    pl.n_cta = (n_warps + wpb - 1) / wpb;
    pl.slot_g.resize((size_t)pl.n_cta * wpb * 32, 0xFFFFFFFFu);
    pl.smem = (size_t)wpb * tpdr_warp_bytes_for(c->LD);
    return KMC_OK;
}

// CTAs of `wpb` warps for a thread plan: a phase takes as many rounds as its
// busiest thread has domains, so the threads are the domains of a colour
// divided by the rounds that up to three CTAs of 4 warps per SM need (the
// fastest grid on the 512-replica batch, measured; more resident warps left
// threads with one domain beside threads with two).
int balanced_thread_ctas(const kmc_ctx *c, int wpb)
{
    const int64_t per_colour = (c->n_dom + 3) / 4;
    const int64_t tmax = (int64_t)3 * 128 * c->sm_count;
    const int64_t rounds = std::max<int64_t>(1, (per_colour + tmax - 1) / tmax);
    const int64_t threads = (per_colour + rounds - 1) / rounds;
    const int64_t per_cta = (int64_t)wpb * 32;
    return (int)std::max<int64_t>(1, (threads + per_cta - 1) / per_cta);
}

// Can this plan run?  Shared memory, cluster support and (GRID) co-residency.
// Only the kernels this context can launch are checked: both clock modes,
// and the score-carrying variant only while scores are on (it holds more
// registers, so fewer of its CTAs fit an SM; kmc_enable_grad re-checks).
kmc_status check_plan(kmc_ctx *c, const Plan &pl)
{
    if (pl.mode == KMC_LAUNCH_THREADS) {
        if (c->grad && (c->LD == 8 || c->LD == 64))
            return fail(c, KMC_EINVAL, "the thread-per-domain plan of L_d = %d has no score kernel", c->LD);
        for (int e = 0; e < 2; ++e) {
            const void *kern = (const void *)tpd_kernel_for(c->LD, e == 0, c->grad);
            if (pl.smem > 0) {
                if (pl.smem > (size_t)c->smem_optin)
                    return fail(c, KMC_EINVAL, "thread plan needs %zu bytes of shared memory per CTA (%d available)",
                                pl.smem, c->smem_optin);
                cudaFuncAttributes fa;
                CUDA_TRY(c, cudaFuncGetAttributes(&fa, kern));
                if ((size_t)fa.maxDynamicSharedSizeBytes < pl.smem)
                    CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
            }
            int nb = 0;
            CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, pl.wpb * 32, pl.smem));
            if ((int64_t)nb * c->sm_count < pl.n_cta)
                return fail(c, KMC_EINVAL, "%d CTAs of %d warps cannot be co-resident (%d per SM)", pl.n_cta, pl.wpb, nb);
        }
        if (c->LD != 8) return KMC_OK;
        if (!c->d_obs_dom) {
            kmc_status st = dev_alloc(c, &c->d_obs_dom, (size_t)c->n_dom * TPD_OBS_WORDS);
            if (st != KMC_OK) return st;
        }
        return KMC_OK;
    }
    for (int e = 0; e < 2; ++e) {
        for (int gv = 0; gv < 2; ++gv) {
            if (gv == 1 && !c->grad) continue;
            RunKernel kern = run_kernel_for(c->LD, e == 0, gv == 1, pl.mode == KMC_LAUNCH_CLUSTER);
            // the attribute belongs to the kernel, not to the context: only
            // ever raise it, so that plans of other contexts stay launchable
            cudaFuncAttributes fa;
            CUDA_TRY(c, cudaFuncGetAttributes(&fa, (const void *)kern));
            if ((size_t)fa.maxDynamicSharedSizeBytes < pl.smem)
                CUDA_TRY(c, cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
            if (pl.mode == KMC_LAUNCH_CLUSTER) {
                if (pl.cluster > 8)
                    CUDA_TRY(c, cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(pl.n_cta);
                cfg.blockDim = dim3(pl.wpb * 32);
                cfg.dynamicSmemBytes = pl.smem;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = pl.cluster;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                int ncl = 0;
                cudaError_t ce = cudaOccupancyMaxActiveClusters(&ncl, (const void *)kern, &cfg);
                if (ce != cudaSuccess || ncl < 1) {
                    cudaGetLastError();
                    return fail(c, KMC_EINVAL, "clusters of %d CTAs x %d warps with %zu bytes cannot be scheduled (%s)",
                                pl.cluster, pl.wpb, pl.smem, ce != cudaSuccess ? cudaGetErrorString(ce) : "0 active clusters");
                }
            } else {
                int nb = 0;
                CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)kern, pl.wpb * 32, pl.smem));
                if ((int64_t)nb * c->sm_count < pl.n_cta)
                    return fail(c, KMC_EINVAL, "%d CTAs of %d warps cannot be co-resident (%d per SM)", pl.n_cta, pl.wpb, nb);
            }
        }
    }
    return KMC_OK;
}

kmc_status install_plan(kmc_ctx *c, Plan &pl)
{
    kmc_status s = check_plan(c, pl);
    if (s != KMC_OK) return s;
    std::vector<uint32_t> flat;
    for (auto *v : {&pl.cta_slot_off, &pl.cta_col_off, &pl.cta_rt_off, &pl.rt_rep, &pl.slot_g, &pl.slot_rt, &pl.slot_nb})
        flat.insert(flat.end(), v->begin(), v->end());
    if (flat.size() > c->plan_words) {
        if (c->d_plan) cudaFree(c->d_plan);
        c->d_plan = nullptr;
        c->plan_words = 0;
        if ((s = dev_alloc(c, &c->d_plan, flat.size())) != KMC_OK) return s;
        c->plan_words = flat.size();
    }
    CUDA_TRY(c, cudaMemcpy(c->d_plan, flat.data(), flat.size() * 4, cudaMemcpyHostToDevice));
    c->plan = std::move(pl);
    return KMC_OK;
}

kmc_status default_warp_plan(kmc_ctx *c);

// The library's plan: one thread per domain (a warp then runs 32 domain
// processes): for 8x8 domains with state in L2 and for 64x64 domains with
// state in shared memory while scores are off, for 16x16 and 32x32 domains
// with state in shared memory with or without scores, when it fits the GPU;
// else the warp plans below.
kmc_status default_plan(kmc_ctx *c)
{
    if ((!c->grad && (c->LD == 8 || c->LD == 64)) || c->LD == 16 || c->LD == 32) {
        Plan pl;
        const kmc_status st = (c->LD == 8) ? plan_threads(c, balanced_thread_ctas(c, 4), 4, pl)
                                           : plan_thread_rows(c, 1, pl, false);
        if (st == KMC_OK && install_plan(c, pl) == KMC_OK) return KMC_OK;
        cudaGetLastError();
    }
    return default_warp_plan(c);
}

// Warp plans: clusters when every replica fits one (smallest power of two
// that covers the largest replica at one visit per warp and phase, up to 16);
// otherwise the cooperative grid; if the batch's state does not fit the
// grid's shared memory, clusters of 16 CTAs with several visits per warp and
// phase (clusters run in waves, so the batch need not be resident at once).
kmc_status default_warp_plan(kmc_ctx *c)
{
    int need = 1;
    for (int r = 0; r < c->n_rep; ++r) {
        const int per_colour = c->Dx[r] * c->Dx[r] / 4;
        need = std::max(need, (per_colour + MAX_WPB - 1) / MAX_WPB);
    }
    int C = 1;
    while (C < need) C *= 2;
    std::string why;
    if (C <= 16) {
        int total_pc = 0;
        for (int r = 0; r < c->n_rep; ++r) total_pc += c->Dx[r] * c->Dx[r] / 4;
        for (int cl = C; cl <= 16; cl *= 2) {
            // domains of one colour per warp: keep the CTA count within one wave
            int load = 1;
            while (load < 64 && (int64_t)((total_pc + MAX_WPB * load - 1) / (MAX_WPB * load)) > (int64_t)c->sm_count)
                ++load;
            Plan pl;
            if (plan_cluster(c, cl, MAX_WPB, load, pl) == KMC_OK && install_plan(c, pl) == KMC_OK) return KMC_OK;
            why = c->err;
        }
    }
    // cooperative grids, most resident warps per SM first (the 80-register
    // kernels fit three CTAs of 8 warps or two of 12 on an SM, the 96-register
    // ones two of 10)
    const int grid_shapes[][2] = {{8, 3}, {12, 2}, {10, 2}, {16, 1}, {8, 2}, {8, 1}, {4, 1}};
    for (const auto &gs : grid_shapes) {
        Plan pl;
        if (plan_grid(c, c->sm_count * gs[1], gs[0], pl) == KMC_OK && install_plan(c, pl) == KMC_OK) return KMC_OK;
        why = c->err;
    }
    {
        const int load = (need + 15) / 16;
        Plan pl;
        if (plan_cluster(c, 16, MAX_WPB, load, pl) == KMC_OK && install_plan(c, pl) == KMC_OK) return KMC_OK;
        why = c->err;
    }
    return fail(c, KMC_EINVAL, "no launch plan fits this batch: %s", why.c_str());
}

// Endpoint observables of the packed state into acc[n_rep][OBS_WORDS]
// (bond sum, magnetisation, summed domain clocks, summed scores).
kmc_status launch_observe(kmc_ctx *c, cudaStream_t s, int time_mode, unsigned long long *acc)
{
    CUDA_TRY(c, cudaMemsetAsync(acc, 0, (size_t)c->n_rep * OBS_WORDS * 8, s));
    RunParams P = run_params(c);
    const bool expo = time_mode == KMC_TIME_EXPONENTIAL;
    P.horizon = time_mode == KMC_TIME_HORIZON;
    P.dtau = c->dtau;
    const int blocks = grid_for(c->n_dom, 8);
#define KMC_OBS(LDV)                                                                                         \
    if (expo) observe_kernel<LDV, true><<<blocks, 256, 0, s>>>(P, c->d_dom_rep, c->n_dom, c->visits_done, acc); \
    else observe_kernel<LDV, false><<<blocks, 256, 0, s>>>(P, c->d_dom_rep, c->n_dom, c->visits_done, acc);
    switch (c->LD) {
    case 8: KMC_OBS(8) break;
    case 16: KMC_OBS(16) break;
    case 32: KMC_OBS(32) break;
    default: KMC_OBS(64) break;
    }
#undef KMC_OBS
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    return KMC_OK;
}

// Fixed-point products x_c = a_c dlog a_c / d(beta, h) for the score of null
// steps, in two words: X_c = round(x_c 2^Q) (int64) and the low word Y_c =
// round((x_c 2^Q - X_c) 2^GFIX_LO_BITS) (int32, |Y_c| <= 2^17).  Q is as large
// as keeps the device's per-state sum sum_c n_c X_c 2^GFIX_T_BITS inside
// int64: sum_c n_c |x_c| 2^Q < n_d 2^e 2^Q = 2^58 with |x_c| < 2^e.  Also
// stores 2^-(Q + GFIX_T_BITS), the unit of the combined per-state sum.
// Returns false when Q would fall below 8 fraction bits (|a dlog a| of order
// 2^(50 - log2 n_d) or more).
bool build_gfix(const double *a, const double *gb, const double *gh, int log2nd, int64_t *out)
{
    double mx = 0.0;
    for (int c = 0; c < 10; ++c) mx = std::max(mx, std::max(std::fabs(a[c] * gb[c]), std::fabs(a[c] * gh[c])));
    int Q = 62;
    if (mx > 0.0) {
        int e = 0;
        std::frexp(mx, &e); // mx < 2^e
        Q = std::min(62, 58 - log2nd - e);
        if (Q < 8) return false;
    }
    int32_t *yb = reinterpret_cast<int32_t *>(&out[GFIX_YB]);
    int32_t *yh = reinterpret_cast<int32_t *>(&out[GFIX_YH]);
    // x_c = a_c * g_c as the exact real product of the two doubles: the
    // rounded product p and its rounding error fma(a, g, -p) (exact), so
    // that the words do not carry the product's rounding, which would be the
    // same in every state.  p 2^Q is exact (power-of-two scaling) and so is
    // its difference from the nearest integer.
    auto split = [&](double av, double gv, int64_t &X, int32_t &Y) {
        const double p = av * gv;
        const double perr = std::fma(av, gv, -p);
        const double x = std::ldexp(p, Q);
        const double Xd = std::nearbyint(x);
        X = (int64_t)Xd;
        Y = (int32_t)std::nearbyint(std::ldexp((x - Xd) + std::ldexp(perr, Q), GFIX_LO_BITS));
    };
    for (int c = 0; c < 10; ++c) {
        split(a[c], gb[c], out[c], yb[c]);
        split(a[c], gh[c], out[10 + c], yh[c]);
    }
    const double scale = std::ldexp(1.0, -(Q + GFIX_T_BITS));
    std::memcpy(&out[20], &scale, 8);
    out[21] = 0;
    return true;
}

kmc_status sync_ctx(kmc_ctx *c);

// Per-domain counters to host arrays of n_dom entries (any may be NULL).
kmc_status domain_state(kmc_ctx *c, uint64_t *hash, int64_t *flips, double *t, int64_t *steps)
{
    cudaStream_t s = c->stream;
    uint64_t *dh = reinterpret_cast<uint64_t *>(c->d_tmp);
    int64_t *df = reinterpret_cast<int64_t *>(dh + c->n_dom);
    double *dt = reinterpret_cast<double *>(df + c->n_dom);
    int64_t *ds = reinterpret_cast<int64_t *>(dt + c->n_dom);
    const double lambda = (double)(c->LD * c->LD) * c->nu;
    const double dtau = c->last_time_mode == KMC_TIME_HORIZON ? c->dtau : 0.0;
    if (c->last_time_mode == KMC_TIME_EXPONENTIAL)
        domain_state_kernel<true><<<grid_for(c->n_dom, 256), 256, 0, s>>>(
            c->d_dctr, c->n_dom, c->visits_done, c->d_dom_rep, c->d_k, lambda, dtau, dh, df, dt, ds);
    else
        domain_state_kernel<false><<<grid_for(c->n_dom, 256), 256, 0, s>>>(
            c->d_dctr, c->n_dom, c->visits_done, c->d_dom_rep, c->d_k, lambda, dtau, dh, df, dt, ds);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    const size_t n = (size_t)c->n_dom;
    if (hash) CUDA_TRY(c, cudaMemcpyAsync(hash, dh, n * 8, cudaMemcpyDeviceToHost, s));
    if (flips) CUDA_TRY(c, cudaMemcpyAsync(flips, df, n * 8, cudaMemcpyDeviceToHost, s));
    if (t) CUDA_TRY(c, cudaMemcpyAsync(t, dt, n * 8, cudaMemcpyDeviceToHost, s));
    if (steps) CUDA_TRY(c, cudaMemcpyAsync(steps, ds, n * 8, cudaMemcpyDeviceToHost, s));
    return sync_ctx(c);
}

// Poisson CDF thresholds of the fixed-time visit: floor(F(k) 2^64) for
// k < kmax = ceil(mu + 12 sqrt(mu) + 30), mu = n_d nu dtau, with the pmf
// exp(-mu + k ln mu - lnGamma(k + 1)) summed in k order.
kmc_status upload_horizon(kmc_ctx *c)
{
    if (!(c->dtau > 0.0)) return KMC_OK;
    const double mu = (double)(c->LD * c->LD) * c->nu * c->dtau;
    const int kmax = (int)std::ceil(mu + 12.0 * std::sqrt(mu) + 30.0);
    if (kmax > HORIZON_MAX_STEPS)
        return fail(c, KMC_EINVAL, "visit time too long: n_d nu dtau = %g needs %d > %d table entries", mu, kmax,
                    HORIZON_MAX_STEPS);
    if (!c->d_htab) {
        kmc_status st = dev_alloc(c, &c->d_htab, HORIZON_MAX_STEPS);
        if (st != KMC_OK) return st;
    }
    std::vector<uint64_t> tab(kmax);
    const double logmu = std::log(mu);
    double F = 0.0;
    for (int k = 0; k < kmax; ++k) {
        const double lp = -mu + (double)k * logmu - std::lgamma((double)k + 1.0);
        F += std::exp(lp);
        tab[k] = (F >= 1.0) ? UINT64_MAX : (uint64_t)std::ldexp(F, 64);
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_htab, tab.data(), (size_t)kmax * 8, cudaMemcpyHostToDevice, c->stream));
    c->hkmax = kmax;
    return KMC_OK; // pageable source: consumed when the copy returns
}

kmc_status upload_rates(kmc_ctx *c)
{
    std::vector<uint64_t> A16((size_t)c->n_rep * 16, 0);
    std::vector<int64_t> gfix((size_t)c->n_rep * GFIX_WORDS, 0);
    std::vector<double> g32((size_t)c->n_rep * 32, 0.0);
    for (int r = 0; r < c->n_rep; ++r) {
        for (int q = 0; q < 10; ++q) {
            A16[(size_t)r * 16 + q] = c->A[(size_t)r * 10 + q];
            g32[(size_t)r * 32 + q] = c->a[(size_t)r * 10 + q];
            g32[(size_t)r * 32 + 10 + q] = c->gb[(size_t)r * 10 + q];
            g32[(size_t)r * 32 + 20 + q] = c->gh[(size_t)r * 10 + q];
        }
    }
    // ordered on the context's stream, after any run already queued there; the
    // sources are pageable, so each copy has consumed them when the call returns
    CUDA_TRY(c, cudaMemcpyAsync(c->d_A, A16.data(), A16.size() * 8, cudaMemcpyHostToDevice, c->stream));
    for (int r = 0; r < c->n_rep; ++r)
        if (!build_gfix(&c->a[(size_t)r * 10], &c->gb[(size_t)r * 10], &c->gh[(size_t)r * 10], c->log2nd,
                        &gfix[(size_t)r * GFIX_WORDS]))
            return fail(c, KMC_EINVAL, "replica %d: score products a_c dlog a_c too large for fixed point", r);
    CUDA_TRY(c, cudaMemcpyAsync(c->d_gfix, gfix.data(), gfix.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_grad, g32.data(), g32.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_h, c->h.data(), c->h.size() * 8, cudaMemcpyHostToDevice, c->stream));
    return upload_horizon(c); // the table depends on nu
}

kmc_status launch_pack(kmc_ctx *c, cudaStream_t s)
{
    LayoutParams P = layout_params(c);
    const int blocks = grid_for(c->n_dom, 8);
    switch (c->LD) {
    case 8: pack_kernel<8><<<blocks, 256, 0, s>>>(P); break;
    case 16: pack_kernel<16><<<blocks, 256, 0, s>>>(P); break;
    case 32: pack_kernel<32><<<blocks, 256, 0, s>>>(P); break;
    default: pack_kernel<64><<<blocks, 256, 0, s>>>(P); break;
    }
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    return KMC_OK;
}

kmc_status launch_unpack(kmc_ctx *c, cudaStream_t s)
{
    LayoutParams P = layout_params(c);
    const int blocks = grid_for(c->n_dom, 8);
    switch (c->LD) {
    case 8: unpack_kernel<8><<<blocks, 256, 0, s>>>(P); break;
    case 16: unpack_kernel<16><<<blocks, 256, 0, s>>>(P); break;
    case 32: unpack_kernel<32><<<blocks, 256, 0, s>>>(P); break;
    default: unpack_kernel<64><<<blocks, 256, 0, s>>>(P); break;
    }
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    return KMC_OK;
}

kmc_status launch_init(kmc_ctx *c, int init, cudaStream_t s)
{
    LayoutParams P = layout_params(c);
    const uint64_t total = c->blk_off[c->n_rep];
    const int blocks = (int)std::min<uint64_t>((total + 255) / 256, 65535);
    init_spins_kernel<<<std::max(blocks, 1), 256, 0, s>>>(P, init);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    return KMC_OK;
}

kmc_status launch_reset_counters(kmc_ctx *c, cudaStream_t s)
{
    reset_counters_kernel<<<grid_for(c->n_dom, 256), 256, 0, s>>>(c->d_dctr, c->n_dom);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    return KMC_OK;
}

kmc_status check_device_error(kmc_ctx *c)
{
    int e = 0;
    CUDA_TRY(c, cudaMemcpy(&e, c->d_err, sizeof e, cudaMemcpyDeviceToHost));
    if (e == 0) return KMC_OK;
    int zero = 0;
    CUDA_TRY(c, cudaMemcpy(c->d_err, &zero, sizeof zero, cudaMemcpyHostToDevice));
    if (e == ERR_TIMEOUT) return fail(c, KMC_ETIMEOUT, "a bounded wait for a neighbour's visit gave up");
    if (e == ERR_SPIN) return fail(c, KMC_EDEVICE, "spin buffer holds a byte that is not +1 or -1");
    return fail(c, KMC_EDEVICE, "device error word %d", e);
}

kmc_status sync_ctx(kmc_ctx *c)
{
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

void free_all(kmc_ctx *c)
{
    void **ptrs[] = {(void **)&c->d_L, (void **)&c->d_Dx, (void **)&c->d_k, (void **)&c->d_init, (void **)&c->d_dom_off, (void **)&c->d_dom_rep,
                     (void **)&c->d_site_off, (void **)&c->d_blk_off, (void **)&c->d_seed, (void **)&c->d_A,
                     (void **)&c->d_gfix, (void **)&c->d_grad, (void **)&c->d_h, (void **)&c->d_tiles,
                     (void **)&c->d_edges, (void **)&c->d_dctr, (void **)&c->d_err,
                     (void **)&c->d_obs_acc, (void **)&c->d_tmp, (void **)&c->d_plan, (void **)&c->d_htab,
                     (void **)&c->d_polls, (void **)&c->d_obs_dom};
    for (void **p : ptrs) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    c->obs_acc_words = 0;
    c->plan_words = 0;
}

} // namespace

namespace {

const int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

void noalloc_message(char *err, int32_t err_len, const std::string &msg)
{
    if (err && err_len > 0) {
        std::strncpy(err, msg.c_str(), (size_t)err_len - 1);
        err[err_len - 1] = '\0';
    }
}

// Carves aligned sub-arrays out of the static scratch array.
struct Carver {
    unsigned char *base;
    size_t off = 0;
    template <typename T> T *take(size_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += n * sizeof(T);
        return p;
    }
};

} // namespace

// Score of the exponential clock variates with respect to the rate
// prefactor nu (Sec. 2.1: a domain's waiting time per uniformised step is
// Exp(Lambda_d), Lambda_d = n_d nu, with log density ln Lambda_d - Lambda_d tau,
// so d/dnu = 1/nu - n_d tau): per domain (steps_d - Lambda_d t_d) / nu with
// Lambda_d t_d = -ln(product of its variates); one thread per replica sums
// its domains in order.
__global__ void score_nu_kernel(const uint64_t *dctr, const uint32_t *rep_dom_off, int n_rep, double nu,
                                double *score)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rep) return;
    double s = 0.0;
    for (uint32_t g = rep_dom_off[r]; g < rep_dom_off[r + 1]; ++g) {
        const uint64_t *ctr = dctr + (uint64_t)g * DCTR_WORDS;
        // Lambda_d t_d = -ln(M 2^-63) - E ln 2
        const double lam_t = domain_time(true, ctr[DCTR_CLKM], (int64_t)ctr[DCTR_CLKE], 0, 1.0);
        s += (double)(int64_t)ctr[DCTR_STEPS] - lam_t;
    }
    score[r] = s / nu;
}

extern "C" {

int32_t kmc_version(void) { return 10100; }

const char *kmc_last_error(const kmc_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t kmc_kernel_launches(const kmc_ctx *ctx) { return ctx ? ctx->launches : 0; }

int32_t kmc_domain_side(const kmc_ctx *ctx) { return ctx ? ctx->LD : 0; }

kmc_status kmc_create_lattice(kmc_ctx **out, int32_t n_replicas, const int32_t *L, int32_t L_d,
                              int32_t k_steps, int32_t init, const uint64_t *seeds, int8_t *spins_dev,
                              void *stream)
{
    if (!out) return KMC_EINVAL;
    *out = nullptr;
    kmc_ctx *c = new (std::nothrow) kmc_ctx();
    if (!c) return KMC_ENOMEM;
    auto bail = [&](kmc_status s) {
        free_all(c);
        // keep the context so that kmc_last_error works; the caller destroys it
        *out = c;
        return s;
    };
    if (n_replicas < 1 || !L || !seeds || !spins_dev)
        return bail(fail(c, KMC_EINVAL, "n_replicas >= 1 and non-null L, seeds, spins_dev required"));
    if (L_d == 0) {
        // automatic domain side: the largest of 64, 32, 16, 8 that divides every
        // lattice into an even number of domains per side and still gives each
        // colour phase 20 visits per SM (one per warp of two 10-warp CTAs);
        // the smallest valid side if none does.  The measured choice over
        // sides, steps per visit and plans is the autotuner's (autotune.py).
        int sms = 0, dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(c, KMC_ECUDA, "device attributes for the automatic domain side"));
        }
        int smallest = 0;
        for (int cand = 64; cand >= 8; cand /= 2) {
            bool ok = true;
            uint64_t doms = 0;
            for (int r = 0; r < n_replicas && ok; ++r) {
                ok = L[r] >= 2 * cand && L[r] % (2 * cand) == 0;
                doms += ok ? (uint64_t)(L[r] / cand) * (uint64_t)(L[r] / cand) : 0;
            }
            if (!ok) continue;
            smallest = cand;
            if (L_d == 0 && doms / 4 >= (uint64_t)sms * 20) L_d = cand;
        }
        if (L_d == 0) L_d = smallest;
        if (L_d == 0) return bail(fail(c, KMC_EINVAL, "no domain side of 8, 16, 32 or 64 fits every lattice"));
    }
    if (ld_index(L_d) < 0) return bail(fail(c, KMC_EINVAL, "L_d must be 8, 16, 32 or 64, or 0 (got %d)", L_d));
    if (k_steps < 1 || k_steps > 65535) return bail(fail(c, KMC_EINVAL, "k_steps must be in 1..65535"));
    if (init < KMC_INIT_RANDOM || init > KMC_INIT_KEEP) return bail(fail(c, KMC_EINVAL, "bad init mode"));
    if (((uintptr_t)spins_dev) % 8 != 0) return bail(fail(c, KMC_EINVAL, "spins_dev must be 8-byte aligned"));
    c->n_rep = n_replicas;
    c->LD = L_d;
    c->log2nd = 2 * (L_d == 8 ? 3 : L_d == 16 ? 4 : L_d == 32 ? 5 : 6);
    c->k = k_steps;
    c->spins = spins_dev;
    c->stream = (cudaStream_t)stream;
    c->L.assign(L, L + n_replicas);
    c->kr.assign(n_replicas, k_steps);
    c->init_r.assign(n_replicas, init);
    c->seed.assign(seeds, seeds + n_replicas);
    c->Dx.resize(n_replicas);
    c->dom_off.assign(n_replicas + 1, 0);
    c->site_off.assign(n_replicas, 0);
    c->blk_off.assign(n_replicas + 1, 0);
    uint64_t site = 0, ndom = 0, blk = 0;
    for (int r = 0; r < n_replicas; ++r) {
        const int Lr = L[r];
        if (Lr < 2 * L_d || Lr % (2 * L_d) != 0 || Lr > 65536)
            return bail(fail(c, KMC_EINVAL, "replica %d: L = %d must be a positive multiple of 2*L_d = %d", r, Lr, 2 * L_d));
        c->Dx[r] = Lr / L_d;
        c->site_off[r] = site;
        c->dom_off[r] = (uint32_t)ndom;
        c->blk_off[r] = blk;
        site += (uint64_t)Lr * Lr;
        ndom += (uint64_t)c->Dx[r] * c->Dx[r];
        blk += (uint64_t)Lr * Lr / 128;
    }
    if (ndom >= (1ull << 24)) return bail(fail(c, KMC_EINVAL, "too many domains (%llu)", (unsigned long long)ndom));
    c->dom_off[n_replicas] = (uint32_t)ndom;
    c->blk_off[n_replicas] = blk;
    c->n_dom = (int)ndom;
    c->dom_rep.resize(ndom);
    for (int r = 0; r < n_replicas; ++r)
        for (uint32_t g = c->dom_off[r]; g < c->dom_off[r + 1]; ++g) c->dom_rep[g] = (uint32_t)r;

    cudaError_t ce = cudaGetDevice(&c->dev);
    if (ce != cudaSuccess) return bail(fail(c, KMC_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(ce)));
    ce = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev);
    if (ce != cudaSuccess) return bail(fail(c, KMC_ECUDA, "device attributes: %s", cudaGetErrorString(ce)));
    c->smem_optin -= 1024; // static shared memory of the run kernel and slack

    kmc_status s;
    const size_t tile = (size_t)L_d * L_d / 8;
#define ALLOC(p, n) if ((s = dev_alloc(c, &(p), (n))) != KMC_OK) return bail(s)
    ALLOC(c->d_L, n_replicas);
    ALLOC(c->d_Dx, n_replicas);
    ALLOC(c->d_k, n_replicas);
    ALLOC(c->d_init, n_replicas);
    ALLOC(c->d_dom_off, n_replicas + 1);
    ALLOC(c->d_dom_rep, ndom);
    ALLOC(c->d_site_off, n_replicas);
    ALLOC(c->d_blk_off, n_replicas + 1);
    ALLOC(c->d_seed, n_replicas);
    ALLOC(c->d_A, (size_t)n_replicas * 16);
    ALLOC(c->d_gfix, (size_t)n_replicas * GFIX_WORDS);
    ALLOC(c->d_grad, (size_t)n_replicas * 32);
    ALLOC(c->d_h, n_replicas);
    ALLOC(c->d_tiles, ndom * tile);
    ALLOC(c->d_edges, ndom * EDGE_WORDS);
    ALLOC(c->d_dctr, ndom * DCTR_WORDS);
    ALLOC(c->d_err, 1);
    {
        uint8_t *tmp = nullptr;
        ALLOC(tmp, ndom * 32 + (size_t)n_replicas * 64);
        c->d_tmp = tmp;
    }
#undef ALLOC
    struct Up { void *dst; const void *src; size_t bytes; } ups[] = {
        {c->d_L, c->L.data(), (size_t)n_replicas * 4},
        {c->d_Dx, c->Dx.data(), (size_t)n_replicas * 4},
        {c->d_k, c->kr.data(), (size_t)n_replicas * 4},
        {c->d_init, c->init_r.data(), (size_t)n_replicas * 4},
        {c->d_dom_off, c->dom_off.data(), (size_t)(n_replicas + 1) * 4},
        {c->d_dom_rep, c->dom_rep.data(), (size_t)ndom * 4},
        {c->d_site_off, c->site_off.data(), (size_t)n_replicas * 8},
        {c->d_blk_off, c->blk_off.data(), (size_t)(n_replicas + 1) * 8},
        {c->d_seed, c->seed.data(), (size_t)n_replicas * 8},
    };
    for (const Up &u : ups) {
        ce = cudaMemcpy(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) return bail(fail(c, KMC_ECUDA, "upload: %s", cudaGetErrorString(ce)));
    }
    ce = cudaMemset(c->d_err, 0, sizeof(int));
    if (ce != cudaSuccess) return bail(fail(c, KMC_ECUDA, "memset: %s", cudaGetErrorString(ce)));

    // default rates: Metropolis, beta = 0.4, J = 1, h = 0, nu = 1
    std::vector<double> b0(n_replicas, 0.4), h0(n_replicas, 0.0);
    *out = c;
    if ((s = kmc_set_rates(c, 1.0, b0.data(), h0.data(), 1.0, KMC_RATE_METROPOLIS)) != KMC_OK) return bail(s);
    if ((s = default_plan(c)) != KMC_OK) return bail(s);
    if ((s = kmc_reset(c, init, stream)) != KMC_OK) return bail(s);
    return KMC_OK;
}

kmc_status kmc_reset(kmc_ctx *c, int32_t init, void *stream)
{
    if (!c) return KMC_EINVAL;
    if (init < KMC_INIT_RANDOM || init > KMC_INIT_PER_REPLICA) return fail(c, KMC_EINVAL, "bad init mode");
    c->stream = (cudaStream_t)stream;
    kmc_status s;
    bool any = init != KMC_INIT_KEEP;
    if (init == KMC_INIT_PER_REPLICA) {
        any = false;
        for (int32_t m : c->init_r) any = any || m != KMC_INIT_KEEP;
    }
    if (any && (s = launch_init(c, init, c->stream)) != KMC_OK) return s;
    if ((s = launch_reset_counters(c, c->stream)) != KMC_OK) return s;
    c->sched_done = 0;
    c->visits_done = 0;
    c->clocks_exponential = true;
    return KMC_OK;
}

kmc_status kmc_set_rates(kmc_ctx *c, double J, const double *beta, const double *h, double nu, int32_t rate_law)
{
    if (!c) return KMC_EINVAL;
    if (refuse_capture(c, "kmc_set_rates") != KMC_OK) return KMC_EINVAL;
    if (!beta || !h) return fail(c, KMC_EINVAL, "beta and h arrays required");
    if (rate_law != KMC_RATE_METROPOLIS && rate_law != KMC_RATE_BARKER) return fail(c, KMC_EINVAL, "bad rate law");
    if (!std::isfinite(J) || !(nu > 0.0) || !std::isfinite(nu)) return fail(c, KMC_EINVAL, "J finite and nu > 0 required");
    for (int r = 0; r < c->n_rep; ++r)
        if (!(beta[r] >= 0.0) || !std::isfinite(beta[r]) || !std::isfinite(h[r]))
            return fail(c, KMC_EINVAL, "replica %d: beta >= 0 and finite h required", r);
    const size_t n = (size_t)c->n_rep * 10;
    std::vector<double> a(n), gb(n), gh(n);
    std::vector<uint64_t> A(n);
    for (int r = 0; r < c->n_rep; ++r) {
        build_table(J, beta[r], h[r], rate_law, c->log2nd, &a[r * 10], &A[r * 10], &gb[r * 10], &gh[r * 10]);
        const int z = zero_rate_class(&A[r * 10], 10);
        if (z >= 0)
            return fail(c, KMC_ENOTBALANCED,
                        "replica %d class %d: a_c = %.3g rounds to 0 at 2^-%d; the quantised chain would have a "
                        "one-way rate (Eq. 4)", r, z, a[r * 10 + z], 63 - c->log2nd);
    }
    c->J = J;
    c->nu = nu;
    c->law = rate_law;
    c->beta.assign(beta, beta + c->n_rep);
    c->h.assign(h, h + c->n_rep);
    c->a = a;
    c->A = A;
    c->gb = gb;
    c->gh = gh;
    return upload_rates(c);
}

kmc_status kmc_set_rate_table(kmc_ctx *c, double J, const double *beta, const double *h, double nu, const double *a)
{
    if (!c) return KMC_EINVAL;
    if (refuse_capture(c, "kmc_set_rate_table") != KMC_OK) return KMC_EINVAL;
    if (!beta || !h || !a) return fail(c, KMC_EINVAL, "beta, h and a arrays required");
    if (!std::isfinite(J) || !(nu > 0.0)) return fail(c, KMC_EINVAL, "J finite and nu > 0 required");
    const int P = 63 - c->log2nd;
    const size_t n = (size_t)c->n_rep * 10;
    std::vector<double> av(a, a + n), gb(n, 0.0), gh(n, 0.0);
    std::vector<uint64_t> A(n);
    for (int r = 0; r < c->n_rep; ++r) {
        if (!(beta[r] >= 0.0) || !std::isfinite(h[r])) return fail(c, KMC_EINVAL, "replica %d: bad beta/h", r);
        for (int q = 0; q < 10; ++q) {
            const double ac = a[r * 10 + q];
            if (!(ac > 0.0 && ac <= 1.0)) return fail(c, KMC_EINVAL, "replica %d class %d: a must be in (0, 1]", r, q);
            const int up = q / 5, qq = q % 5;
            const double sigma = up ? 1.0 : -1.0;
            const double dE = 2.0 * sigma * (J * (double)(2 * qq - 4) + h[r]);
            const int qbar = 5 * (1 - up) + qq;
            const double ratio = ac / a[r * 10 + qbar];
            const double want = std::exp(-beta[r] * dE);
            if (std::fabs(ratio - want) > 1e-12 * want)
                return fail(c, KMC_ENOTBALANCED,
                            "replica %d class %d: a_c/a_cbar = %.17g but exp(-beta dE) = %.17g (detailed balance, Eq. 4)",
                            r, q, ratio, want);
            A[r * 10 + q] = (uint64_t)std::nearbyint(std::ldexp(ac, P));
            if (A[r * 10 + q] == 0)
                return fail(c, KMC_ENOTBALANCED,
                            "replica %d class %d: a_c = %.3g rounds to 0 at 2^-%d; the quantised chain would have a "
                            "one-way rate (Eq. 4)", r, q, ac, P);
        }
    }
    c->J = J;
    c->nu = nu;
    c->beta.assign(beta, beta + c->n_rep);
    c->h.assign(h, h + c->n_rep);
    c->a = av;
    c->A = A;
    c->gb = gb; // no closed-form derivatives for a user table
    c->gh = gh;
    return upload_rates(c);
}

kmc_status kmc_rate_table_error(const kmc_ctx *c, double *max_rel_err)
{
    if (!c || !max_rel_err) return KMC_EINVAL;
    if (c->a.empty()) return KMC_EINVAL; // no table yet
    const int P = 63 - c->log2nd;
    double worst = 0.0;
    for (size_t i = 0; i < c->a.size(); ++i) {
        const double q = std::ldexp((double)c->A[i], -P); // exact: A_c < 2^53 or a multiple of its ulp
        worst = std::max(worst, std::fabs(q - c->a[i]) / c->a[i]);
    }
    *max_rel_err = worst;
    return KMC_OK;
}

kmc_status kmc_get_rate_table(const kmc_ctx *c, int32_t replica, double *a, uint64_t *A)
{
    if (!c || replica < 0 || replica >= c->n_rep) return KMC_EINVAL;
    for (int q = 0; q < 10; ++q) {
        if (a) a[q] = c->a[(size_t)replica * 10 + q];
        if (A) A[q] = c->A[(size_t)replica * 10 + q];
    }
    return KMC_OK;
}

kmc_status kmc_set_launch(kmc_ctx *c, int32_t mode, int32_t size, int32_t warps_per_cta)
{
    if (!c) return KMC_EINVAL;
    if (refuse_capture(c, "kmc_set_launch") != KMC_OK) return KMC_EINVAL;
    if (mode == KMC_LAUNCH_AUTO) {
        const kmc_status s = default_plan(c);
        if (s == KMC_OK) c->req_mode = KMC_LAUNCH_AUTO;
        return s;
    }
    if (warps_per_cta < 1 || warps_per_cta > MAX_WPB) return fail(c, KMC_EINVAL, "warps_per_cta must be 1..%d", MAX_WPB);
    Plan pl;
    kmc_status s;
    if (mode == KMC_LAUNCH_CLUSTER) {
        if (size != 1 && size != 2 && size != 4 && size != 8 && size != 16)
            return fail(c, KMC_EINVAL, "cluster size must be 1, 2, 4, 8 or 16");
        int need = 1;
        for (int r = 0; r < c->n_rep; ++r)
            need = std::max(need, (c->Dx[r] * c->Dx[r] / 4 + warps_per_cta * size - 1) / (warps_per_cta * size));
        if ((s = plan_cluster(c, size, warps_per_cta, need, pl)) != KMC_OK) return s;
    } else if (mode == KMC_LAUNCH_GRID) {
        if (size < 1) return fail(c, KMC_EINVAL, "grid needs >= 1 CTA");
        if ((s = plan_grid(c, size, warps_per_cta, pl)) != KMC_OK) return s;
    } else if (mode == KMC_LAUNCH_THREADS) {
        if (warps_per_cta > 4) return fail(c, KMC_EINVAL, "thread plans take 1..4 warps per CTA");
        if (c->LD == 16 || c->LD == 32 || c->LD == 64) {
            // one domain per thread: the grid follows from the domains; size
            // 0 or 1: the replicas one after another, 2: round-robin
            if (size < 0 || size > 2) return fail(c, KMC_EINVAL, "thread plans of L_d = %d take size 0, 1 or 2", c->LD);
            if ((s = plan_thread_rows(c, warps_per_cta, pl, size == 2)) != KMC_OK) return s;
        } else if ((s = plan_threads(c, size > 0 ? size : balanced_thread_ctas(c, warps_per_cta), warps_per_cta, pl)) !=
                   KMC_OK) {
            // size 0: the balanced grid of the library's choice
            return s;
        }
    } else {
        return fail(c, KMC_EINVAL, "bad launch mode %d", mode);
    }
    if ((s = install_plan(c, pl)) != KMC_OK) return s;
    c->req_mode = mode;
    c->req_size = size;
    c->req_wpb = warps_per_cta;
    return KMC_OK;
}

kmc_status kmc_set_horizon(kmc_ctx *c, double dtau)
{
    if (!c) return KMC_EINVAL;
    if (refuse_capture(c, "kmc_set_horizon") != KMC_OK) return KMC_EINVAL;
    if (!(dtau >= 0.0) || !std::isfinite(dtau)) return fail(c, KMC_EINVAL, "dtau must be finite and >= 0");
    const double old = c->dtau;
    c->dtau = dtau;
    kmc_status st = upload_horizon(c);
    if (st != KMC_OK) c->dtau = old;
    return st;
}

kmc_status kmc_set_observation(kmc_ctx *c, int32_t unit)
{
    if (!c) return KMC_EINVAL;
    if (unit != KMC_OBS_SCHEDULE && unit != KMC_OBS_PASS) return fail(c, KMC_EINVAL, "bad observation unit %d", unit);
    c->obs_unit = unit;
    return KMC_OK;
}

kmc_status kmc_set_replica_params(kmc_ctx *c, const int32_t *k_steps, const int32_t *init)
{
    if (!c) return KMC_EINVAL;
    kmc_status s;
    if ((s = refuse_capture(c, "kmc_set_replica_params")) != KMC_OK) return s;
    if (k_steps) {
        if (c->sched_done != 0) return fail(c, KMC_EINVAL, "per-replica k can only change before the first run after a reset");
        for (int r = 0; r < c->n_rep; ++r)
            if (k_steps[r] < 1 || k_steps[r] > 65535) return fail(c, KMC_EINVAL, "replica %d: k_steps must be in 1..65535", r);
    }
    if (init)
        for (int r = 0; r < c->n_rep; ++r)
            if (init[r] < KMC_INIT_RANDOM || init[r] > KMC_INIT_KEEP) return fail(c, KMC_EINVAL, "replica %d: bad init mode", r);
    if (init) {
        c->init_r.assign(init, init + c->n_rep);
        CUDA_TRY(c, cudaMemcpyAsync(c->d_init, c->init_r.data(), (size_t)c->n_rep * 4, cudaMemcpyHostToDevice, c->stream));
    }
    if (k_steps) {
        const std::vector<int32_t> old = c->kr;
        c->kr.assign(k_steps, k_steps + c->n_rep);
        CUDA_TRY(c, cudaMemcpyAsync(c->d_k, c->kr.data(), (size_t)c->n_rep * 4, cudaMemcpyHostToDevice, c->stream));
        // cost-aware plans depend on k: rebuild the requested plan
        if ((s = kmc_set_launch(c, c->req_mode, c->req_size, c->req_wpb)) != KMC_OK) {
            c->kr = old;
            const std::string why = c->err;
            CUDA_TRY(c, cudaMemcpyAsync(c->d_k, c->kr.data(), (size_t)c->n_rep * 4, cudaMemcpyHostToDevice, c->stream));
            return fail(c, s, "%s", why.c_str());
        }
    }
    // pageable sources: consumed when the copies return
    return KMC_OK;
}

kmc_status kmc_get_launch(const kmc_ctx *c, int32_t *mode, int32_t *size, int32_t *ctas, int32_t *warps_per_cta,
                          int32_t *smem_bytes)
{
    if (!c) return KMC_EINVAL;
    if (mode) *mode = c->plan.mode;
    if (size) *size = c->plan.mode == KMC_LAUNCH_CLUSTER ? c->plan.cluster : c->plan.n_cta;
    if (ctas) *ctas = c->plan.n_cta;
    if (warps_per_cta) *warps_per_cta = c->plan.wpb;
    if (smem_bytes) *smem_bytes = (int32_t)c->plan.smem;
    return KMC_OK;
}

kmc_status kmc_debug_barrier(kmc_ctx *c, int32_t extra, int64_t limit_ns)
{
    if (!c || extra < 0 || limit_ns < 0) return KMC_EINVAL;
    c->debug_extra = extra;
    c->bar_limit_ns = limit_ns > 0 ? (uint64_t)limit_ns : DEFAULT_BAR_LIMIT_NS;
    return KMC_OK;
}

kmc_status kmc_enable_grad(kmc_ctx *c, int32_t enable)
{
    if (!c) return KMC_EINVAL;
    const bool was = c->grad;
    c->grad = enable != 0;
    if (c->grad && !was) {
        if (refuse_capture(c, "kmc_enable_grad") != KMC_OK) {
            c->grad = was;
            return KMC_EINVAL;
        }
        // the score kernels may not fit the current plan's shape: re-plan
        Plan pl = c->plan;
        if (check_plan(c, pl) != KMC_OK &&
            kmc_set_launch(c, c->req_mode, c->req_size, c->req_wpb) != KMC_OK && default_plan(c) != KMC_OK) {
            const std::string why = c->err;
            c->grad = was;
            return fail(c, KMC_EINVAL, "no launch plan fits the score kernels: %s", why.c_str());
        }
    }
    return KMC_OK;
}

kmc_status kmc_run_schedule(kmc_ctx *c, int64_t n_schedules, int32_t schedule, int32_t time_mode,
                            int32_t obs_every, double *obs_dev, void *stream)
{
    if (!c) return KMC_EINVAL;
    if (n_schedules < 0) return fail(c, KMC_EINVAL, "n_schedules must be >= 0");
    if (schedule < KMC_SCHEDULE_PALINDROME || schedule > KMC_SCHEDULE_RANDOM_PERM)
        return fail(c, KMC_EINVAL, "bad schedule kind");
    if (time_mode != KMC_TIME_EXPONENTIAL && time_mode != KMC_TIME_EXPECTED && time_mode != KMC_TIME_HORIZON)
        return fail(c, KMC_EINVAL, "bad time mode");
    if (time_mode == KMC_TIME_HORIZON && !(c->dtau > 0.0))
        return fail(c, KMC_EINVAL, "KMC_TIME_HORIZON needs a visit time (kmc_set_horizon)");
    if (obs_every < 0) return fail(c, KMC_EINVAL, "obs_every must be >= 0");
    if (c->sched_done + n_schedules >= (1ll << 52)) return fail(c, KMC_EINVAL, "schedule index overflow");
    c->stream = (cudaStream_t)stream;
    if (n_schedules == 0) return KMC_OK;
    NvtxRange range("kmc_run_schedule %d replicas L_d=%d %lld schedules%s", c->n_rep, c->LD,
                    (long long)n_schedules, c->grad ? " scores" : "");
    cudaStream_t s = c->stream;
    kmc_status st;
    const bool want_obs = obs_every > 0 && obs_dev != nullptr;
    const bool pass_obs = c->obs_unit == KMC_OBS_PASS;
    const int64_t units = pass_obs ? n_schedules * (schedule == KMC_SCHEDULE_PALINDROME ? 8 : 4) : n_schedules;
    const int64_t n_obs = want_obs ? units / obs_every : 0;
    const bool cap = capturing(c);
    if (c->plan.mode == KMC_LAUNCH_THREADS && ((c->grad && (c->LD == 8 || c->LD == 64)) ||
                                               time_mode == KMC_TIME_HORIZON || schedule == KMC_SCHEDULE_RANDOM_PERM)) {
        // the thread kernels cover fixed-length visits of the palindromic
        // and fixed schedules (with scores at L_d = 16, 32): this run takes a warp plan
        // (installed once the stream has drained: earlier launches read the
        // plan buffer)
        if (cap) return fail(c, KMC_EINVAL, "this run needs a warp launch plan; set one before capturing");
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if ((st = default_warp_plan(c)) != KMC_OK) return st;
    }
    if (want_obs && n_obs > 0) {
        const size_t words = (size_t)n_obs * c->n_rep * OBS_WORDS;
        if (words > c->obs_acc_words && cap)
            return fail(c, KMC_EINVAL, "observation buffer must be sized by an uncaptured run of at least as many records");
        if (words > c->obs_acc_words) {
            if (c->d_obs_acc) cudaFree(c->d_obs_acc);
            c->d_obs_acc = nullptr;
            c->obs_acc_words = 0;
            if ((st = dev_alloc(c, &c->d_obs_acc, words)) != KMC_OK) return st;
            c->obs_acc_words = words;
        }
        CUDA_TRY(c, cudaMemsetAsync(c->d_obs_acc, 0, words * 8, s));
    }
    if ((st = launch_pack(c, s)) != KMC_OK) return st;
    // records are built from the state before the launch plus per-visit changes
    unsigned long long *base = reinterpret_cast<unsigned long long *>(c->d_tmp);
    if (n_obs > 0 && (st = launch_observe(c, s, time_mode, base)) != KMC_OK) return st;
    RunParams P = run_params(c);
    P.schedule = schedule;
    P.obs_every = want_obs ? obs_every : 0;
    P.obs_acc = (want_obs && n_obs > 0) ? c->d_obs_acc : nullptr;
    P.obs_pass = (pass_obs && n_obs > 0) ? 1 : 0;
    P.n_obs = n_obs;
    if (time_mode == KMC_TIME_HORIZON) {
        P.horizon = 1;
        P.hkmax = c->hkmax;
        P.htab = c->d_htab;
        P.dtau = c->dtau;
    }
    P.sched_begin = c->sched_done;
    P.n_sched = n_schedules;
    P.visits_before = c->visits_done;
    const Plan &pl = c->plan;
    const bool cluster = pl.mode == KMC_LAUNCH_CLUSTER;
    const bool threads = pl.mode == KMC_LAUNCH_THREADS;
    RunKernel kern = threads ? tpd_kernel_for(c->LD, time_mode == KMC_TIME_EXPONENTIAL, c->grad)
                             : run_kernel_for(c->LD, time_mode == KMC_TIME_EXPONENTIAL, c->grad, cluster);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const bool prof = c->prof && !cap;
    if (prof) P.polls = c->d_polls;
    if (prof) {
        CUDA_TRY(c, cudaEventCreate(&ev0));
        CUDA_TRY(c, cudaEventCreate(&ev1));
        CUDA_TRY(c, cudaEventRecord(ev0, s));
    }
    if (cluster) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(pl.n_cta);
        cfg.blockDim = dim3(pl.wpb * 32);
        cfg.dynamicSmemBytes = pl.smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = pl.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CUDA_TRY(c, cudaLaunchKernelEx(&cfg, kern, P));
    } else {
        void *args[] = {(void *)&P};
        CUDA_TRY(c, cudaLaunchCooperativeKernel((const void *)kern, dim3(pl.n_cta), dim3(pl.wpb * 32), args, pl.smem, s));
    }
    ++c->launches;
    if (prof) {
        CUDA_TRY(c, cudaEventRecord(ev1, s));
        c->prof_events.emplace_back(ev0, ev1);
    }
    if (want_obs && n_obs > 0) {
        finalize_obs_kernel<<<grid_for(c->n_rep, 128), 128, 0, s>>>(base, c->d_obs_acc, n_obs, c->n_rep, c->d_L, c->d_Dx,
                                                                    c->J, c->d_h, obs_dev, c->grad ? 6 : 4);
        ++c->launches;
        CUDA_TRY(c, cudaGetLastError());
    }
    if ((st = launch_unpack(c, s)) != KMC_OK) return st;
    c->sched_done += n_schedules;
    c->visits_done += n_schedules * (schedule == KMC_SCHEDULE_PALINDROME ? 2 : 1);
    c->last_time_mode = time_mode;
    if (time_mode != KMC_TIME_EXPONENTIAL) c->clocks_exponential = false;
    return KMC_OK;
}

kmc_status kmc_sync(kmc_ctx *c)
{
    if (!c) return KMC_EINVAL;
    return sync_ctx(c);
}

kmc_status kmc_observables(kmc_ctx *c, double *E_per_site, double *m, double *t, int64_t *steps, int64_t *flips)
{
    if (!c) return KMC_EINVAL;
    if (refuse_capture(c, "kmc_observables") != KMC_OK) return KMC_EINVAL;
    kmc_status st;
    cudaStream_t s = c->stream;
    if ((st = launch_pack(c, s)) != KMC_OK) return st;
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(c->d_tmp);
    const size_t words = (size_t)c->n_rep * OBS_WORDS;
    if ((st = launch_observe(c, s, c->last_time_mode, acc)) != KMC_OK) return st;
    std::vector<unsigned long long> h_acc(words);
    CUDA_TRY(c, cudaMemcpyAsync(h_acc.data(), acc, words * 8, cudaMemcpyDeviceToHost, s));
    if ((st = sync_ctx(c)) != KMC_OK) return st;
    for (int r = 0; r < c->n_rep; ++r) {
        const unsigned long long *a = &h_acc[(size_t)r * OBS_WORDS];
        const double N = (double)c->L[r] * (double)c->L[r];
        const double b = (double)(long long)a[0];
        const double mg = (double)(long long)a[1];
        double tsum;
        std::memcpy(&tsum, &a[2], 8);
        const double e = (-c->J * b - c->h[r] * mg) / N;
        if (E_per_site) E_per_site[r] = e;
        if (m) m[r] = mg / N;
        if (t) t[r] = tsum / ((double)c->Dx[r] * c->Dx[r]);
    }
    if (flips || steps) {
        // per-domain counts, summed per replica (Eq. 11: the step counter)
        std::vector<int64_t> fl(c->n_dom), sp(c->n_dom);
        if ((st = domain_state(c, nullptr, fl.data(), nullptr, sp.data())) != KMC_OK) return st;
        for (int r = 0; r < c->n_rep; ++r) {
            int64_t f = 0, q = 0;
            for (uint32_t g = c->dom_off[r]; g < c->dom_off[r + 1]; ++g) {
                f += fl[g];
                q += sp[g];
            }
            if (flips) flips[r] = f;
            if (steps) steps[r] = q;
        }
    }
    return KMC_OK;
}

kmc_status kmc_domain_state(kmc_ctx *c, uint64_t *hash, int64_t *flips, double *t)
{
    if (!c) return KMC_EINVAL;
    if (refuse_capture(c, "kmc_domain_state") != KMC_OK) return KMC_EINVAL;
    return domain_state(c, hash, flips, t, nullptr);
}

kmc_status kmc_grad_nu(kmc_ctx *c, double *score_dev)
{
    if (!c) return KMC_EINVAL;
    if (refuse_capture(c, "kmc_grad_nu") != KMC_OK) return KMC_EINVAL;
    if (!score_dev) return fail(c, KMC_EINVAL, "score_dev required");
    if (!c->clocks_exponential)
        return fail(c, KMC_EINVAL, "the rate-prefactor score needs exponential clocks in every run since the last reset");
    score_nu_kernel<<<grid_for(c->n_rep, 128), 128, 0, c->stream>>>(c->d_dctr, c->d_dom_off, c->n_rep, c->nu,
                                                                       score_dev);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    return sync_ctx(c);
}

kmc_status kmc_grad(kmc_ctx *c, double *score_dev, int32_t reset)
{
    if (!c) return KMC_EINVAL;
    if (refuse_capture(c, "kmc_grad") != KMC_OK) return KMC_EINVAL;
    if (!score_dev) return fail(c, KMC_EINVAL, "score_dev required");
    score_reduce_kernel<<<grid_for(c->n_rep, 128), 128, 0, c->stream>>>(c->d_dctr, c->d_dom_off, c->n_rep, score_dev,
                                                                          reset, c->d_dctr);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    return sync_ctx(c);
}

kmc_status kmc_run_schedule_noalloc(int32_t L, int32_t L_d, int32_t k_steps, uint64_t seed, double J, double beta,
                                    double h, double nu, int32_t rate_law, int64_t sched_begin, int64_t n_schedules,
                                    int32_t schedule, int32_t time_mode, int32_t obs_every, int8_t *spins_dev,
                                    double *obs_dev, void *stream, char *err, int32_t err_len)
{
    // A host-side context holds the geometry and the launch plan; it owns no
    // device memory: every device pointer below points into g_noalloc_scratch.
    kmc_ctx c;
    auto bad = [&](kmc_status st, const std::string &msg) {
        noalloc_message(err, err_len, msg);
        return st;
    };
    if (ld_index(L_d) < 0) return bad(KMC_EINVAL, "L_d must be 8, 16, 32 or 64");
    if (L < 2 * L_d || L % (2 * L_d) != 0 || L > 65536) return bad(KMC_EINVAL, "L must be a positive multiple of 2*L_d");
    if (k_steps < 1 || k_steps > 65535) return bad(KMC_EINVAL, "k_steps must be in 1..65535");
    if (!spins_dev || ((uintptr_t)spins_dev) % 8 != 0) return bad(KMC_EINVAL, "spins_dev must be non-null and 8-byte aligned");
    if (n_schedules < 0 || sched_begin < 0 || sched_begin + n_schedules >= (1ll << 52))
        return bad(KMC_EINVAL, "bad schedule range");
    if (schedule < KMC_SCHEDULE_PALINDROME || schedule > KMC_SCHEDULE_RANDOM_PERM) return bad(KMC_EINVAL, "bad schedule kind");
    if (time_mode != KMC_TIME_EXPONENTIAL && time_mode != KMC_TIME_EXPECTED) return bad(KMC_EINVAL, "bad time mode");
    if (obs_every < 0) return bad(KMC_EINVAL, "obs_every must be >= 0");
    if (rate_law != KMC_RATE_METROPOLIS && rate_law != KMC_RATE_BARKER) return bad(KMC_EINVAL, "bad rate law");
    if (!(beta >= 0.0) || !std::isfinite(beta) || !std::isfinite(h) || !std::isfinite(J) || !(nu > 0.0))
        return bad(KMC_EINVAL, "beta >= 0, finite J and h, nu > 0 required");

    c.n_rep = 1;
    c.LD = L_d;
    c.log2nd = 2 * (L_d == 8 ? 3 : L_d == 16 ? 4 : L_d == 32 ? 5 : 6);
    c.k = k_steps;
    c.kr.assign(1, k_steps);
    c.init_r.assign(1, KMC_INIT_KEEP);
    c.spins = spins_dev;
    c.stream = (cudaStream_t)stream;
    c.L.assign(1, L);
    c.Dx.assign(1, L / L_d);
    c.seed.assign(1, seed);
    c.dom_off = {0u, (uint32_t)(c.Dx[0] * c.Dx[0])};
    c.site_off = {0ull};
    c.blk_off = {0ull, (uint64_t)L * L / 128};
    c.n_dom = c.Dx[0] * c.Dx[0];
    c.dom_rep.assign(c.n_dom, 0u);
    c.J = J;
    c.nu = nu;
    c.h.assign(1, h);
    c.a.resize(10);
    c.A.resize(10);
    c.gb.resize(10);
    c.gh.resize(10);
    build_table(J, beta, h, rate_law, c.log2nd, c.a.data(), c.A.data(), c.gb.data(), c.gh.data());
    if (zero_rate_class(c.A.data(), 10) >= 0)
        return bad(KMC_ENOTBALANCED, "an acceptance a_c rounds to 0 in fixed point (one-way rate, Eq. 4)");

    cudaError_t ce = cudaGetDevice(&c.dev);
    if (ce != cudaSuccess) return bad(KMC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    if (c.dev < 0 || c.dev >= NOALLOC_MAX_DEVICES) return bad(KMC_EINVAL, "device index out of range");
    ce = cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, c.dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&c.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.dev);
    if (ce != cudaSuccess) return bad(KMC_ECUDA, std::string("device attributes: ") + cudaGetErrorString(ce));
    c.smem_optin -= 1024;

    // the replica must fit one cluster of at most 16 CTAs
    const int per_colour = c.n_dom / 4;
    const int need = (per_colour + MAX_WPB - 1) / MAX_WPB;
    int C = 1;
    while (C < need) C *= 2;
    if (C > 16) return bad(KMC_EINVAL, "lattice too large for the no-alloc path: more than one cluster of 16 CTAs");
    Plan pl;
    kmc_status st = plan_cluster(&c, C, MAX_WPB, 1, pl);
    if (st != KMC_OK) return bad(st, c.err);
    st = check_plan(&c, pl);
    if (st != KMC_OK) return bad(st, c.err);

    // scratch layout (every sub-array 256-byte aligned)
    const int64_t n_obs = (obs_every > 0 && obs_dev) ? n_schedules / obs_every : 0;
    std::vector<uint32_t> flat;
    for (auto *v : {&pl.cta_slot_off, &pl.cta_col_off, &pl.cta_rt_off, &pl.rt_rep, &pl.slot_g, &pl.slot_rt, &pl.slot_nb})
        flat.insert(flat.end(), v->begin(), v->end());
    const size_t tile = (size_t)L_d * L_d / 8;
    // one carving sequence, run twice: to measure (null base) and to place
    auto carve = [&](Carver &cv) {
        c.d_tiles = cv.take<uint8_t>((size_t)c.n_dom * tile);
        c.d_edges = cv.take<uint64_t>((size_t)c.n_dom * EDGE_WORDS);
        c.d_dctr = cv.take<uint64_t>((size_t)c.n_dom * DCTR_WORDS);
        c.d_dom_rep = cv.take<uint32_t>((size_t)c.n_dom);
        c.d_plan = cv.take<uint32_t>(flat.size());
        c.d_obs_acc = cv.take<unsigned long long>((size_t)std::max<int64_t>(n_obs, 1) * OBS_WORDS);
        c.d_L = cv.take<int32_t>(1);
        c.d_Dx = cv.take<int32_t>(1);
        c.d_k = cv.take<int32_t>(1);
        c.d_dom_off = cv.take<uint32_t>(2);
        c.d_site_off = cv.take<uint64_t>(1);
        c.d_blk_off = cv.take<uint64_t>(2);
        c.d_seed = cv.take<uint64_t>(1);
        c.d_A = cv.take<uint64_t>(16);
        c.d_gfix = cv.take<int64_t>(GFIX_WORDS);
        c.d_grad = cv.take<double>(32);
        c.d_h = cv.take<double>(1);
        c.d_err = cv.take<int>(1);
        c.d_tmp = cv.take<unsigned long long>(OBS_WORDS); // observation base of the replica
    };
    Carver measure{nullptr};
    carve(measure);
    const size_t need_bytes = measure.off;
    if (need_bytes > (size_t)KMC_NOALLOC_MAX_BYTES) {
        char msg[160];
        snprintf(msg, sizeof msg, "needs %zu bytes of working memory; the no-alloc path holds %d", need_bytes,
                 KMC_NOALLOC_MAX_BYTES);
        return bad(KMC_EINVAL, msg);
    }

    // device address of the scratch array on this device (resolved once per device)
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[c.dev]) {
            void *p = nullptr;
            ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (ce != cudaSuccess) return bad(KMC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
            g_noalloc_ptr[c.dev] = static_cast<unsigned char *>(p);
        }
        base = g_noalloc_ptr[c.dev];
    }
    Carver cv{base};
    carve(cv);
    c.plan_words = flat.size();

    // inputs of this call; the array keeps the previous call's contents, so
    // everything the kernels read is written (or cleared) here first
    cudaStream_t s = c.stream;
    std::vector<uint64_t> A16(16, 0);
    std::vector<int64_t> gfix(GFIX_WORDS, 0);
    (void)build_gfix(c.a.data(), c.gb.data(), c.gh.data(), c.log2nd, gfix.data()); // staged, unused: no scores here
    std::vector<double> g32(32, 0.0);
    for (int q = 0; q < 10; ++q) {
        A16[q] = c.A[q];
        g32[q] = c.a[q];
        g32[10 + q] = c.gb[q];
        g32[20 + q] = c.gh[q];
    }
    struct Up { void *dst; const void *src; size_t bytes; } ups[] = {
        {c.d_L, c.L.data(), 4}, {c.d_Dx, c.Dx.data(), 4}, {c.d_k, c.kr.data(), 4}, {c.d_dom_off, c.dom_off.data(), 8},
        {c.d_site_off, c.site_off.data(), 8}, {c.d_blk_off, c.blk_off.data(), 16}, {c.d_seed, c.seed.data(), 8},
        {c.d_A, A16.data(), 128}, {c.d_gfix, gfix.data(), GFIX_WORDS * 8}, {c.d_grad, g32.data(), 256}, {c.d_h, c.h.data(), 8},
        {c.d_dom_rep, c.dom_rep.data(), (size_t)c.n_dom * 4}, {c.d_plan, flat.data(), flat.size() * 4},
    };
    for (const Up &u : ups) {
        // pageable host source: the copy has completed when the call returns
        ce = cudaMemcpyAsync(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, s);
        if (ce != cudaSuccess) return bad(KMC_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(ce));
    }
    ce = cudaMemsetAsync(c.d_err, 0, sizeof(int), s);
    if (ce == cudaSuccess && n_obs > 0) ce = cudaMemsetAsync(c.d_obs_acc, 0, (size_t)n_obs * c.n_rep * OBS_WORDS * 8, s);
    if (ce != cudaSuccess) return bad(KMC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(ce));
    c.plan = std::move(pl);

    if ((st = launch_reset_counters(&c, s)) != KMC_OK) return bad(st, c.err);
    if (n_schedules > 0) {
        if ((st = launch_pack(&c, s)) != KMC_OK) return bad(st, c.err);
        if (n_obs > 0 &&
            (st = launch_observe(&c, s, time_mode, reinterpret_cast<unsigned long long *>(c.d_tmp))) != KMC_OK)
            return bad(st, c.err);
        RunParams P = run_params(&c);
        P.schedule = schedule;
        P.obs_every = n_obs > 0 ? obs_every : 0;
        P.obs_acc = n_obs > 0 ? c.d_obs_acc : nullptr;
        P.n_obs = n_obs;
        P.sched_begin = sched_begin;
        P.n_sched = n_schedules;
        P.visits_before = 0;
        RunKernel kern = run_kernel_for(c.LD, time_mode == KMC_TIME_EXPONENTIAL, false, true);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c.plan.n_cta);
        cfg.blockDim = dim3(c.plan.wpb * 32);
        cfg.dynamicSmemBytes = c.plan.smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c.plan.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ce = cudaLaunchKernelEx(&cfg, kern, P);
        if (ce != cudaSuccess) return bad(KMC_ECUDA, std::string("cudaLaunchKernelEx: ") + cudaGetErrorString(ce));
        if (n_obs > 0) {
            finalize_obs_kernel<<<1, 32, 0, s>>>(reinterpret_cast<unsigned long long *>(c.d_tmp), c.d_obs_acc, n_obs, 1,
                                                 c.d_L, c.d_Dx, J, c.d_h, obs_dev, 4);
            ce = cudaGetLastError();
            if (ce != cudaSuccess) return bad(KMC_ECUDA, std::string("finalize: ") + cudaGetErrorString(ce));
        }
        if ((st = launch_unpack(&c, s)) != KMC_OK) return bad(st, c.err);
    }
    // synchronising: the device error word lives in the shared array
    st = sync_ctx(&c);
    // c lives on this stack frame and is never handed to free_all or
    // kmc_destroy (the only places that free device memory), so its device
    // pointers into the static array are simply dropped here
    if (st != KMC_OK) return bad(st, c.err);
    noalloc_message(err, err_len, "");
    return KMC_OK;
}

kmc_status kmc_lr_estimate(kmc_ctx *c, const double *A_dev, double *grad_dev)
{
    if (!c) return KMC_EINVAL;
    if (!A_dev || !grad_dev) return fail(c, KMC_EINVAL, "A_dev and grad_dev required");
    if (c->n_rep < 2) return fail(c, KMC_EINVAL, "the estimate needs at least two replicas");
    // the kernel writes {mean, d/dbeta, d/dh}: the mean goes to scratch
    double *out3 = reinterpret_cast<double *>(c->d_tmp);
    lr_estimate_kernel<<<1, 256, 0, c->stream>>>(A_dev, nullptr, 1, 0, c->d_dctr, c->d_dom_off, c->n_rep, out3);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(grad_dev, out3 + 1, 2 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return KMC_OK;
}

kmc_status kmc_lr_observable(kmc_ctx *c, const double *rec_dev, int32_t stride, int32_t observable, double *out_dev)
{
    if (!c) return KMC_EINVAL;
    if (!rec_dev || !out_dev) return fail(c, KMC_EINVAL, "rec_dev and out_dev required");
    if (observable < 0 || observable > 2) return fail(c, KMC_EINVAL, "observable must be 0 (e), 1 (m) or 2 (e*m)");
    if (stride < 4) return fail(c, KMC_EINVAL, "stride must be at least 4 (a record holds e, m, e*m, T)");
    if (c->n_rep < 2) return fail(c, KMC_EINVAL, "the estimate needs at least two replicas");
    // explicit h-dependence: e = (-J bonds - h M)/N gives de/dh = -m and
    // d(e m)/dh = -m^2; m has none, and none of them depends on beta
    const int xsel = (observable == 0) ? 1 : (observable == 2) ? 2 : 0;
    lr_estimate_kernel<<<1, 256, 0, c->stream>>>(rec_dev + observable, rec_dev + 1, stride, xsel, c->d_dctr,
                                                 c->d_dom_off, c->n_rep, out_dev);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    return KMC_OK;
}

kmc_status kmc_profile(kmc_ctx *c, int32_t enable)
{
    if (!c) return KMC_EINVAL;
    if (enable && !c->d_polls) {
        kmc_status st = dev_alloc(c, &c->d_polls, 1);
        if (st != KMC_OK) return st;
        CUDA_TRY(c, cudaMemset(c->d_polls, 0, sizeof(unsigned long long)));
    }
    c->prof = enable != 0;
    return KMC_OK;
}

kmc_status kmc_profile_polls(kmc_ctx *c, int64_t *polls)
{
    if (!c || !polls) return KMC_EINVAL;
    unsigned long long v = 0;
    if (c->d_polls) {
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        CUDA_TRY(c, cudaMemcpy(&v, c->d_polls, sizeof v, cudaMemcpyDeviceToHost));
        CUDA_TRY(c, cudaMemset(c->d_polls, 0, sizeof v));
    }
    *polls = (int64_t)v;
    return KMC_OK;
}

kmc_status kmc_profile_read(kmc_ctx *c, double *run_kernel_ms, int64_t *run_kernel_launches)
{
    if (!c) return KMC_EINVAL;
    double tot = 0.0;
    int64_t n = 0;
    for (auto &pr : c->prof_events) {
        CUDA_TRY(c, cudaEventSynchronize(pr.second));
        float ms = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&ms, pr.first, pr.second));
        tot += ms;
        ++n;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    c->prof_events.clear();
    if (run_kernel_ms) *run_kernel_ms = tot;
    if (run_kernel_launches) *run_kernel_launches = n;
    return KMC_OK;
}

void kmc_destroy(kmc_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (auto &pr : c->prof_events) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    c->prof_events.clear();
    free_all(c);
    delete c;
}

} // extern "C"

// ---------------------------------------------------------------------------
// The 1D ring (Sec. 3.1): one thread per trajectory, see kmc_ring.cuh.
// ---------------------------------------------------------------------------
struct kmc_ring {
    int n_traj = 0, NS = 0, Ld = 0, k = 0, log2nd = 0;
    cudaStream_t stream = nullptr;
    uint64_t *d_seed = nullptr, *d_A = nullptr, *d_state = nullptr, *d_hash = nullptr, *d_clkM = nullptr;
    int64_t *d_clkE = nullptr, *d_flips = nullptr, *d_steps = nullptr;
    double *d_h = nullptr, *d_t = nullptr;
    double J = 1.0, nu = 1.0;
    int64_t sched_done = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

kmc_status ring_fail(kmc_ring *g, kmc_status s, const char *fmt, ...)
{
    if (g) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        g->err = buf;
    }
    return s;
}

#define RING_CUDA_TRY(g, call)                                                                   \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return ring_fail((g), KMC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

// Ring acceptance table (App. A, Eq. Glauber_TM) for classes c = 3 up + q:
// dE_c = 2 s (J (2q - 2) + h); A_c = round(a_c 2^P), P = 63 - log2(L_d).
void ring_table(double J, double beta, double h, int law, int log2nd, double *a, uint64_t *A)
{
    const int P = 63 - log2nd;
    for (int c = 0; c < kmcring::RING_CLASSES; ++c) {
        const int up = c / 3, q = c % 3;
        const double sigma = up ? 1.0 : -1.0;
        const double dE = 2.0 * sigma * (J * (double)(2 * q - 2) + h);
        double ac;
        if (law == KMC_RATE_METROPOLIS) ac = (dE <= 0.0) ? 1.0 : std::exp(-beta * dE);
        else ac = 1.0 / (1.0 + std::exp(beta * dE));
        a[c] = ac;
        A[c] = (uint64_t)std::nearbyint(std::ldexp(ac, P));
    }
}

void ring_free(kmc_ring *g)
{
    void *ptrs[] = {g->d_seed, g->d_A, g->d_state, g->d_hash, g->d_clkM, g->d_clkE, g->d_flips, g->d_steps,
                    g->d_h, g->d_t};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

template <typename T>
kmc_status ring_alloc(kmc_ring *g, T **p, size_t n)
{
    cudaError_t e = cudaMalloc((void **)p, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ring_fail(g, alloc_status(e), "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
    }
    return KMC_OK;
}

int ring_passes(int schedule, int ND)
{
    if (schedule == KMC_SCHEDULE_RANDOM_PERM) return ND;
    const int ncol = (ND == 1) ? 1 : 2;
    return schedule == KMC_SCHEDULE_PALINDROME ? 2 * ncol : ncol;
}

} // namespace

extern "C" {

kmc_status kmc_ring_set_rates(kmc_ring *g, double J, const double *beta, const double *h, double nu, int32_t rate_law)
{
    if (!g) return KMC_EINVAL;
    if (!beta || !h) return ring_fail(g, KMC_EINVAL, "beta and h arrays required");
    if (rate_law != KMC_RATE_METROPOLIS && rate_law != KMC_RATE_BARKER) return ring_fail(g, KMC_EINVAL, "bad rate law");
    if (!std::isfinite(J) || !(nu > 0.0) || !std::isfinite(nu)) return ring_fail(g, KMC_EINVAL, "J finite and nu > 0 required");
    const int nc = kmcring::RING_CLASSES;
    std::vector<double> a((size_t)g->n_traj * nc);
    std::vector<uint64_t> A((size_t)g->n_traj * nc);
    for (int i = 0; i < g->n_traj; ++i) {
        if (!(beta[i] >= 0.0) || !std::isfinite(beta[i]) || !std::isfinite(h[i]))
            return ring_fail(g, KMC_EINVAL, "trajectory %d: beta >= 0 and finite h required", i);
        ring_table(J, beta[i], h[i], rate_law, g->log2nd, &a[(size_t)i * nc], &A[(size_t)i * nc]);
        const int z = zero_rate_class(&A[(size_t)i * nc], nc);
        if (z >= 0)
            return ring_fail(g, KMC_ENOTBALANCED, "trajectory %d class %d: a_c = %.3g rounds to 0 in fixed point "
                             "(one-way rate, Eq. 4)", i, z, a[(size_t)i * nc + z]);
        for (int c = 0; c < nc; ++c) {
            const int up = c / 3, q = c % 3;
            const double dE = 2.0 * (up ? 1.0 : -1.0) * (J * (double)(2 * q - 2) + h[i]);
            const double ratio = a[(size_t)i * nc + c] / a[(size_t)i * nc + 3 * (1 - up) + q];
            const double want = std::exp(-beta[i] * dE);
            if (std::fabs(ratio - want) > 1e-12 * want)
                return ring_fail(g, KMC_ENOTBALANCED, "trajectory %d class %d: a_c/a_cbar = %.17g, exp(-beta dE) = %.17g",
                                 i, c, ratio, want);
        }
    }
    RING_CUDA_TRY(g, cudaMemcpyAsync(g->d_A, A.data(), A.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, g->stream));
    RING_CUDA_TRY(g, cudaMemcpyAsync(g->d_h, h, (size_t)g->n_traj * sizeof(double), cudaMemcpyHostToDevice, g->stream));
    RING_CUDA_TRY(g, cudaStreamSynchronize(g->stream)); // the host vectors go out of scope
    g->J = J;
    g->nu = nu;
    return KMC_OK;
}

kmc_status kmc_ring_create(kmc_ring **out, int32_t n_traj, int32_t n_sites, int32_t L_d, int32_t k_steps,
                           const uint64_t *seeds, const uint64_t *init, void *stream)
{
    if (!out) return KMC_EINVAL;
    *out = nullptr;
    if (n_traj < 1 || n_sites < 2 || n_sites > 64 || L_d < 1 || L_d > 64 || (L_d & (L_d - 1)) ||
        n_sites % L_d != 0 || k_steps < 0 || k_steps > 65535 || !seeds || !init)
        return KMC_EINVAL;
    const uint64_t NM = (n_sites == 64) ? ~0ull : ((1ull << n_sites) - 1ull);
    for (int i = 0; i < n_traj; ++i)
        if (init[i] & ~NM) return KMC_EINVAL;
    kmc_ring *g = new kmc_ring();
    g->n_traj = n_traj;
    g->NS = n_sites;
    g->Ld = L_d;
    g->k = k_steps;
    while ((1 << g->log2nd) < L_d) ++g->log2nd;
    g->stream = (cudaStream_t)stream;
    const size_t n = (size_t)n_traj;
    kmc_status st = KMC_OK;
    if ((st = ring_alloc(g, &g->d_seed, n)) || (st = ring_alloc(g, &g->d_A, n * kmcring::RING_CLASSES)) ||
        (st = ring_alloc(g, &g->d_state, n)) || (st = ring_alloc(g, &g->d_hash, n)) ||
        (st = ring_alloc(g, &g->d_clkM, n)) || (st = ring_alloc(g, &g->d_clkE, n)) ||
        (st = ring_alloc(g, &g->d_flips, n)) || (st = ring_alloc(g, &g->d_steps, n)) ||
        (st = ring_alloc(g, &g->d_h, n)) || (st = ring_alloc(g, &g->d_t, n))) {
        ring_free(g);
        delete g;
        return st;
    }
    std::vector<uint64_t> basis(n, HASH_BASIS), one(n, 1ull << 63);
    if (cudaMemcpyAsync(g->d_seed, seeds, n * 8, cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
        cudaMemcpyAsync(g->d_state, init, n * 8, cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
        cudaMemcpyAsync(g->d_hash, basis.data(), n * 8, cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
        cudaMemcpyAsync(g->d_clkM, one.data(), n * 8, cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->d_clkE, 0, n * 8, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->d_flips, 0, n * 8, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->d_steps, 0, n * 8, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->d_t, 0, n * 8, g->stream) != cudaSuccess || cudaStreamSynchronize(g->stream) != cudaSuccess) {
        cudaGetLastError();
        ring_free(g);
        delete g;
        return KMC_ECUDA;
    }
    std::vector<double> beta(n, 0.5), h(n, 0.0);
    if ((st = kmc_ring_set_rates(g, 1.0, beta.data(), h.data(), 1.0, KMC_RATE_BARKER)) != KMC_OK) {
        ring_free(g);
        delete g;
        return st;
    }
    *out = g;
    return KMC_OK;
}

kmc_status kmc_ring_run(kmc_ring *g, int64_t n_schedules, int32_t schedule, int32_t time_mode, int32_t obs_every,
                        double *obs_dev, uint64_t *state_dev, int64_t *ens_dev, void *stream)
{
    if (!g) return KMC_EINVAL;
    const int ND = g->NS / g->Ld;
    if (n_schedules < 0) return ring_fail(g, KMC_EINVAL, "n_schedules must be >= 0");
    if (schedule != KMC_SCHEDULE_PALINDROME && schedule != KMC_SCHEDULE_FIXED && schedule != KMC_SCHEDULE_RANDOM_PERM)
        return ring_fail(g, KMC_EINVAL, "bad schedule %d", schedule);
    if (schedule != KMC_SCHEDULE_RANDOM_PERM && ND != 1 && (ND & 1))
        return ring_fail(g, KMC_EINVAL, "colour schedules need N_D = 1 or even (N_D = %d)", ND);
    if (time_mode != KMC_TIME_EXPONENTIAL && time_mode != KMC_TIME_EXPECTED)
        return ring_fail(g, KMC_EINVAL, "the ring supports KMC_TIME_EXPONENTIAL and KMC_TIME_EXPECTED");
    if (obs_every < 0) return ring_fail(g, KMC_EINVAL, "obs_every must be >= 0");
    if ((reinterpret_cast<uintptr_t>(obs_dev) & 31u) != 0)
        return ring_fail(g, KMC_EINVAL, "obs_dev must be 32-byte aligned");
    if ((reinterpret_cast<uintptr_t>(state_dev) & 7u) != 0 || (reinterpret_cast<uintptr_t>(ens_dev) & 7u) != 0)
        return ring_fail(g, KMC_EINVAL, "state_dev and ens_dev must be 8-byte aligned");
    if (g->sched_done > (int64_t)(((1ull << 56) / kmcring::RING_PHASE_SLOTS) - (uint64_t)n_schedules))
        return ring_fail(g, KMC_EINVAL, "schedule count past the Philox phase range");
    const int64_t n_rec = obs_every > 0 ? n_schedules * ring_passes(schedule, ND) / obs_every : 0;
    g->stream = (cudaStream_t)stream;
    if (ens_dev && n_rec > 0)
        RING_CUDA_TRY(g, cudaMemsetAsync(ens_dev, 0, (size_t)n_rec * (kmcring::RING_ENS_FIXED + g->NS) * 8, g->stream));
    if (n_schedules == 0) return KMC_OK;
    NvtxRange range("kmc_ring_run %d trajectories N_S=%d %lld schedules", g->n_traj, g->NS, (long long)n_schedules);
    kmcring::RingParams P;
    P.n_traj = g->n_traj;
    P.NS = g->NS;
    P.Ld = g->Ld;
    P.k = g->k;
    P.schedule = schedule;
    P.obs_every = n_rec > 0 ? obs_every : 0;
    P.sched_begin = g->sched_done;
    P.n_sched = n_schedules;
    P.J = g->J;
    P.nu = g->nu;
    P.seed = g->d_seed;
    P.A = g->d_A;
    P.h = g->d_h;
    P.state = g->d_state;
    P.hash = g->d_hash;
    P.clkM = g->d_clkM;
    P.clkE = g->d_clkE;
    P.flips = g->d_flips;
    P.steps = g->d_steps;
    P.t = g->d_t;
    P.obs = n_rec > 0 ? obs_dev : nullptr;
    P.obs_state = n_rec > 0 ? state_dev : nullptr;
    P.ens = n_rec > 0 ? reinterpret_cast<unsigned long long *>(ens_dev) : nullptr;
    const int blocks = (g->n_traj + kmcring::RING_BLOCK - 1) / kmcring::RING_BLOCK;
    if (time_mode == KMC_TIME_EXPONENTIAL)
        kmcring::ring_kernel<true><<<blocks, kmcring::RING_BLOCK, 0, g->stream>>>(P);
    else
        kmcring::ring_kernel<false><<<blocks, kmcring::RING_BLOCK, 0, g->stream>>>(P);
    RING_CUDA_TRY(g, cudaGetLastError());
    ++g->launches;
    g->sched_done += n_schedules;
    return KMC_OK;
}

kmc_status kmc_ring_state(kmc_ring *g, uint64_t *state, uint64_t *hash, int64_t *flips, int64_t *steps, double *t)
{
    if (!g) return KMC_EINVAL;
    RING_CUDA_TRY(g, cudaStreamSynchronize(g->stream));
    const size_t n = (size_t)g->n_traj * 8;
    if (state) RING_CUDA_TRY(g, cudaMemcpy(state, g->d_state, n, cudaMemcpyDeviceToHost));
    if (hash) RING_CUDA_TRY(g, cudaMemcpy(hash, g->d_hash, n, cudaMemcpyDeviceToHost));
    if (flips) RING_CUDA_TRY(g, cudaMemcpy(flips, g->d_flips, n, cudaMemcpyDeviceToHost));
    if (steps) RING_CUDA_TRY(g, cudaMemcpy(steps, g->d_steps, n, cudaMemcpyDeviceToHost));
    if (t) RING_CUDA_TRY(g, cudaMemcpy(t, g->d_t, n, cudaMemcpyDeviceToHost));
    return KMC_OK;
}

const char *kmc_ring_last_error(const kmc_ring *g) { return g ? g->err.c_str() : "null ring"; }

void kmc_ring_destroy(kmc_ring *g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    ring_free(g);
    delete g;
}

} // extern "C"

// ---------------------------------------------------------------------------
// Small lattices under block or stripe partitions (Sec. 3.2): one warp per
// trajectory, see kmc_part.cuh.
// ---------------------------------------------------------------------------
struct kmc_part {
    int n_traj = 0, L = 0, kind = 0, ND = 0, k = 0, Dx = 0, W = 0, H = 0, ncol = 1, P = 0;
    uint64_t M = 0;
    int8_t *spins = nullptr;
    cudaStream_t stream = nullptr;
    uint64_t *d_seed = nullptr, *d_A = nullptr, *d_hash = nullptr, *d_clkM = nullptr;
    int64_t *d_clkE = nullptr, *d_flips = nullptr, *d_steps = nullptr;
    double *d_h = nullptr, *d_t = nullptr;
    int *d_err = nullptr;
    double J = 1.0, nu = 1.0;
    int64_t sched_done = 0;
    std::string err;
};

namespace {

kmc_status part_fail(kmc_part *g, kmc_status s, const char *fmt, ...)
{
    if (g) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        g->err = buf;
    }
    return s;
}

#define PART_CUDA_TRY(g, call)                                                                   \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return part_fail((g), KMC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

void part_free(kmc_part *g)
{
    void *ptrs[] = {g->d_seed, g->d_A, g->d_hash, g->d_clkM, g->d_clkE, g->d_flips, g->d_steps, g->d_h, g->d_t,
                    g->d_err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

// Allocates unless an earlier allocation failed; keeps the first error.
template <typename T>
bool part_alloc(T **p, size_t n, cudaError_t &first)
{
    if (first != cudaSuccess) return false;
    first = cudaMalloc((void **)p, (n ? n : 1) * sizeof(T));
    return first == cudaSuccess;
}

} // namespace

extern "C" {

kmc_status kmc_part_set_rates(kmc_part *g, double J, const double *beta, const double *h, double nu, int32_t rate_law)
{
    if (!g) return KMC_EINVAL;
    if (!beta || !h) return part_fail(g, KMC_EINVAL, "beta and h arrays required");
    if (rate_law != KMC_RATE_METROPOLIS && rate_law != KMC_RATE_BARKER) return part_fail(g, KMC_EINVAL, "bad rate law");
    if (!std::isfinite(J) || !(nu > 0.0) || !std::isfinite(nu)) return part_fail(g, KMC_EINVAL, "J finite and nu > 0 required");
    std::vector<double> a((size_t)g->n_traj * 10), gb(10), gh(10);
    std::vector<uint64_t> A((size_t)g->n_traj * 10);
    for (int i = 0; i < g->n_traj; ++i) {
        if (!(beta[i] >= 0.0) || !std::isfinite(beta[i]) || !std::isfinite(h[i]))
            return part_fail(g, KMC_EINVAL, "trajectory %d: beta >= 0 and finite h required", i);
        // A_c = round(a_c 2^P), P = 63 - ceil(log2 n_d): the lattice table with log2 n_d rounded up
        build_table(J, beta[i], h[i], rate_law, 63 - g->P, &a[(size_t)i * 10], &A[(size_t)i * 10], gb.data(), gh.data());
        const int z = zero_rate_class(&A[(size_t)i * 10], 10);
        if (z >= 0)
            return part_fail(g, KMC_ENOTBALANCED, "trajectory %d class %d: a_c = %.3g rounds to 0 in fixed point "
                             "(one-way rate, Eq. 4)", i, z, a[(size_t)i * 10 + z]);
        for (int c = 0; c < 10; ++c) {
            const int up = c / 5, q = c % 5;
            const double dE = 2.0 * (up ? 1.0 : -1.0) * (J * (double)(2 * q - 4) + h[i]);
            const double ratio = a[(size_t)i * 10 + c] / a[(size_t)i * 10 + 5 * (1 - up) + q];
            const double want = std::exp(-beta[i] * dE);
            if (std::fabs(ratio - want) > 1e-12 * want)
                return part_fail(g, KMC_ENOTBALANCED, "trajectory %d class %d: a_c/a_cbar = %.17g, exp(-beta dE) = %.17g",
                                 i, c, ratio, want);
        }
    }
    PART_CUDA_TRY(g, cudaMemcpyAsync(g->d_A, A.data(), A.size() * 8, cudaMemcpyHostToDevice, g->stream));
    PART_CUDA_TRY(g, cudaMemcpyAsync(g->d_h, h, (size_t)g->n_traj * 8, cudaMemcpyHostToDevice, g->stream));
    PART_CUDA_TRY(g, cudaStreamSynchronize(g->stream));
    g->J = J;
    g->nu = nu;
    return KMC_OK;
}

kmc_status kmc_part_create(kmc_part **out, int32_t n_traj, int32_t L, int32_t partition, int32_t n_domains,
                           int32_t k_steps, const uint64_t *seeds, int8_t *spins_dev, void *stream)
{
    if (!out) return KMC_EINVAL;
    *out = nullptr;
    if (n_traj < 1 || L < 2 || L > kmcpart::PART_MAX_L || n_domains < 1 || n_domains > 64 || k_steps < 0 ||
        k_steps > 65535 || !seeds || !spins_dev)
        return KMC_EINVAL;
    int Dx = 0, W = 0, H = 0, ncol = 1;
    if (partition == KMC_PART_BLOCKS) {
        while ((Dx + 1) * (Dx + 1) <= n_domains) ++Dx;
        if (Dx * Dx != n_domains || L % Dx != 0) return KMC_EINVAL;
        W = H = L / Dx;
        ncol = (Dx == 1) ? 1 : 4;
    } else if (partition == KMC_PART_STRIPES) {
        if (L % n_domains != 0) return KMC_EINVAL;
        W = L / n_domains;
        H = L;
        ncol = (n_domains == 1) ? 1 : 2;
    } else {
        return KMC_EINVAL;
    }
    const int nd = W * H;
    if (nd > 16384) return KMC_EINVAL;
    int lg = 0;
    while ((1 << lg) < nd) ++lg;
    kmc_part *g = new kmc_part();
    g->n_traj = n_traj;
    g->L = L;
    g->kind = partition;
    g->ND = n_domains;
    g->k = k_steps;
    g->Dx = Dx;
    g->W = W;
    g->H = H;
    g->ncol = ncol;
    g->P = 63 - lg;
    g->M = (uint64_t)nd << g->P;
    g->spins = spins_dev;
    g->stream = (cudaStream_t)stream;
    const size_t n = (size_t)n_traj;
    cudaError_t ae = cudaSuccess;
    if (!part_alloc(&g->d_seed, n, ae) || !part_alloc(&g->d_A, n * 10, ae) || !part_alloc(&g->d_hash, n, ae) ||
        !part_alloc(&g->d_clkM, n, ae) || !part_alloc(&g->d_clkE, n, ae) || !part_alloc(&g->d_flips, n, ae) ||
        !part_alloc(&g->d_steps, n, ae) || !part_alloc(&g->d_h, n, ae) || !part_alloc(&g->d_t, n, ae) ||
        !part_alloc(&g->d_err, 1, ae)) {
        cudaGetLastError();
        part_free(g);
        delete g;
        return alloc_status(ae);
    }
    std::vector<uint64_t> basis(n, HASH_BASIS), one(n, 1ull << 63);
    if (cudaMemcpyAsync(g->d_seed, seeds, n * 8, cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
        cudaMemcpyAsync(g->d_hash, basis.data(), n * 8, cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
        cudaMemcpyAsync(g->d_clkM, one.data(), n * 8, cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->d_clkE, 0, n * 8, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->d_flips, 0, n * 8, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->d_steps, 0, n * 8, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->d_t, 0, n * 8, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess) {
        cudaGetLastError();
        part_free(g);
        delete g;
        return KMC_ECUDA;
    }
    std::vector<double> beta(n, 1.0 / 2.4), h(n, 0.0);
    kmc_status st = kmc_part_set_rates(g, 1.0, beta.data(), h.data(), 1.0, KMC_RATE_BARKER);
    if (st != KMC_OK) {
        part_free(g);
        delete g;
        return st;
    }
    *out = g;
    return KMC_OK;
}

kmc_status kmc_part_run(kmc_part *g, int64_t n_schedules, int32_t schedule, int32_t time_mode, int32_t obs_every,
                        double *obs_dev, void *stream)
{
    if (!g) return KMC_EINVAL;
    if (n_schedules < 0 || obs_every < 0) return part_fail(g, KMC_EINVAL, "n_schedules and obs_every must be >= 0");
    if (schedule != KMC_SCHEDULE_PALINDROME && schedule != KMC_SCHEDULE_FIXED && schedule != KMC_SCHEDULE_RANDOM_PERM)
        return part_fail(g, KMC_EINVAL, "bad schedule %d", schedule);
    if (schedule != KMC_SCHEDULE_RANDOM_PERM) {
        const int per_side = (g->kind == KMC_PART_BLOCKS) ? g->Dx : g->ND;
        if (per_side != 1 && (per_side & 1))
            return part_fail(g, KMC_EINVAL, "colour schedules need an even number of %s (or one domain)",
                             g->kind == KMC_PART_BLOCKS ? "blocks per side" : "stripes");
    }
    if (time_mode != KMC_TIME_EXPONENTIAL && time_mode != KMC_TIME_EXPECTED)
        return part_fail(g, KMC_EINVAL, "KMC_TIME_EXPONENTIAL or KMC_TIME_EXPECTED required");
    if ((reinterpret_cast<uintptr_t>(obs_dev) & 31u) != 0) return part_fail(g, KMC_EINVAL, "obs_dev must be 32-byte aligned");
    if (g->sched_done > (int64_t)(((1ull << 56) / kmcpart::PART_PHASE_SLOTS) - (uint64_t)n_schedules))
        return part_fail(g, KMC_EINVAL, "schedule count past the Philox phase range");
    if (n_schedules == 0) return KMC_OK;
    const int passes = (schedule == KMC_SCHEDULE_RANDOM_PERM) ? g->ND
                       : (schedule == KMC_SCHEDULE_PALINDROME ? 2 * g->ncol : g->ncol);
    const int64_t n_rec = obs_every > 0 ? n_schedules * passes / obs_every : 0;
    g->stream = (cudaStream_t)stream;
    NvtxRange range("kmc_part_run %d trajectories L=%d N_D=%d %lld schedules", g->n_traj, g->L, g->ND,
                    (long long)n_schedules);
    kmcpart::PartParams P;
    P.n_traj = g->n_traj;
    P.L = g->L;
    P.kind = g->kind;
    P.ND = g->ND;
    P.k = g->k;
    P.Dx = g->Dx;
    P.W = g->W;
    P.H = g->H;
    P.ncol = g->ncol;
    P.schedule = schedule;
    P.obs_every = n_rec > 0 ? obs_every : 0;
    P.sched_begin = g->sched_done;
    P.n_sched = n_schedules;
    P.M = g->M;
    P.J = g->J;
    P.nu = g->nu;
    P.seed = g->d_seed;
    P.A = g->d_A;
    P.h = g->d_h;
    P.spins = g->spins;
    P.hash = g->d_hash;
    P.clkM = g->d_clkM;
    P.clkE = g->d_clkE;
    P.flips = g->d_flips;
    P.steps = g->d_steps;
    P.t = g->d_t;
    P.obs = n_rec > 0 ? obs_dev : nullptr;
    P.err = g->d_err;
    const int blocks = (g->n_traj + kmcpart::PART_WARPS - 1) / kmcpart::PART_WARPS;
    const size_t smem = (size_t)kmcpart::PART_WARPS * kmcpart::PART_WARP_WORDS * sizeof(uint64_t);
    if (time_mode == KMC_TIME_EXPONENTIAL)
        kmcpart::part_kernel<true><<<blocks, kmcpart::PART_WARPS * 32, smem, g->stream>>>(P);
    else
        kmcpart::part_kernel<false><<<blocks, kmcpart::PART_WARPS * 32, smem, g->stream>>>(P);
    PART_CUDA_TRY(g, cudaGetLastError());
    g->sched_done += n_schedules;
    return KMC_OK;
}

kmc_status kmc_part_state(kmc_part *g, uint64_t *hash, int64_t *flips, int64_t *steps, double *t)
{
    if (!g) return KMC_EINVAL;
    PART_CUDA_TRY(g, cudaStreamSynchronize(g->stream));
    int err = 0;
    PART_CUDA_TRY(g, cudaMemcpy(&err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    const size_t n = (size_t)g->n_traj * 8;
    if (hash) PART_CUDA_TRY(g, cudaMemcpy(hash, g->d_hash, n, cudaMemcpyDeviceToHost));
    if (flips) PART_CUDA_TRY(g, cudaMemcpy(flips, g->d_flips, n, cudaMemcpyDeviceToHost));
    if (steps) PART_CUDA_TRY(g, cudaMemcpy(steps, g->d_steps, n, cudaMemcpyDeviceToHost));
    if (t) PART_CUDA_TRY(g, cudaMemcpy(t, g->d_t, n, cudaMemcpyDeviceToHost));
    if (err & 1) return part_fail(g, KMC_EDEVICE, "a spin byte was not +1 or -1");
    if (err) return part_fail(g, KMC_EDEVICE, "device error word %d", err);
    return KMC_OK;
}

const char *kmc_part_last_error(const kmc_part *g) { return g ? g->err.c_str() : "null partitioned lattice"; }

void kmc_part_destroy(kmc_part *g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    part_free(g);
    delete g;
}

} // extern "C"
