// kmc_kernels.cuh -- sm_103a device code of the sequential-update parallel
// kinetic Monte Carlo (Nilmeier & Marian, arXiv:1403.4674).
//
// Data layout (device memory, between launches):
//   * caller spins: int8, replicas concatenated, row-major.
//   * bit tiles: replica r, domain d = by*Dx + bx owns LD*LD bits, row y of
//     the domain at bits [y*LD, (y+1)*LD) of the tile, bit x = column x,
//     1 = spin up.  Tile bytes = LD*LD/8.  Global domain id g = dom_off[r] + d.
//   * edges[g*4 + {N,S,W,E}]: the domain's first row, last row, first column
//     and last column as bit masks.  Column bit of row y is
//     (y % RPL)*32 + y / RPL (RPL = rows per lane, 2 for LD = 64, else 1).
//   * per-domain counters dctr[g*6 + ...]: event hash, real flips, clock
//     mantissa, clock exponent, score d/dbeta, score d/dh.
//
// The run kernel is persistent: every CTA owns a fixed set of domains (its
// "slots") for the whole launch; their tiles, edges, counters and the rate
// tables of their replicas live in shared memory.  Between colour phases the
// only communication is the frozen halo (Sec. 2.2) -- the four edge words of
// each neighbour:
//   * CLUSTER mode: every replica is resident in one thread-block cluster
//     (1..16 CTAs); halos are read from the owner CTA through distributed
//     shared memory and phases are separated by the hardware cluster barrier;
//   * GRID mode (a replica larger than a cluster can hold): one cooperative
//     grid; halos go through L2 and phases are separated by a bounded grid
//     barrier.
#pragma once

#include <cstdint>
#include <type_traits>

namespace kmcdev {

constexpr uint32_t FULL_WARP = 0xffffffffu;
constexpr int EDGE_N = 0, EDGE_S = 1, EDGE_W = 2, EDGE_E = 3;
constexpr int DCTR_HASH = 0, DCTR_FLIPS = 1, DCTR_CLKM = 2, DCTR_CLKE = 3,
              DCTR_SB = 4, DCTR_SH = 5, DCTR_WORDS = 6;
constexpr uint64_t HASH_BASIS = 0xcbf29ce484222325ull; // FNV-1a 64 offset basis
constexpr uint64_t HASH_PRIME = 0x00000100000001b3ull; // FNV-1a 64 prime
constexpr uint32_t TAG_INIT = 1u, TAG_PERM = 2u;       // step draws use tag 0
constexpr int ERR_TIMEOUT = 1, ERR_SPIN = 2, ERR_INTERNAL = 3;
constexpr int SCHED_PALINDROME = 0, SCHED_FIXED = 1, SCHED_RANDOM_PERM = 2;
constexpr int OBS_WORDS = 5; // bonds, mag, clock sum, score beta sum, score h sum

// Replica table staged in shared memory (bytes):
//   [0,128) A[16] fixed-point acceptance, [128,256) inv[16] = floor((2^64-1)/A),
//   [256,512) grad[32] = a[10], dlog a/dbeta[10], dlog a/dh[10],
//   [512] seed, [520] dom_off, [524] Dx.
constexpr int RT_BYTES = 528;
constexpr int RT_SEED = 512, RT_DOMOFF = 520, RT_DX = 524;
// Slot: [tile][edges 32][counters 48][meta 32]; meta u32: g, replica, d, rt, nb[4].
constexpr int SLOT_EXTRA = 32 + 48 + 32;
constexpr int META_G = 0, META_R = 1, META_D = 2, META_RT = 3, META_NB = 4;

template <int LD> __host__ __device__ constexpr int slot_bytes() { return ((LD * LD / 8 + SLOT_EXTRA) + 15) / 16 * 16; }

struct RunParams {
    int n_rep;
    int k;
    int schedule;
    int obs_every;
    int64_t sched_begin;
    int64_t n_sched;
    int64_t visits_before; // per-domain visits before this launch (clock mode EXPECTED)
    // per replica (global)
    const int32_t *rep_Dx;
    const uint32_t *rep_dom_off;
    const uint64_t *rep_seed;
    const uint64_t *rep_A;   // [n_rep][16]
    const uint64_t *rep_inv; // [n_rep][16]
    const double *rep_grad;  // [n_rep][32]
    // plan: per CTA slot ranges (colour-sorted), replica tables, neighbours
    const uint32_t *cta_slot_off; // [n_cta + 1]
    const uint32_t *cta_col_off;  // [n_cta][5], relative to the CTA's first slot
    const uint32_t *cta_rt_off;   // [n_cta + 1]
    const uint32_t *rt_rep;       // replica id of each staged table
    const uint32_t *slot_g;       // global domain id of each slot
    const uint32_t *slot_rt;      // local table index of each slot
    const uint32_t *slot_nb;      // [n_slots][4]: GRID: neighbour g; CLUSTER: rank << 24 | local slot
    int max_rt;                   // table capacity per CTA (uniform layout)
    int cluster;                  // 0 = GRID mode, else cluster size
    // state
    uint8_t *tiles;
    uint64_t *dctr;
    uint64_t *edges;
    // observables scratch [n_obs][n_rep][OBS_WORDS]
    unsigned long long *obs_acc;
    // grid barrier
    unsigned *bar_count;
    int *err;
    uint64_t bar_limit_ns;
    int debug_extra;
    double lambda; // n_d * nu
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), device side.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 key)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ key.x, lo1, hi0 ^ c.w ^ key.y, lo0);
        key.x += 0x9E3779B9u;
        key.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint64_t ld_cg(const uint64_t *p)
{
    return (uint64_t)__ldcg((const unsigned long long *)p);
}
__device__ __forceinline__ void st_cg(uint64_t *p, uint64_t v)
{
    __stcg((unsigned long long *)p, (unsigned long long)v);
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// distributed shared memory (thread-block clusters)
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t map_rank(uint32_t local_addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
    return r;
}
__device__ __forceinline__ uint64_t ld_dsmem(uint32_t addr)
{
    uint64_t v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Per-domain-size geometry.
// ---------------------------------------------------------------------------
template <int LD> struct Geo {
    static_assert(LD == 8 || LD == 16 || LD == 32 || LD == 64, "domain side");
    static constexpr int RPL = LD > 32 ? LD / 32 : 1;  // rows per lane
    static constexpr int NACT = LD >= 32 ? 32 : LD;    // lanes holding rows
    static constexpr int TILE_BYTES = LD * LD / 8;
    using row_t = typename std::conditional<(LD > 32), uint64_t, uint32_t>::type;
    using mem_t = typename std::conditional<
        LD == 64, uint64_t,
        typename std::conditional<LD == 32, uint32_t,
                                  typename std::conditional<LD == 16, uint16_t, uint8_t>::type>::type>::type;
    static constexpr row_t FULL = (LD >= 64) ? (row_t)~0ull : (row_t)((1ull << LD) - 1ull);
};

__device__ __forceinline__ int popc_row(uint32_t v) { return __popc(v); }
__device__ __forceinline__ int popc_row(uint64_t v) { return __popcll(v); }

// Position of the rr-th (0-based) set bit of m; rr < popc(m).
__device__ __forceinline__ int select_bit(uint64_t m, uint32_t rr)
{
    int pos = 0;
    uint32_t w = (uint32_t)m;
    uint32_t c = __popc(w);
    if (rr >= c) { rr -= c; w = (uint32_t)(m >> 32); pos = 32; }
    c = __popc(w & 0xFFFFu); if (rr >= c) { rr -= c; w >>= 16; pos += 16; }
    c = __popc(w & 0xFFu);   if (rr >= c) { rr -= c; w >>= 8;  pos += 8; }
    c = __popc(w & 0xFu);    if (rr >= c) { rr -= c; w >>= 4;  pos += 4; }
    c = __popc(w & 0x3u);    if (rr >= c) { rr -= c; w >>= 2;  pos += 2; }
    if (rr >= (w & 1u)) pos += 1;
    return pos;
}

// Exclusive prefix over lanes of a small count v < 2^NBITS, from NBITS ballots
// of its bit planes (no shuffle chain).
template <int NBITS>
__device__ __forceinline__ uint32_t excl_prefix_small(uint32_t v, int lane)
{
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t s = 0;
#pragma unroll
    for (int b = 0; b < NBITS; ++b) s += (uint32_t)__popc(__ballot_sync(FULL_WARP, (v >> b) & 1u) & lt) << b;
    return s;
}

// Normalised unsigned mantissa product for the exponential clock:
// value = (m / 2^63) * 2^e with m in [2^63, 2^64).
__device__ __forceinline__ void mant_mul(uint64_t &m, int64_t &e, uint64_t m2, int64_t e2)
{
    const uint64_t hi = __umul64hi(m, m2);
    const uint64_t lo = m * m2;
    if (hi >> 63) {
        m = hi;
        e = e + e2 + 1;
    } else {
        m = (hi << 1) | (lo >> 63);
        e = e + e2;
    }
}

// Domain clock from its state: EXPONENTIAL: -ln(prod v)/Lambda; EXPECTED: steps/Lambda.
__device__ __forceinline__ double domain_time(bool expo, uint64_t M, int64_t E, int64_t steps,
                                              double lambda)
{
    if (expo) {
        const double lnm = log(ldexp((double)M, -63));
        const double tot = __dadd_rn(lnm, __dmul_rn((double)E, 0.69314718055994530942));
        return __ddiv_rn(-tot, lambda);
    }
    return __ddiv_rn((double)steps, lambda);
}

// ---------------------------------------------------------------------------
// Row-plane state of one domain held by one warp: lane l holds rows
// l*RPL .. l*RPL+RPL-1 (bit x = column x), plus the bit-sliced count of up
// neighbours b2 b1 b0 of every site (App. A: the site's class is
// 5*(spin up) + number of up neighbours).
// ---------------------------------------------------------------------------
template <int LD> struct Planes {
    using G = Geo<LD>;
    using row_t = typename G::row_t;
    row_t S[G::RPL], b0[G::RPL], b1[G::RPL], b2[G::RPL];
    row_t valid;

    __device__ __forceinline__ void build(int lane, row_t hN, row_t hS, uint64_t hW, uint64_t hE)
    {
        row_t U[G::RPL], D[G::RPL];
        if (G::RPL == 2) {
            const row_t up = __shfl_up_sync(FULL_WARP, S[G::RPL - 1], 1);
            U[0] = (lane == 0) ? hN : up;
            D[0] = S[1 % G::RPL];
            U[1 % G::RPL] = S[0];
            const row_t dn = __shfl_down_sync(FULL_WARP, S[0], 1);
            D[G::RPL - 1] = (lane == G::NACT - 1) ? hS : dn;
        } else {
            const row_t up = __shfl_up_sync(FULL_WARP, S[0], 1);
            const row_t dn = __shfl_down_sync(FULL_WARP, S[0], 1);
            U[0] = (lane == 0) ? hN : up;
            D[0] = (lane == G::NACT - 1) ? hS : dn;
        }
#pragma unroll
        for (int t = 0; t < G::RPL; ++t) {
            const int y = lane * G::RPL + t;
            const int cb = (y % G::RPL) * 32 + y / G::RPL;
            const row_t hw = (row_t)((hW >> cb) & 1ull);
            const row_t he = (row_t)((hE >> cb) & 1ull);
            const row_t Wn = (row_t)(((S[t] << 1) | hw) & G::FULL);
            const row_t En = (row_t)((S[t] >> 1) | (he << (LD - 1)));
            const row_t s1 = U[t] ^ D[t], c1 = U[t] & D[t];
            const row_t s2 = Wn ^ En, c2 = Wn & En;
            const row_t t0 = s1 & s2;
            b0[t] = s1 ^ s2;
            b1[t] = c1 ^ c2 ^ t0;
            b2[t] = (c1 & c2) | (c1 & t0) | (c2 & t0);
        }
    }

    // sites of class c = 5*up + q in row t
    __device__ __forceinline__ row_t mask(int c, int t) const
    {
        const bool up = c >= 5;
        const int q = up ? c - 5 : c;
        const row_t sp = up ? S[t] : (row_t)~S[t];
        row_t e;
        if (q == 4) {
            e = b2[t];
        } else {
            e = (row_t)~b2[t] & ((q & 2) ? b1[t] : (row_t)~b1[t]) & ((q & 1) ? b0[t] : (row_t)~b0[t]);
        }
        return sp & e & valid;
    }
};

// Class counts of the warp's domain: lane c (< 10) receives n_c.
template <int LD>
__device__ __forceinline__ uint32_t class_counts(const Planes<LD> &P, int lane)
{
    uint32_t mine = 0;
#pragma unroll
    for (int c = 0; c < 10; ++c) {
        uint32_t cnt = 0;
#pragma unroll
        for (int t = 0; t < Geo<LD>::RPL; ++t) cnt += popc_row(P.mask(c, t));
        const uint32_t tot = __reduce_add_sync(FULL_WARP, cnt);
        if (lane == c) mine = tot;
    }
    return mine;
}

// Inclusive prefix over lanes 0..15 of w (64-bit).
__device__ __forceinline__ uint64_t prefix16(uint64_t w, int lane)
{
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
        const uint64_t v = __shfl_up_sync(FULL_WARP, w, off);
        if (lane >= off) w += v;
    }
    return w;
}

__device__ __forceinline__ double warp_sum10(double v)
{
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) v += __shfl_xor_sync(FULL_WARP, v, off);
    return v;
}

// Per-domain counters, identical in every lane during a visit.
struct Counters {
    uint64_t H, flips, clkM;
    int64_t clkE;
    double sb, sh;
};

// ---------------------------------------------------------------------------
// One domain visit (Sec. 2.2): nfused consecutive global phases of the same
// colour, k uniformised steps each, with the halo hN/hS/hW/hE frozen.
//
// Step j of global phase np draws Philox {j, d, np_lo, np_hi} with the replica
// seed: target = (w0 | w1<<32) >> 1 uniform on [0, n_d 2^P), V = (w2 | w3<<32)
// >> 11 plus 1.  target >= R' = sum_c n_c A_c is a null step (the diagonal of
// App. A Eq. Glauber_TM); otherwise class c = first class whose inclusive
// cumulative rate exceeds target, member jj = (target - C_{c-1}) / A_c in
// row-major order flips (the n-fold way's cumulative selection, Sec. 2.1).
// Steps are drawn 32 at a time (lane i draws step base+i); runs of null steps
// are skipped with one ballot since the state does not change between real
// events.  rt: the replica table in shared memory.
// ---------------------------------------------------------------------------
template <int LD, bool EXPO, bool GRAD>
__device__ __forceinline__ void visit_core(Planes<LD> &pl, Counters &cn, const uint8_t *rt,
                                           typename Geo<LD>::row_t hN, typename Geo<LD>::row_t hS,
                                           uint64_t hW, uint64_t hE, uint32_t d, uint64_t np0,
                                           int nfused, int k, int lane, int *err)
{
    using G = Geo<LD>;
    using row_t = typename G::row_t;
    const uint64_t seed = *reinterpret_cast<const uint64_t *>(rt + RT_SEED);
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    uint64_t Ac = 0, invc = 0;
    double a_c = 0.0, gb_c = 0.0, gh_c = 0.0;
    if (lane < 10) {
        Ac = reinterpret_cast<const uint64_t *>(rt)[lane];
        invc = reinterpret_cast<const uint64_t *>(rt + 128)[lane];
        if (GRAD) {
            const double *gr = reinterpret_cast<const double *>(rt + 256);
            a_c = gr[lane];
            gb_c = gr[10 + lane];
            gh_c = gr[20 + lane];
        }
    }
    pl.build(lane, hN, hS, hW, hE);
    uint32_t n_c = class_counts<LD>(pl, lane);
    uint64_t Wc = (uint64_t)n_c * Ac;
    uint64_t Cinc = prefix16(Wc, lane);
    uint64_t R = __shfl_sync(FULL_WARP, Cinc, 9);

    double nd_minus_R = 0.0, Db = 0.0, Dh = 0.0;
    auto grad_state = [&]() {
        if (GRAD) {
            const double w = (double)n_c * a_c;
            const double Rr = warp_sum10(w);
            Db = warp_sum10(w * gb_c);
            Dh = warp_sum10(w * gh_c);
            nd_minus_R = (double)(LD * LD) - Rr;
        }
    };
    grad_state();

    const int total = nfused * k;
    for (int base = 0; base < total; base += 32) {
        const int s = base + lane;
        uint64_t tgt = ~0ull;
        uint64_t V = 1ull << 53;
        if (s < total) {
            const int f = s / k;
            const int j = s - f * k;
            const uint64_t np = np0 + (uint64_t)f;
            const uint4 w = philox4x32_10(
                make_uint4((uint32_t)j, d, (uint32_t)np, (uint32_t)(np >> 32) & 0xFFFFFFu), key);
            tgt = (((uint64_t)w.y << 32) | w.x) >> 1;
            V = ((((uint64_t)w.w << 32) | w.z) >> 11) + 1ull;
        }
        const int chunk_end = min(32, total - base);
        int pos = 0;
        while (true) {
            const unsigned real = __ballot_sync(FULL_WARP, lane >= pos && tgt < R);
            const int jx = real ? __ffs(real) - 1 : chunk_end;
            if (GRAD && jx > pos) {
                // (jx - pos) null steps in the current state: d log(1 - R/n_d)
                const double q = (double)(jx - pos);
                cn.sb -= q * Db / nd_minus_R;
                cn.sh -= q * Dh / nd_minus_R;
            }
            if (!real) break;
            const uint64_t t = __shfl_sync(FULL_WARP, tgt, jx);
            const unsigned sel = __ballot_sync(FULL_WARP, lane < 10 && t < Cinc);
            const int c = __ffs(sel) - 1;
            uint64_t q = 0;
            if (lane == c) {
                const uint64_t x = t - (Cinc - Wc);
                q = __umul64hi(x, invc);
                if ((q + 1) * Ac <= x) ++q;
                if ((q + 1) * Ac <= x) ++q;
                if ((q + 1) * Ac <= x) ++q;
            }
            const uint32_t jj = (uint32_t)__shfl_sync(FULL_WARP, q, c);
            if (GRAD) {
                cn.sb += __shfl_sync(FULL_WARP, gb_c, c);
                cn.sh += __shfl_sync(FULL_WARP, gh_c, c);
            }
            // rank selection: jj-th member of class c in row-major order
            row_t m[G::RPL];
            uint32_t cl = 0;
#pragma unroll
            for (int tt = 0; tt < G::RPL; ++tt) {
                m[tt] = pl.mask(c, tt);
                cl += popc_row(m[tt]);
            }
            const uint32_t excl = excl_prefix_small<(LD > 32) ? 8 : 7>(cl, lane);
            const unsigned win = __ballot_sync(FULL_WARP, jj >= excl && jj < excl + cl);
            if (!win) {
                if (lane == 0) atomicCAS(err, 0, ERR_INTERNAL);
                break;
            }
            const int wl = __ffs(win) - 1;
            uint32_t yc = 0;
            if (lane == wl) {
                uint32_t rr = jj - excl;
                int tsel = 0;
                if (G::RPL == 2) {
                    const uint32_t p0 = (uint32_t)popc_row(m[0]);
                    if (rr >= p0) { rr -= p0; tsel = 1; }
                }
                const int col = select_bit((uint64_t)(tsel ? m[G::RPL - 1] : m[0]), rr);
                yc = ((uint32_t)(lane * G::RPL + tsel) << 8) | (uint32_t)col;
            }
            yc = __shfl_sync(FULL_WARP, yc, wl);
            const int y = (int)(yc >> 8), col = (int)(yc & 255u);
#pragma unroll
            for (int tt = 0; tt < G::RPL; ++tt)
                if (lane * G::RPL + tt == y) pl.S[tt] ^= (row_t)1 << col;
            {
                const int sx = base + jx;
                const int f = sx / k;
                const int j = sx - f * k;
                const uint64_t np = np0 + (uint64_t)f;
                const uint64_t e = (np << 32) | ((uint64_t)j << 16) | (uint64_t)(y * LD + col);
                cn.H = (cn.H ^ e) * HASH_PRIME;
                ++cn.flips;
            }
            pl.build(lane, hN, hS, hW, hE);
            n_c = class_counts<LD>(pl, lane);
            Wc = (uint64_t)n_c * Ac;
            Cinc = prefix16(Wc, lane);
            R = __shfl_sync(FULL_WARP, Cinc, 9);
            grad_state();
            pos = jx + 1;
        }
        if (EXPO) {
            const int z = __clzll((long long)V);
            uint64_t m = V << z;
            int64_t e = 10 - z;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const uint64_t m2 = __shfl_xor_sync(FULL_WARP, m, off);
                const int64_t e2 = __shfl_xor_sync(FULL_WARP, e, off);
                mant_mul(m, e, m2, e2);
            }
            mant_mul(cn.clkM, cn.clkE, m, e);
        }
    }
}

// Four edge words of the warp's domain (N row, S row, W column, E column);
// lane i (< 4) returns edge i.
template <int LD>
__device__ __forceinline__ uint64_t edge_words(const typename Geo<LD>::row_t (&S)[Geo<LD>::RPL], int lane)
{
    using G = Geo<LD>;
    uint64_t colW = 0, colE = 0;
#pragma unroll
    for (int t = 0; t < G::RPL; ++t) {
        colW |= (uint64_t)__ballot_sync(FULL_WARP, (S[t] & 1u) != 0) << (32 * t);
        colE |= (uint64_t)__ballot_sync(FULL_WARP, ((S[t] >> (LD - 1)) & 1u) != 0) << (32 * t);
    }
    const uint64_t rowN = (uint64_t)__shfl_sync(FULL_WARP, S[0], 0);
    const uint64_t rowS = (uint64_t)__shfl_sync(FULL_WARP, S[G::RPL - 1], G::NACT - 1);
    return (lane == EDGE_N) ? rowN : (lane == EDGE_S) ? rowS : (lane == EDGE_W) ? colW : colE;
}

// ---------------------------------------------------------------------------
// Endpoint observables of one domain (Sec. 2.3): bond sum over the bonds to
// the east and south neighbours of every site, and the spin sum.
// ---------------------------------------------------------------------------
template <int LD>
__device__ __forceinline__ void domain_bonds_mag(const typename Geo<LD>::row_t (&S)[Geo<LD>::RPL],
                                                 uint64_t hE_col, uint64_t hS_row, int lane,
                                                 int &bonds, int &mag)
{
    using G = Geo<LD>;
    using row_t = typename G::row_t;
    row_t D[G::RPL];
    const row_t dn = __shfl_down_sync(FULL_WARP, S[0], 1);
    if (G::RPL == 2) {
        D[0] = S[1 % G::RPL];
        D[G::RPL - 1] = (lane == G::NACT - 1) ? (row_t)hS_row : dn;
    } else {
        D[0] = (lane == G::NACT - 1) ? (row_t)hS_row : dn;
    }
    int b = 0, m = 0;
    if (lane < G::NACT) {
#pragma unroll
        for (int t = 0; t < G::RPL; ++t) {
            const int y = lane * G::RPL + t;
            const int cb = (y % G::RPL) * 32 + y / G::RPL;
            const row_t s = S[t];
            const row_t dif = (row_t)((s ^ (s >> 1)) & (G::FULL >> 1));
            b += (LD - 1) - 2 * popc_row(dif);
            const int a = (int)((s >> (LD - 1)) & 1u);
            const int e = (int)((hE_col >> cb) & 1ull);
            b += (a == e) ? 1 : -1;
            b += LD - 2 * popc_row((row_t)(s ^ D[t]));
            m += 2 * popc_row(s) - LD;
        }
    }
    bonds = (int)__reduce_add_sync(FULL_WARP, (unsigned)b);
    mag = (int)__reduce_add_sync(FULL_WARP, (unsigned)m);
}

// ---------------------------------------------------------------------------
// Bounded grid barrier (GRID mode).  Thread 0 of every CTA arrives on a
// monotone counter and spins (acquire loads) until all CTAs of barrier `no`
// arrived, or until the limit expires / another CTA reported an error.
// Returns false on error; the caller then leaves the kernel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier(const RunParams &P, unsigned &no, int *s_ok)
{
    __syncthreads();
    ++no;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = no * gridDim.x + (unsigned)P.debug_extra;
        __threadfence();
        atomicAdd(P.bar_count, 1u);
        const uint64_t t0 = global_ns();
        unsigned spins = 0;
        while (ld_acquire(P.bar_count) < target) {
            if ((++spins & 255u) == 0) {
                if (*(volatile int *)P.err != 0) { ok = 0; break; }
                if (global_ns() - t0 > P.bar_limit_ns) {
                    atomicCAS(P.err, 0, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Colour order of schedule n for replica seed (RANDOM_PERM), Lehmer decode of
// floor(x * 24 / 2^64), x = w0 | w1 << 32 of Philox {0, 0, n_lo, n_hi | TAG_PERM << 24}.
__device__ __forceinline__ int perm_colour(uint64_t seed, uint64_t n, int p)
{
    const uint4 w = philox4x32_10(
        make_uint4(0u, 0u, (uint32_t)n, ((uint32_t)(n >> 32) & 0xFFFFFFu) | (TAG_PERM << 24)),
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const uint64_t x = ((uint64_t)w.y << 32) | w.x;
    int idx = (int)__umul64hi(x, 24ull);
    int pool = 0x3210; // nibbles: remaining colours in order
    int colour = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int f = (q == 0) ? 6 : (q == 1) ? 2 : 1; // (3 - q)!
        const int sel = idx / f;
        idx -= sel * f;
        const int c = (pool >> (4 * sel)) & 0xF;
        const int low = pool & ((1 << (4 * sel)) - 1);
        const int high = pool >> (4 * (sel + 1));
        pool = low | (high << (4 * sel));
        if (q == p) colour = c;
    }
    return colour;
}

__device__ __forceinline__ int fixed_colour(int schedule, int p)
{
    if (schedule == SCHED_PALINDROME) return (p < 4) ? p : 7 - p;
    return p;
}

// ---------------------------------------------------------------------------
// Persistent run kernel (both modes).
// ---------------------------------------------------------------------------
template <int LD, bool EXPO, bool GRAD, bool CLUSTER>
__global__ void __launch_bounds__(512, 1) run_kernel(const RunParams P)
{
    using G = Geo<LD>;
    using row_t = typename G::row_t;
    using mem_t = typename G::mem_t;
    constexpr int TB = G::TILE_BYTES;
    constexpr int SB = slot_bytes<LD>();
    constexpr int OFF_EDGE = TB, OFF_CTR = TB + 32, OFF_META = TB + 80;

    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int b = blockIdx.x;
    uint8_t *tables = smem;
    uint8_t *slots = smem + (size_t)P.max_rt * RT_BYTES;
    const uint32_t slot0 = P.cta_slot_off[b];
    const int nslot = (int)(P.cta_slot_off[b + 1] - slot0);
    const uint32_t *col_off = P.cta_col_off + (size_t)b * 5;

    // ---- stage replica tables and owned slots ----
    const uint32_t rt0 = P.cta_rt_off[b];
    const int nrt = (int)(P.cta_rt_off[b + 1] - rt0);
    for (int i = wib; i < nrt; i += nwarps) {
        const uint32_t r = P.rt_rep[rt0 + i];
        uint8_t *t = tables + (size_t)i * RT_BYTES;
        if (lane < 16) {
            reinterpret_cast<uint64_t *>(t)[lane] = P.rep_A[(size_t)r * 16 + lane];
            reinterpret_cast<uint64_t *>(t + 128)[lane] = P.rep_inv[(size_t)r * 16 + lane];
        }
        reinterpret_cast<double *>(t + 256)[lane] = P.rep_grad[(size_t)r * 32 + lane];
        if (lane == 0) {
            *reinterpret_cast<uint64_t *>(t + RT_SEED) = P.rep_seed[r];
            *reinterpret_cast<uint32_t *>(t + RT_DOMOFF) = P.rep_dom_off[r];
            *reinterpret_cast<int32_t *>(t + RT_DX) = P.rep_Dx[r];
        }
    }
    for (int i = wib; i < nslot; i += nwarps) {
        const uint32_t s = slot0 + (uint32_t)i;
        const uint32_t g = P.slot_g[s];
        const uint32_t rt = P.slot_rt[s];
        const uint32_t r = P.rt_rep[rt0 + rt];
        uint8_t *sl = slots + (size_t)i * SB;
        for (int q = lane * 4; q < TB; q += 128)
            *reinterpret_cast<uint32_t *>(sl + q) = *reinterpret_cast<const uint32_t *>(P.tiles + (size_t)g * TB + q);
        if (lane < DCTR_WORDS)
            reinterpret_cast<uint64_t *>(sl + OFF_CTR)[lane] = P.dctr[(size_t)g * DCTR_WORDS + lane];
        uint32_t *meta = reinterpret_cast<uint32_t *>(sl + OFF_META);
        if (lane == 0) {
            meta[META_G] = g;
            meta[META_R] = r;
            meta[META_D] = g - P.rep_dom_off[r];
            meta[META_RT] = rt;
        }
        if (lane < 4) {
            const uint32_t nb = P.slot_nb[(size_t)s * 4 + lane];
            if (CLUSTER) {
                // address of the edge word this slot reads from its neighbour:
                // the N neighbour's S row, the S neighbour's N row, the W
                // neighbour's E column, the E neighbour's W column
                const int want = (lane == EDGE_N) ? EDGE_S : (lane == EDGE_S) ? EDGE_N : (lane == EDGE_W) ? EDGE_E : EDGE_W;
                const uint32_t nrank = nb >> 24, nslot_ = nb & 0xFFFFFFu;
                const uint32_t local = smem_addr(slots + (size_t)nslot_ * SB + OFF_EDGE + 8 * want);
                meta[META_NB + lane] = map_rank(local, nrank);
            } else {
                meta[META_NB + lane] = nb;
            }
        }
        if (CLUSTER) {
            // edges of the staged tile, published in shared memory
            row_t S[G::RPL];
            const mem_t *trow = reinterpret_cast<const mem_t *>(sl);
#pragma unroll
            for (int t = 0; t < G::RPL; ++t) S[t] = (lane < G::NACT) ? (row_t)trow[lane * G::RPL + t] : (row_t)0;
            const uint64_t ew = edge_words<LD>(S, lane);
            if (lane < 4) reinterpret_cast<uint64_t *>(sl + OFF_EDGE)[lane] = ew;
        }
    }
    if (CLUSTER) cluster_sync();
    else __syncthreads();

    // halo of a slot: four edge words of its neighbours
    auto read_halo = [&](const uint32_t *meta, uint64_t &hN, uint64_t &hS, uint64_t &hW, uint64_t &hE) {
        if (CLUSTER) {
            hN = ld_dsmem(meta[META_NB + EDGE_N]);
            hS = ld_dsmem(meta[META_NB + EDGE_S]);
            hW = ld_dsmem(meta[META_NB + EDGE_W]);
            hE = ld_dsmem(meta[META_NB + EDGE_E]);
        } else {
            hN = ld_cg(&P.edges[(size_t)meta[META_NB + EDGE_N] * 4 + EDGE_S]);
            hS = ld_cg(&P.edges[(size_t)meta[META_NB + EDGE_S] * 4 + EDGE_N]);
            hW = ld_cg(&P.edges[(size_t)meta[META_NB + EDGE_W] * 4 + EDGE_E]);
            hE = ld_cg(&P.edges[(size_t)meta[META_NB + EDGE_E] * 4 + EDGE_W]);
        }
    };

    auto visit = [&](uint8_t *sl, uint64_t np0, int nf) {
        const uint32_t *meta = reinterpret_cast<const uint32_t *>(sl + OFF_META);
        uint64_t hN, hS, hW, hE;
        read_halo(meta, hN, hS, hW, hE);
        const uint8_t *rt = tables + (size_t)meta[META_RT] * RT_BYTES;
        Planes<LD> pl;
        pl.valid = (lane < G::NACT) ? G::FULL : (row_t)0;
        const mem_t *trow = reinterpret_cast<const mem_t *>(sl);
#pragma unroll
        for (int t = 0; t < G::RPL; ++t) pl.S[t] = (lane < G::NACT) ? (row_t)trow[lane * G::RPL + t] : (row_t)0;
        uint64_t *ctr = reinterpret_cast<uint64_t *>(sl + OFF_CTR);
        Counters cn;
        cn.H = ctr[DCTR_HASH];
        cn.flips = 0;
        cn.clkM = ctr[DCTR_CLKM];
        cn.clkE = (int64_t)ctr[DCTR_CLKE];
        cn.sb = 0.0;
        cn.sh = 0.0;
        visit_core<LD, EXPO, GRAD>(pl, cn, rt, (row_t)hN, (row_t)hS, hW, hE, meta[META_D], np0, nf, P.k, lane, P.err);
        mem_t *wrow = reinterpret_cast<mem_t *>(sl);
        if (lane < G::NACT) {
#pragma unroll
            for (int t = 0; t < G::RPL; ++t) wrow[lane * G::RPL + t] = (mem_t)pl.S[t];
        }
        const uint64_t ew = edge_words<LD>(pl.S, lane);
        if (lane < 4) {
            if (CLUSTER) reinterpret_cast<uint64_t *>(sl + OFF_EDGE)[lane] = ew;
            else st_cg(&P.edges[(size_t)meta[META_G] * 4 + lane], ew);
        }
        if (lane == 0) {
            ctr[DCTR_HASH] = cn.H;
            ctr[DCTR_FLIPS] += cn.flips;
            ctr[DCTR_CLKM] = cn.clkM;
            ctr[DCTR_CLKE] = (uint64_t)cn.clkE;
            if (GRAD) {
                reinterpret_cast<double *>(ctr)[DCTR_SB] += cn.sb;
                reinterpret_cast<double *>(ctr)[DCTR_SH] += cn.sh;
            }
        }
        __syncwarp();
    };

    auto phase_sync = [&](unsigned &bar_no) -> bool {
        if (CLUSTER) {
            cluster_sync();
            return true;
        }
        return grid_barrier(P, bar_no, &s_ok);
    };

    const int nph = (P.schedule == SCHED_PALINDROME) ? 8 : 4;
    const uint64_t gp_begin = (uint64_t)P.sched_begin * nph;
    const uint64_t gp_end = (uint64_t)(P.sched_begin + P.n_sched) * nph;
    unsigned bar_no = 0;
    bool started = false;
    bool ok = true;
    uint64_t gp = gp_begin;
    while (gp < gp_end && ok) {
        const uint64_t n = gp / nph;
        const int p = (int)(gp % nph);
        // global phase index of the Philox counter: 8 slots per schedule for every
        // schedule kind; the palindrome's fused phases (3,4) and seam (7 | next 0)
        // have consecutive indices
        const uint64_t np0 = n * 8 + (uint64_t)p;
        int nf = 1;
        int colour = 0;
        if (P.schedule != SCHED_RANDOM_PERM) {
            colour = fixed_colour(P.schedule, p);
            // fuse following phases of the same colour unless an observation intervenes
            while (gp + nf < gp_end) {
                const uint64_t g2 = gp + nf;
                const int p2 = (int)(g2 % nph);
                if (fixed_colour(P.schedule, p2) != colour) break;
                if (p2 == 0) {
                    const int64_t nl_prev = (int64_t)(g2 / nph - 1 - (uint64_t)P.sched_begin);
                    if (P.obs_every > 0 && ((nl_prev + 1) % P.obs_every) == 0) break;
                }
                ++nf;
            }
        }
        if (started) ok = phase_sync(bar_no);
        started = true;
        if (!ok) break;
        if (P.schedule != SCHED_RANDOM_PERM) {
            const int i0 = (int)col_off[colour], i1 = (int)col_off[colour + 1];
            for (int i = i0 + wib; i < i1; i += nwarps) visit(slots + (size_t)i * SB, np0, nf);
        } else {
            for (int i = wib; i < nslot; i += nwarps) {
                uint8_t *sl = slots + (size_t)i * SB;
                const uint32_t *meta = reinterpret_cast<const uint32_t *>(sl + OFF_META);
                const uint32_t d = meta[META_D];
                const uint8_t *rt = tables + (size_t)meta[META_RT] * RT_BYTES;
                const int Dx = *reinterpret_cast<const int32_t *>(rt + RT_DX);
                const int c = (int)((d % (uint32_t)Dx) & 1u) | (int)(((d / (uint32_t)Dx) & 1u) << 1);
                if (perm_colour(*reinterpret_cast<const uint64_t *>(rt + RT_SEED), n, p) != c) continue;
                visit(sl, np0, 1);
            }
        }
        gp += (uint64_t)nf;
        // endpoint observation after a completed schedule (Sec. 2.3)
        if (gp % nph == 0) {
            const int64_t nl_done = (int64_t)(gp / nph - (uint64_t)P.sched_begin);
            if (P.obs_every > 0 && P.obs_acc != nullptr && nl_done > 0 && (nl_done % P.obs_every) == 0) {
                ok = phase_sync(bar_no);
                if (!ok) break;
                const int64_t o = nl_done / P.obs_every - 1;
                const int64_t visits = P.visits_before + nl_done * (nph == 8 ? 2 : 1);
                for (int i = wib; i < nslot; i += nwarps) {
                    const uint8_t *sl = slots + (size_t)i * SB;
                    const uint32_t *meta = reinterpret_cast<const uint32_t *>(sl + OFF_META);
                    uint64_t hN, hS, hW, hE;
                    read_halo(meta, hN, hS, hW, hE);
                    row_t S[G::RPL];
                    const mem_t *trow = reinterpret_cast<const mem_t *>(sl);
#pragma unroll
                    for (int t = 0; t < G::RPL; ++t) S[t] = (lane < G::NACT) ? (row_t)trow[lane * G::RPL + t] : (row_t)0;
                    int bonds, mag;
                    domain_bonds_mag<LD>(S, hE, hS, lane, bonds, mag);
                    if (lane == 0) {
                        const uint64_t *ctr = reinterpret_cast<const uint64_t *>(sl + OFF_CTR);
                        const double tdom = domain_time(EXPO, ctr[DCTR_CLKM], (int64_t)ctr[DCTR_CLKE],
                                                        visits * (int64_t)P.k, P.lambda);
                        unsigned long long *acc = P.obs_acc + ((size_t)o * P.n_rep + meta[META_R]) * OBS_WORDS;
                        atomicAdd(&acc[0], (unsigned long long)(long long)bonds);
                        atomicAdd(&acc[1], (unsigned long long)(long long)mag);
                        atomicAdd(reinterpret_cast<double *>(&acc[2]), tdom);
                        atomicAdd(reinterpret_cast<double *>(&acc[3]), reinterpret_cast<const double *>(ctr)[DCTR_SB]);
                        atomicAdd(reinterpret_cast<double *>(&acc[4]), reinterpret_cast<const double *>(ctr)[DCTR_SH]);
                    }
                }
            }
        }
    }
    if (CLUSTER) {
        // no CTA may leave while another still reads its shared memory
        cluster_sync();
    } else if (!ok) {
        return;
    }
    // write owned tiles and counters back (and edges, for the observables kernel)
    for (int i = wib; i < nslot; i += nwarps) {
        const uint8_t *sl = slots + (size_t)i * SB;
        const uint32_t g = reinterpret_cast<const uint32_t *>(sl + OFF_META)[META_G];
        for (int q = lane * 4; q < TB; q += 128)
            *reinterpret_cast<uint32_t *>(P.tiles + (size_t)g * TB + q) = *reinterpret_cast<const uint32_t *>(sl + q);
        if (lane < DCTR_WORDS)
            P.dctr[(size_t)g * DCTR_WORDS + lane] = reinterpret_cast<const uint64_t *>(sl + OFF_CTR)[lane];
        if (CLUSTER && lane < 4)
            P.edges[(size_t)g * 4 + lane] = reinterpret_cast<const uint64_t *>(sl + OFF_EDGE)[lane];
    }
}

// ---------------------------------------------------------------------------
// Set-up kernels.
// ---------------------------------------------------------------------------
struct LayoutParams {
    int n_rep;
    int n_dom;
    const int32_t *rep_L;
    const int32_t *rep_Dx;
    const uint32_t *rep_dom_off;
    const uint64_t *rep_site_off;
    const uint64_t *rep_blk_off; // prefix of L^2/128 init blocks, n_rep+1 entries
    const uint64_t *rep_seed;
    const uint32_t *dom_rep;
    int8_t *spins;
    uint8_t *tiles;
    uint64_t *edges;
    uint64_t *dctr;
    int *err;
};

// iid +-1 from Philox (block b of 128 sites: counter {b_lo, b_hi, 0, TAG_INIT<<24}) or all up.
__global__ void init_spins_kernel(const LayoutParams P, int init)
{
    const uint64_t total = P.rep_blk_off[P.n_rep];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = P.n_rep - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.rep_blk_off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int r = lo;
        const uint64_t b = t - P.rep_blk_off[r];
        uint4 w = make_uint4(~0u, ~0u, ~0u, ~0u);
        if (init == 0) {
            const uint64_t seed = P.rep_seed[r];
            w = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(b >> 32), 0u, TAG_INIT << 24),
                              make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        }
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
        uint64_t *out = reinterpret_cast<uint64_t *>(P.spins + P.rep_site_off[r] + b * 128);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const uint32_t byte = (words[q >> 2] >> (8 * (q & 3))) & 0xFFu;
            uint64_t v = ((uint64_t)byte * 0x0101010101010101ull) & 0x8040201008040201ull;
            v = ((v + 0x7F7F7F7F7F7F7F7Full) >> 7) & 0x0101010101010101ull;
            out[q] = ~0ull ^ (v * 0xFEull);
        }
    }
}

// int8 spins -> bit tiles + edges; one warp per domain; bytes must be +-1.
template <int LD>
__global__ void pack_kernel(const LayoutParams P)
{
    using G = Geo<LD>;
    using row_t = typename G::row_t;
    using mem_t = typename G::mem_t;
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int g = wg; g < P.n_dom; g += nw) {
        const uint32_t r = P.dom_rep[g];
        const int L = P.rep_L[r], Dx = P.rep_Dx[r];
        const uint32_t d = (uint32_t)g - P.rep_dom_off[r];
        const int bx = (int)(d % (uint32_t)Dx), by = (int)(d / (uint32_t)Dx);
        row_t S[G::RPL];
        bool bad = false;
#pragma unroll
        for (int t = 0; t < G::RPL; ++t) {
            S[t] = 0;
            if (lane < G::NACT) {
                const int y = lane * G::RPL + t;
                const uint64_t *src = reinterpret_cast<const uint64_t *>(
                    P.spins + P.rep_site_off[r] + (uint64_t)(by * LD + y) * L + (uint64_t)bx * LD);
                uint64_t row = 0;
#pragma unroll
                for (int q = 0; q < LD / 8; ++q) {
                    const uint64_t x = src[q];
                    const uint64_t neg = (x >> 7) & 0x0101010101010101ull;
                    bad |= (x != (0x0101010101010101ull | (neg * 0xFEull)));
                    const uint64_t up = (~x >> 7) & 0x0101010101010101ull;
                    row |= ((up * 0x0102040810204080ull) >> 56) << (8 * q);
                }
                S[t] = (row_t)row;
            }
        }
        if (__any_sync(FULL_WARP, bad) && lane == 0) atomicCAS(P.err, 0, ERR_SPIN);
        mem_t *trow = reinterpret_cast<mem_t *>(P.tiles + (uint64_t)g * G::TILE_BYTES);
        if (lane < G::NACT) {
#pragma unroll
            for (int t = 0; t < G::RPL; ++t) trow[lane * G::RPL + t] = (mem_t)S[t];
        }
        const uint64_t ew = edge_words<LD>(S, lane);
        if (lane < 4) P.edges[(uint64_t)g * 4 + lane] = ew;
    }
}

// bit tiles -> int8 spins; one warp per domain.
template <int LD>
__global__ void unpack_kernel(const LayoutParams P)
{
    using G = Geo<LD>;
    using mem_t = typename G::mem_t;
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int g = wg; g < P.n_dom; g += nw) {
        const uint32_t r = P.dom_rep[g];
        const int L = P.rep_L[r], Dx = P.rep_Dx[r];
        const uint32_t d = (uint32_t)g - P.rep_dom_off[r];
        const int bx = (int)(d % (uint32_t)Dx), by = (int)(d / (uint32_t)Dx);
        const mem_t *trow = reinterpret_cast<const mem_t *>(P.tiles + (uint64_t)g * G::TILE_BYTES);
        if (lane < G::NACT) {
#pragma unroll
            for (int t = 0; t < G::RPL; ++t) {
                const int y = lane * G::RPL + t;
                const uint64_t row = (uint64_t)trow[y];
                uint64_t *dst = reinterpret_cast<uint64_t *>(
                    P.spins + P.rep_site_off[r] + (uint64_t)(by * LD + y) * L + (uint64_t)bx * LD);
#pragma unroll
                for (int q = 0; q < LD / 8; ++q) {
                    const uint64_t byte = (row >> (8 * q)) & 0xFFull;
                    uint64_t v = (byte * 0x0101010101010101ull) & 0x8040201008040201ull;
                    v = ((v + 0x7F7F7F7F7F7F7F7Full) >> 7) & 0x0101010101010101ull;
                    dst[q] = ~0ull ^ (v * 0xFEull);
                }
            }
        }
    }
}

// Observables of the current state from the global tiles and edges (kmc_observables).
template <int LD, bool EXPO>
__global__ void observe_kernel(const RunParams P, const uint32_t *dom_rep, int n_dom, int64_t visits,
                               unsigned long long *acc /* [n_rep][OBS_WORDS] */)
{
    using G = Geo<LD>;
    using row_t = typename G::row_t;
    using mem_t = typename G::mem_t;
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int g = wg; g < n_dom; g += nw) {
        const uint32_t r = dom_rep[g];
        const int Dx = P.rep_Dx[r];
        const uint32_t d = (uint32_t)g - P.rep_dom_off[r];
        const int bx = (int)(d % (uint32_t)Dx), by = (int)(d / (uint32_t)Dx);
        const uint64_t gbase = (uint64_t)g - d;
        const uint64_t hS = P.edges[(gbase + (uint32_t)(((by + 1) % Dx) * Dx + bx)) * 4 + EDGE_N];
        const uint64_t hE = P.edges[(gbase + (uint32_t)(by * Dx + (bx + 1) % Dx)) * 4 + EDGE_W];
        row_t S[G::RPL];
        const mem_t *trow = reinterpret_cast<const mem_t *>(P.tiles + (uint64_t)g * G::TILE_BYTES);
#pragma unroll
        for (int t = 0; t < G::RPL; ++t) S[t] = (lane < G::NACT) ? (row_t)trow[lane * G::RPL + t] : (row_t)0;
        int bonds, mag;
        domain_bonds_mag<LD>(S, hE, hS, lane, bonds, mag);
        if (lane == 0) {
            const uint64_t *ctr = P.dctr + (uint64_t)g * DCTR_WORDS;
            const double t = domain_time(EXPO, ctr[DCTR_CLKM], (int64_t)ctr[DCTR_CLKE], visits * (int64_t)P.k,
                                         P.lambda);
            unsigned long long *a = acc + (size_t)r * OBS_WORDS;
            atomicAdd(&a[0], (unsigned long long)(long long)bonds);
            atomicAdd(&a[1], (unsigned long long)(long long)mag);
            atomicAdd(reinterpret_cast<double *>(&a[2]), t);
            atomicAdd(reinterpret_cast<double *>(&a[3]), __longlong_as_double((long long)ctr[DCTR_SB]));
            atomicAdd(reinterpret_cast<double *>(&a[4]), __longlong_as_double((long long)ctr[DCTR_SH]));
        }
    }
}

// obs_acc -> {e, m, e*m, T (, score beta, score h)} per record; same FP order as the oracle.
__global__ void finalize_obs_kernel(const unsigned long long *acc, int n_rec, int n_rep,
                                    const int32_t *rep_L, const int32_t *rep_Dx, double J,
                                    const double *rep_h, double *out, int stride)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rec) return;
    const int r = i % n_rep;
    const unsigned long long *a = acc + (size_t)i * OBS_WORDS;
    const double N = (double)rep_L[r] * (double)rep_L[r];
    const double b = (double)(long long)a[0];
    const double m = (double)(long long)a[1];
    const double e = __ddiv_rn(__dsub_rn(__dmul_rn(-J, b), __dmul_rn(rep_h[r], m)), N);
    const double mm = __ddiv_rn(m, N);
    const double nD = (double)rep_Dx[r] * (double)rep_Dx[r];
    double *o = out + (size_t)i * stride;
    o[0] = e;
    o[1] = mm;
    o[2] = __dmul_rn(e, mm);
    o[3] = __ddiv_rn(__longlong_as_double((long long)a[2]), nD);
    if (stride >= 6) {
        o[4] = __longlong_as_double((long long)a[3]);
        o[5] = __longlong_as_double((long long)a[4]);
    }
}

// per-domain counters -> host-facing arrays (hash, flips, clock)
template <bool EXPO>
__global__ void domain_state_kernel(const uint64_t *dctr, int n_dom, int64_t steps, double lambda,
                                    uint64_t *hash, int64_t *flips, double *t)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_dom) return;
    const uint64_t *c = dctr + (uint64_t)g * DCTR_WORDS;
    hash[g] = c[DCTR_HASH];
    flips[g] = (int64_t)c[DCTR_FLIPS];
    t[g] = domain_time(EXPO, c[DCTR_CLKM], (int64_t)c[DCTR_CLKE], steps, lambda);
}

// zero counters: hash basis, flips 0, clock 1.0 (m = 2^63, e = 0), scores 0
__global__ void reset_counters_kernel(uint64_t *dctr, int n_dom)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_dom) return;
    uint64_t *c = dctr + (uint64_t)g * DCTR_WORDS;
    c[DCTR_HASH] = HASH_BASIS;
    c[DCTR_FLIPS] = 0;
    c[DCTR_CLKM] = 1ull << 63;
    c[DCTR_CLKE] = 0;
    c[DCTR_SB] = 0;
    c[DCTR_SH] = 0;
}

// per-replica score sums in fixed domain order (kmc_grad)
__global__ void score_reduce_kernel(const uint64_t *dctr, const uint32_t *rep_dom_off, int n_rep,
                                    double *score, int reset, uint64_t *dctr_w)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rep) return;
    double sb = 0.0, sh = 0.0;
    for (uint32_t g = rep_dom_off[r]; g < rep_dom_off[r + 1]; ++g) {
        sb += __longlong_as_double((long long)dctr[(uint64_t)g * DCTR_WORDS + DCTR_SB]);
        sh += __longlong_as_double((long long)dctr[(uint64_t)g * DCTR_WORDS + DCTR_SH]);
        if (reset) {
            dctr_w[(uint64_t)g * DCTR_WORDS + DCTR_SB] = 0;
            dctr_w[(uint64_t)g * DCTR_WORDS + DCTR_SH] = 0;
        }
    }
    score[2 * r] = sb;
    score[2 * r + 1] = sh;
}

} // namespace kmcdev
