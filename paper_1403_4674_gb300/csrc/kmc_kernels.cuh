// kmc_kernels.cuh -- sm_103a device code of the sequential-update parallel
// kinetic Monte Carlo (Nilmeier & Marian, arXiv:1403.4674).
//
// Data layout (device memory, between launches):
//   * caller spins: int8, replicas concatenated, row-major.
//   * bit tiles: replica r, domain d = by*Dx + bx owns LD*LD bits, row y of
//     the domain at bits [y*LD, (y+1)*LD) of the tile, bit x = column x,
//     1 = spin up.  Tile bytes = LD*LD/8.  Global domain id g = dom_off[r] + d.
//   * edges[g*8 + ...]: the domain's first row, last row, first column and
//     last column (N, S, W, E) as bit masks, each split into 32-bit halves
//     and stamped with the number of visits the domain has completed in the
//     current launch: word 2e+h = count << 32 | half h of edge e.  Column bit
//     of row y is (y % RPL)*32 + y / RPL (RPL = rows per lane, 2 for LD = 64,
//     else 1).  A neighbour reads its halo and checks that it is current with
//     the same 64-bit loads.
//   * per-domain counters dctr[g*7 + ...]: event hash, real flips, clock
//     mantissa, clock exponent, score d/dbeta, score d/dh, steps.
//
// The run kernel is persistent: every CTA owns a fixed set of domains (its
// "slots") for the whole launch; their tiles, edges, counters and the rate
// tables of their replicas live in shared memory.  The only communication
// between domains is the frozen halo (Sec. 2.2) -- the four edge words of
// each neighbour, stamped with the neighbour's visit count, so a visit starts
// as soon as its neighbours have finished their visits of earlier colour
// phases (no barrier per phase, no barrier at observation points):
//   * CLUSTER mode: every replica is resident in one thread-block cluster
//     (1..16 CTAs); halos are read from the owner CTA through distributed
//     shared memory;
//   * GRID mode (a replica larger than a cluster can hold): one cooperative
//     grid; halos go through L2.
// Observation records are sums of per-visit changes (bond sum, magnetisation,
// clock, scores) added to the state before the launch.
#pragma once

#include <cstdint>
#include <type_traits>

namespace kmcdev {

constexpr uint32_t FULL_WARP = 0xffffffffu;
constexpr int EDGE_N = 0, EDGE_S = 1, EDGE_W = 2, EDGE_E = 3;
constexpr int DCTR_HASH = 0, DCTR_FLIPS = 1, DCTR_CLKM = 2, DCTR_CLKE = 3,
              DCTR_SB = 4, DCTR_SH = 5, DCTR_STEPS = 6, DCTR_WORDS = 7;
constexpr uint64_t HASH_BASIS = 0xcbf29ce484222325ull; // FNV-1a 64 offset basis
constexpr uint64_t HASH_PRIME = 0x00000100000001b3ull; // FNV-1a 64 prime
constexpr uint32_t TAG_INIT = 1u, TAG_PERM = 2u, TAG_HORIZON = 3u; // step draws use tag 0
constexpr int HORIZON_MAX_STEPS = 1024; // table length limit of the fixed-time visit
constexpr int ERR_TIMEOUT = 1, ERR_SPIN = 2, ERR_INTERNAL = 3;
constexpr int SCHED_PALINDROME = 0, SCHED_FIXED = 1, SCHED_RANDOM_PERM = 2;
constexpr int INIT_KEEP = 2, INIT_PER_REPLICA = 3;
constexpr int OBS_WORDS = 5; // bonds, mag, clock sum, score beta sum, score h sum

// Replica table staged in shared memory (bytes):
//   [0,128) A[16] fixed-point acceptance,
//   [128,256) Gb[16] = X_c = round(a dlog a/dbeta 2^Q) (int64, scores),
//   [256,512) grad[32] = a[10], dlog a/dbeta[10], dlog a/dh[10],
//   [512] seed, [520] dom_off, [524] Dx, [528] k (steps per visit),
//   [544,624) Gh[10] = X_c of dlog a/dh, [624] 2^-(Q+4) (double),
//   [640,680) Yb[10], [680,720) Yh[10]: the low words Y_c = round((a dlog a
//   2^Q - X_c) 2^GFIX_LO_BITS) (int32), so that X_c 2^-Q + Y_c 2^-(Q+18)
//   holds a dlog a to 2^-(Q+19).
constexpr int RT_BYTES = 720;
constexpr int RT_SEED = 512, RT_DOMOFF = 520, RT_DX = 524, RT_K = 528, RT_GB = 128, RT_GH = 544, RT_GSCALE = 624,
              RT_YB = 640, RT_YH = 680;
// per replica: Xb[10], Xh[10], 2^-(Q+4) bits, pad, Yb[10] and Yh[10] as
// int32 pairs in words 22..26 and 27..31
constexpr int GFIX_WORDS = 32, GFIX_YB = 22, GFIX_YH = 27;
constexpr int GFIX_LO_BITS = 18; // fraction bits of the low word beyond 2^-Q
constexpr int GFIX_T_BITS = 4;   // fraction bits of the combined per-state sum beyond 2^-Q
// Slot: [tile][stamped edges 64][counters 56][meta 32][observation 48];
// meta u32: g, replica, d, rt, nb[4];
// observation, since the record began: u32 record, i32 bond change, i32
// magnetisation change, u32 steps (EXPECTED clock), u64 mantissa and i64
// exponent of the product of clock variates (EXPONENTIAL clock), f64 score
// changes d/dbeta, d/dh.
constexpr int SLOT_EXTRA = 64 + 56 + 32 + 48;
constexpr uint32_t NO_RECORD = 0xFFFFFFFFu;
constexpr int EDGE_WORDS = 8; // stamped 64-bit words per domain

__host__ __device__ constexpr uint64_t stamp(uint32_t count, uint32_t half)
{
    return ((uint64_t)count << 32) | half;
}
constexpr int META_G = 0, META_R = 1, META_D = 2, META_RT = 3, META_NB = 4;

template <int LD> __host__ __device__ constexpr int slot_bytes() { return ((LD * LD / 8 + SLOT_EXTRA) + 15) / 16 * 16; }

struct RunParams {
    int n_rep;
    int schedule;
    int obs_every;
    int64_t sched_begin;
    int64_t n_sched;
    int64_t visits_before; // per-domain visits before this launch (clock mode EXPECTED)
    // per replica (global)
    const int32_t *rep_Dx;
    const int32_t *rep_k;    // steps per domain visit
    const uint32_t *rep_dom_off;
    const uint64_t *rep_seed;
    const uint64_t *rep_A;   // [n_rep][16]
    const int64_t *rep_gfix; // [n_rep][GFIX_WORDS]
    const double *rep_grad;  // [n_rep][32]
    // plan: per CTA slot ranges (colour-sorted), replica tables, neighbours
    const uint32_t *cta_slot_off; // [n_cta + 1]
    const uint32_t *cta_col_off;  // [n_cta][5], relative to the CTA's first slot
    const uint32_t *cta_rt_off;   // [n_cta + 1]
    const uint32_t *rt_rep;       // replica id of each staged table
    const uint32_t *slot_g;       // global domain id of each slot
    const uint32_t *slot_rt;      // local table index of each slot
    const uint32_t *slot_nb;      // [n_slots][4]: CLUSTER: rank << 24 | local slot; GRID: neighbour g, or
                                  // 1 << 31 | local slot when the neighbour is in the same CTA
    int max_rt;                   // table capacity per CTA (uniform layout)
    int cluster;                  // 0 = GRID mode, else cluster size
    // state
    uint8_t *tiles;
    uint64_t *dctr;
    uint64_t *edges;
    // observables scratch [n_obs][n_rep][OBS_WORDS]: schedule mode holds the
    // records, pass mode the per-record changes (bonds, mag, clock, scores)
    unsigned long long *obs_acc;
    int obs_pass;   // 1: a record after every obs_every-th colour pass
    int64_t n_obs;  // records of this launch
    // fixed-time visits: K ~ Poisson(n_d nu dtau) steps by table inversion
    int horizon;
    int hkmax;
    const uint64_t *htab; // [hkmax] floor(F(k) 2^64) of the Poisson CDF
    double dtau;
    int *err;
    uint64_t bar_limit_ns;
    int debug_extra;
    double lambda; // n_d * nu
    // profiling: total over warps of the halo-poll iterations each warp ran
    // beyond the first read (null: not counted)
    unsigned long long *polls;
    // thread-per-domain plans: domain -> replica, and each domain's open
    // observation record
    const uint32_t *dom_rep;
    uint64_t *obs_dom;
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
    asm volatile("ld.volatile.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_volatile_shared(uint32_t addr)
{
    uint64_t v;
    asm volatile("ld.volatile.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_volatile_global(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
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

// 64-bit unsigned integer to FP32, rounded toward zero / upwards, from two
// 32-bit conversions (exact scaling by 2^32, one directed addition).
__device__ __forceinline__ float u64_to_float_rz(uint64_t x)
{
    return __fadd_rz(__fmul_rz(__uint2float_rz((uint32_t)(x >> 32)), 4294967296.0f), __uint2float_rz((uint32_t)x));
}
__device__ __forceinline__ float u64_to_float_ru(uint64_t x)
{
    return __fadd_ru(__fmul_ru(__uint2float_ru((uint32_t)(x >> 32)), 4294967296.0f), __uint2float_ru((uint32_t)x));
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

__device__ __forceinline__ void mant_mul32(uint64_t &m, int &e, uint64_t m2, int e2)
{
    const uint64_t hi = __umul64hi(m, m2);
    const uint64_t lo = m * m2;
    const bool top = (hi >> 63) != 0;
    m = top ? hi : ((hi << 1) | (lo >> 63));
    e = e + e2 + (top ? 1 : 0);
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

    // Bit-sliced +1 / -1 of the up-neighbour count of the sites in mask m of
    // row t (the count stays within 0..4).
    __device__ __forceinline__ void inc(int t, row_t m)
    {
        const row_t c0 = b0[t] & m;
        b0[t] ^= m;
        const row_t c1 = b1[t] & c0;
        b1[t] ^= c0;
        b2[t] ^= c1;
    }
    __device__ __forceinline__ void dec(int t, row_t m)
    {
        const row_t d0 = (row_t)~b0[t] & m;
        b0[t] ^= m;
        const row_t d1 = (row_t)~b1[t] & d0;
        b1[t] ^= d0;
        b2[t] ^= d1;
    }

    // Counts from the domain's own spins only (halo taken as down); the halo
    // is added by add_halo once it has arrived, so a warp builds this part
    // while it waits for its neighbours.
    __device__ __forceinline__ void build_interior(int lane) { build(lane, (row_t)0, (row_t)0, 0ull, 0ull); }

    // Add the frozen halo's up spins: the N row to row 0, the S row to row
    // LD-1, the W and E columns to columns 0 and LD-1 (a corner site takes two
    // halo neighbours, hence two additions).
    __device__ __forceinline__ void add_halo(int lane, row_t hN, row_t hS, uint64_t hW, uint64_t hE)
    {
#pragma unroll
        for (int t = 0; t < G::RPL; ++t) {
            const int y = lane * G::RPL + t;
            const int cb = (y % G::RPL) * 32 + y / G::RPL;
            const row_t mrow = (y == 0) ? hN : ((y == LD - 1) ? hS : (row_t)0);
            const row_t mcol = (row_t)((hW >> cb) & 1ull) | (row_t)(((hE >> cb) & 1ull) << (LD - 1));
            inc(t, mrow);
            inc(t, mcol);
        }
    }

    // After the spin at (y, col) flipped: its in-domain neighbours (row y at
    // col-1 and col+1, rows y-1 and y+1 at col) gain an up neighbour if the
    // spin is now up, else lose one.  Bit-sliced +-1 on the count planes;
    // halo neighbours are outside the domain and unchanged.
    __device__ __forceinline__ void flip_update(int lane, int y, int col, bool now_up)
    {
        const row_t bitc = (row_t)1 << col;
        const row_t mh = (row_t)(((col > 0) ? (bitc >> 1) : (row_t)0) | ((col < LD - 1) ? (bitc << 1) : (row_t)0));
#pragma unroll
        for (int t = 0; t < G::RPL; ++t) {
            const int yy = lane * G::RPL + t;
            const row_t m = (yy == y) ? mh : ((yy == y - 1 || (yy == y + 1 && yy < LD)) ? bitc : (row_t)0);
            if (now_up) inc(t, m);
            else dec(t, m);
        }
    }

    // Sites of one class in row t.  The class c = 5*up + q is given as masks:
    // UP all ones for up spins, Q2/Q1/Q0 all ones where the bit of q is set.
    __device__ __forceinline__ row_t mask_q(int t, row_t UP, row_t Q2, row_t Q1, row_t Q0) const
    {
        const row_t diff = (b2[t] ^ Q2) | (b1[t] ^ Q1) | (b0[t] ^ Q0); // up-neighbour count != q
        return (S[t] ^ (row_t)~UP) & (row_t)~diff & valid;
    }
};

// Class counts of the warp's domain: lane c (< 10) receives n_c.  Per lane,
// class q (down spin) is counted in the low and class q+5 (up spin) in the
// high half-word, so five warp reductions cover the ten classes.
template <int LD>
__device__ __forceinline__ uint32_t class_counts(const Planes<LD> &P, int lane)
{
    using row_t = typename Geo<LD>::row_t;
    uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0;
#pragma unroll
    for (int t = 0; t < Geo<LD>::RPL; ++t) {
        const row_t b2 = P.b2[t], b1 = P.b1[t], b0 = P.b0[t];
        const row_t up = P.S[t], dn = (row_t)~P.S[t] & P.valid;
        const row_t n2 = (row_t)~b2;
        const row_t e0 = n2 & (row_t)~b1 & (row_t)~b0, e1 = n2 & (row_t)~b1 & b0;
        const row_t e2 = n2 & b1 & (row_t)~b0, e3 = n2 & b1 & b0, e4 = b2;
        w0 += (uint32_t)popc_row(dn & e0) | ((uint32_t)popc_row(up & e0) << 16);
        w1 += (uint32_t)popc_row(dn & e1) | ((uint32_t)popc_row(up & e1) << 16);
        w2 += (uint32_t)popc_row(dn & e2) | ((uint32_t)popc_row(up & e2) << 16);
        w3 += (uint32_t)popc_row(dn & e3) | ((uint32_t)popc_row(up & e3) << 16);
        w4 += (uint32_t)popc_row(dn & e4) | ((uint32_t)popc_row(up & e4) << 16);
    }
    const uint32_t t0 = __reduce_add_sync(FULL_WARP, w0), t1 = __reduce_add_sync(FULL_WARP, w1);
    const uint32_t t2 = __reduce_add_sync(FULL_WARP, w2), t3 = __reduce_add_sync(FULL_WARP, w3);
    const uint32_t t4 = __reduce_add_sync(FULL_WARP, w4);
    const int q = (lane < 5) ? lane : lane - 5;
    const uint32_t tw = (q == 0) ? t0 : (q == 1) ? t1 : (q == 2) ? t2 : (q == 3) ? t3 : t4;
    const uint32_t n = (lane < 5) ? (tw & 0xFFFFu) : (tw >> 16);
    return (lane < 10) ? n : 0u;
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

// Sum over lanes 0..15 (every lane receives it).
__device__ __forceinline__ int64_t warp_isum16(int64_t v)
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
    // this visit only: change of the bond sum and of the magnetisation, and
    // the product of its clock variates (mantissa vM, exponent vE)
    int dbonds, dmag;
    uint64_t vM;
    int64_t vE;
};

// ---------------------------------------------------------------------------
// The random numbers of 32 consecutive steps of a visit (lane i: step base+i)
// and the product of their clock variates.  They depend only on the replica
// seed, the domain and the counters, so a warp draws the first chunk of a
// visit before it waits for the halo.
// ---------------------------------------------------------------------------
struct Chunk {
    uint64_t tgt;   // step target, ~0 past the visit's last step
    uint64_t ebase; // np << 32 | j << 16: the step's event word without the site
    uint64_t m;     // clock: product of the chunk's variates, mantissa in [2^63, 2^64)
    int e;          // and its binary exponent (warp-uniform)
};

template <bool EXPO>
__device__ __forceinline__ Chunk draw_chunk(uint2 key, uint32_t d, uint64_t np0, int base, int total, int k,
                                            int lane)
{
    Chunk ch;
    const int s = base + lane;
    ch.tgt = ~0ull;
    ch.ebase = 0;
    uint64_t V = 1ull << 53;
    if (s < total) {
        const int f = s / k;
        const int j = s - f * k;
        const uint64_t np = np0 + (uint64_t)f;
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)j, d, (uint32_t)np, (uint32_t)(np >> 32) & 0xFFFFFFu), key);
        ch.tgt = (((uint64_t)w.y << 32) | w.x) >> 1;
        V = ((((uint64_t)w.w << 32) | w.z) >> 11) + 1ull;
        ch.ebase = (np << 32) | ((uint64_t)j << 16); // site bits added on a flip
    }
    ch.m = 1ull << 63;
    ch.e = 0;
    if (EXPO) {
        // product of this chunk's variates: butterfly over the smallest power of
        // two covering the chunk (lanes past its end hold v = 1)
        const int chunk_end = min(32, total - base);
        const int z = __clzll((long long)V);
        uint64_t m = V << z;
        int e = 10 - z;
        for (int off = 1; off < chunk_end; off <<= 1) {
            const uint64_t m2 = __shfl_xor_sync(FULL_WARP, m, off);
            const int e2 = __shfl_xor_sync(FULL_WARP, e, off);
            mant_mul32(m, e, m2, e2);
        }
        ch.m = __shfl_sync(FULL_WARP, m, 0);
        ch.e = __shfl_sync(FULL_WARP, e, 0);
    }
    return ch;
}

// Steps of a fixed-time visit (domain time dtau): the number of uniformised
// events in that time is Poisson(n_d nu dtau) (Sec. 2.1), drawn by inversion
// with the uniform U = w0 | w1 << 32 of Philox {0, d, np_lo, np_hi |
// TAG_HORIZON << 24}: K = the first k with U < tab[k] = floor(F(k) 2^64), or
// kmax.  Two rounds of 32 parallel comparisons: the last threshold of every
// block of 32, then the thresholds of the first block whose last one exceeds U.
__device__ __forceinline__ int horizon_steps(uint2 key, uint32_t d, uint64_t np, const uint64_t *tab, int kmax,
                                             int lane)
{
    const uint4 w = philox4x32_10(
        make_uint4(0u, d, (uint32_t)np, ((uint32_t)(np >> 32) & 0xFFFFFFu) | (TAG_HORIZON << 24)), key);
    const uint64_t U = ((uint64_t)w.y << 32) | w.x;
    const int nblk = (kmax + 31) / 32; // <= 32: kmax <= HORIZON_MAX_STEPS
    const int last = min(32 * lane + 31, kmax - 1);
    const unsigned mb = __ballot_sync(FULL_WARP, lane < nblk && U < __ldg(&tab[lane < nblk ? last : 0]));
    if (!mb) return kmax;
    const int b = __ffs(mb) - 1;
    const int i = 32 * b + lane;
    const unsigned mk = __ballot_sync(FULL_WARP, i < kmax && U < __ldg(&tab[i < kmax ? i : 0]));
    return 32 * b + __ffs(mk) - 1;
}

// Lane c (< 10) holds class c's fixed-point rate, loaded before the halo
// wait; the score constants stay in the replica table in shared memory
// (rt) and are read where a state or an event needs them.
struct RateRegs {
    uint64_t A;
    const uint8_t *rt;
};

template <bool GRAD>
__device__ __forceinline__ RateRegs load_rates(const uint8_t *rt, int lane)
{
    RateRegs r = {0ull, rt};
    if (lane < 10) r.A = reinterpret_cast<const uint64_t *>(rt)[lane];
    return r;
}

// ---------------------------------------------------------------------------
// One domain visit (Sec. 2.2): `total` uniformised steps with the halo
// hN/hS/hW/hE frozen -- k steps in each of nfused consecutive global phases
// of the same colour, or a Poisson number for a fixed-time visit.
//
// Step j of global phase np draws Philox {j, d, np_lo, np_hi} with the replica
// seed: target = (w0 | w1<<32) >> 1 uniform on [0, n_d 2^P), V = (w2 | w3<<32)
// >> 11 plus 1.  target >= R' = sum_c n_c A_c is a null step (the diagonal of
// App. A Eq. Glauber_TM); otherwise class c = first class whose inclusive
// cumulative rate exceeds target, member jj = (target - C_{c-1}) / A_c in
// row-major order flips (the n-fold way's cumulative selection, Sec. 2.1).
// Steps are drawn 32 at a time (lane i draws step base+i); runs of null steps
// are skipped with one ballot since the state does not change between real
// events.  rr: the replica's rates, held by lanes 0..9.
// ---------------------------------------------------------------------------
// 0, 1, ..., 32 as FP64: the length of a run of null steps without an
// integer-to-FP64 conversion (FP64 is this GPU's slowest pipe)
__constant__ double kRunLength[33] = {0,  1,  2,  3,  4,  5,  6,  7,  8,  9,  10, 11, 12, 13, 14, 15, 16,
                                      17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32};

template <int LD, bool EXPO, bool GRAD>
__device__ __forceinline__ void visit_core(Planes<LD> &pl, Counters &cn, const RateRegs &rr, uint2 key,
                                           typename Geo<LD>::row_t hN, typename Geo<LD>::row_t hS,
                                           uint64_t hW, uint64_t hE, uint32_t d, uint64_t np0,
                                           int k, int lane, int *err, const Chunk &first, int total)
{
    using G = Geo<LD>;
    using row_t = typename G::row_t;
    const uint64_t Ac = rr.A;
    // 1/A_c from below (A_c rounded up, its reciprocal rounded down), so that
    // the FP32 quotient estimate below never exceeds the exact quotient.  The
    // 64-bit integers are converted in two 32-bit halves (the 64-bit integer
    // conversion runs on the FP64 unit).
    const float invAf = (lane < 10) ? __frcp_rd(u64_to_float_ru(Ac)) : 0.0f;
    pl.add_halo(lane, hN, hS, hW, hE); // pl holds the interior counts
    uint32_t n_c = class_counts<LD>(pl, lane);
    uint64_t Wc = (uint64_t)n_c * Ac;
    uint64_t Cinc = prefix16(Wc, lane);
    uint64_t R = __shfl_sync(FULL_WARP, Cinc, 9);

    // Score of a null step in the current state: d log(1 - R/n_d) =
    // -sum_c n_c a_c dlog a_c / (n_d - R).  The numerator is an exact
    // integer sum of the two fixed-point words of a_c dlog a_c (high word
    // X_c at 2^-Q, low word Y_c at 2^-(Q+18)), rounded once per state to
    // 2^-(Q+4); n_d - R comes from the exact fixed-point rate sum,
    // (n_d 2^P - R') 2^-P with n_d 2^P = 2^63.  A single fixed-point word
    // would round every class product the same way in every state, a bias
    // that grows linearly over a run's millions of null-step states; with the
    // low word the per-class error is 2^-(Q+19) and what remains are FP64
    // roundings that change from state to state.  One reciprocal per state,
    // formed only for states that have null steps (a real event that
    // directly follows another needs none): FP64 is this GPU's slowest pipe.
    double nb_over = 0.0, nh_over = 0.0;
    bool state_scored = false; // nb_over / nh_over belong to the current state (warp-uniform)
    constexpr int PBITS = 63 - 2 * (LD == 8 ? 3 : LD == 16 ? 4 : LD == 32 ? 5 : 6);
    auto grad_state = [&]() {
        if (GRAD) {
            const uint8_t *rt = rr.rt;
            const bool cl = lane < 10;
            const int64_t Xb = cl ? reinterpret_cast<const int64_t *>(rt + RT_GB)[lane] : 0;
            const int64_t Xh = cl ? reinterpret_cast<const int64_t *>(rt + RT_GH)[lane] : 0;
            const int Yb = cl ? reinterpret_cast<const int32_t *>(rt + RT_YB)[lane] : 0;
            const int Yh = cl ? reinterpret_cast<const int32_t *>(rt + RT_YH)[lane] : 0;
            // 2^-(Q+4) 2^P: a power of two, so the scaling below is exact
            const double scaleP = *reinterpret_cast<const double *>(rt + RT_GSCALE) * (double)(1ull << PBITS);
            const int64_t xb = warp_isum16((int64_t)n_c * Xb), xh = warp_isum16((int64_t)n_c * Xh);
            // |n_c Y_c| <= n_d 2^17 <= 2^29: exact in one 32-bit warp reduction
            const int yb = __reduce_add_sync(FULL_WARP, (int)n_c * Yb);
            const int yh = __reduce_add_sync(FULL_WARP, (int)n_c * Yh);
            constexpr int SH = GFIX_LO_BITS - GFIX_T_BITS;
            const int64_t tb = xb * (1ll << GFIX_T_BITS) + (int64_t)((yb + (1 << (SH - 1))) >> SH);
            const int64_t th = xh * (1ll << GFIX_T_BITS) + (int64_t)((yh + (1 << (SH - 1))) >> SH);
            const uint64_t gap = (1ull << 63) - R;
            // 2^-P / (n_d - R) = 1/gap from the FP32 reciprocal x0 = (1 - e)/g:
            // x0 (1 + e + e^2) = (1 - e^3)/g, |e| < 2^-21, so the truncation
            // error 2^-63 stays below FP64 rounding (the plain Newton-Raphson
            // step x0 (1 + e) would leave a one-sided error e^2 ~ 2^-44 in
            // every state).  Three FP64 fused multiply-adds.
            const double g = __ull2double_rn(gap);
            const double x0 = (double)__frcp_rn(u64_to_float_rz(gap));
            const double e = __fma_rn(-g, x0, 1.0);
            const double inv = gap ? __fma_rn(x0, __fma_rn(e, e, e), x0) : 0.0;
            const double w = inv * scaleP;
            nb_over = (double)tb * w;
            nh_over = (double)th * w;
            state_scored = true;
        }
    };

    for (int base = 0; base < total; base += 32) {
        const Chunk ch = (base == 0) ? first : draw_chunk<EXPO>(key, d, np0, base, total, k, lane);
        const uint64_t tgt = ch.tgt, ebase = ch.ebase;
        const int chunk_end = min(32, total - base);
        const bool last_chunk = base + 32 >= total;
        if (EXPO) {
            mant_mul(cn.clkM, cn.clkE, ch.m, (int64_t)ch.e);
            mant_mul(cn.vM, cn.vE, ch.m, (int64_t)ch.e);
        }
        int pos = 0;
        while (true) {
            const unsigned real = __ballot_sync(FULL_WARP, lane >= pos && tgt < R);
            const int jx = real ? __ffs(real) - 1 : chunk_end;
            if (GRAD && jx > pos) {
                // (jx - pos) null steps in the current state
                if (!state_scored) grad_state();
                const double q = kRunLength[jx - pos];
                cn.sb -= q * nb_over;
                cn.sh -= q * nh_over;
            }
            if (!real) break;
            const uint64_t t = __shfl_sync(FULL_WARP, tgt, jx);
            const uint64_t ev = __shfl_sync(FULL_WARP, ebase, jx);
            const unsigned sel = __ballot_sync(FULL_WARP, lane < 10 && t < Cinc);
            const int c = __ffs(sel) - 1;
            // exact jj = floor((t - C_{c-1}) / A_c) < n_c <= 4096, computed by
            // every lane for its own class (lane c's is kept).  Every FP32
            // step (x and A_c converted, reciprocal, product) rounds toward
            // the lower side, so the estimate e obeys x/A_c (1 - 2^-20) < e <= x/A_c;
            // as x/A_c < 4096, e truncates to jj or jj - 1, and one exact
            // integer comparison decides which.
            const uint64_t x = t - (Cinc - Wc);
            uint32_t q = (uint32_t)__fmul_rz(u64_to_float_rz(x), invAf);
            q = (x - (uint64_t)q * Ac >= Ac) ? q + 1u : q;
            const uint32_t jj = __shfl_sync(FULL_WARP, q, c);
            if (GRAD) {
                // dlog a_c / d(beta, h) of the chosen class (a broadcast read)
                const double *gr = reinterpret_cast<const double *>(rr.rt + 256);
                cn.sb += gr[10 + c];
                cn.sh += gr[20 + c];
            }
            // rank selection: jj-th member of class c in row-major order
            const int qc = (c >= 5) ? c - 5 : c;
            // flipping spin s with neighbour sum 2qc - 4 changes the bond sum
            // by -2 s (2qc - 4) and the magnetisation by -2 s
            const int sgn = (c >= 5) ? 1 : -1;
            cn.dbonds -= 2 * sgn * (2 * qc - 4);
            cn.dmag -= 2 * sgn;
            const row_t UP = (c >= 5) ? (row_t)~(row_t)0 : (row_t)0;
            const row_t Q2 = (qc & 4) ? (row_t)~(row_t)0 : (row_t)0;
            const row_t Q1 = (qc & 2) ? (row_t)~(row_t)0 : (row_t)0;
            const row_t Q0 = (qc & 1) ? (row_t)~(row_t)0 : (row_t)0;
            row_t m[G::RPL];
            uint32_t cl = 0;
#pragma unroll
            for (int tt = 0; tt < G::RPL; ++tt) {
                m[tt] = pl.mask_q(tt, UP, Q2, Q1, Q0);
                cl += popc_row(m[tt]);
            }
            uint32_t incl = cl;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t v = __shfl_up_sync(FULL_WARP, incl, off);
                if (lane >= off) incl += v;
            }
            const uint32_t excl = incl - cl;
            const unsigned win = __ballot_sync(FULL_WARP, jj >= excl && jj < incl);
            if (!win) {
                if (lane == 0) atomicCAS(err, 0, ERR_INTERNAL);
                break;
            }
            const int wl = __ffs(win) - 1;
            int y, col;
            if (G::RPL == 1) {
                // the (jj - excl)-th set bit of the winning lane's row: lane i
                // tests whether bits 0..i hold more members than that
                const uint32_t mw = (uint32_t)__shfl_sync(FULL_WARP, (uint32_t)m[0], wl);
                const uint32_t rr = __shfl_sync(FULL_WARP, jj - excl, wl);
                const uint32_t upto = (lane == 31) ? 0xFFFFFFFFu : ((2u << lane) - 1u);
                const unsigned past = __ballot_sync(FULL_WARP, (uint32_t)__popc(mw & upto) > rr);
                y = wl;
                col = __ffs(past) - 1;
            } else {
                uint32_t yc = 0;
                if (lane == wl) {
                    uint32_t rr = jj - excl;
                    int tsel = 0;
                    const uint32_t p0 = (uint32_t)popc_row(m[0]);
                    if (rr >= p0) { rr -= p0; tsel = 1; }
                    const int cc = select_bit((uint64_t)(tsel ? m[G::RPL - 1] : m[0]), rr);
                    yc = ((uint32_t)(lane * G::RPL + tsel) << 8) | (uint32_t)cc;
                }
                yc = __shfl_sync(FULL_WARP, yc, wl);
                y = (int)(yc >> 8);
                col = (int)(yc & 255u);
            }
#pragma unroll
            for (int tt = 0; tt < G::RPL; ++tt)
                if (lane * G::RPL + tt == y) pl.S[tt] ^= (row_t)1 << col;
            cn.H = (cn.H ^ (ev | (uint64_t)(y * LD + col))) * HASH_PRIME;
            ++cn.flips;
            pos = jx + 1;
            // the classes are needed again only if a step of this visit remains
            if (last_chunk && pos >= chunk_end) break;
            pl.flip_update(lane, y, col, c < 5);
            n_c = class_counts<LD>(pl, lane);
            Wc = (uint64_t)n_c * Ac;
            Cinc = prefix16(Wc, lane);
            R = __shfl_sync(FULL_WARP, Cinc, 9);
            state_scored = false;
        }
    }
}

// Four edge words of the warp's domain (N row, S row, W column, E column),
// the same in every lane.
struct Edges {
    uint64_t w[4];
};
template <int LD>
__device__ __forceinline__ Edges all_edges(const typename Geo<LD>::row_t (&S)[Geo<LD>::RPL])
{
    using G = Geo<LD>;
    Edges e;
    uint64_t colW = 0, colE = 0;
#pragma unroll
    for (int t = 0; t < G::RPL; ++t) {
        colW |= (uint64_t)__ballot_sync(FULL_WARP, (S[t] & 1u) != 0) << (32 * t);
        colE |= (uint64_t)__ballot_sync(FULL_WARP, ((S[t] >> (LD - 1)) & 1u) != 0) << (32 * t);
    }
    e.w[EDGE_N] = (uint64_t)__shfl_sync(FULL_WARP, S[0], 0);
    e.w[EDGE_S] = (uint64_t)__shfl_sync(FULL_WARP, S[G::RPL - 1], G::NACT - 1);
    e.w[EDGE_W] = colW;
    e.w[EDGE_E] = colE;
    return e;
}

// Stamped word w (0..7) of the warp's edges: half (w & 1) of edge (w >> 1).
__device__ __forceinline__ uint64_t stamped_word(const Edges &e, int w, uint32_t count)
{
    const int q = (w >> 1) & 3;
    const uint64_t x = (q == 0) ? e.w[0] : (q == 1) ? e.w[1] : (q == 2) ? e.w[2] : e.w[3];
    return stamp(count, (w & 1) ? (uint32_t)(x >> 32) : (uint32_t)x);
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
// Registers per thread, the fewest each variant compiles to without spills:
// 80 lets 24 warps share an SM (three CTAs of 8 warps or two of 12), 96 lets
// 20 (two of 10), which hides the latency of the visit's warp-collective
// chains better than 16 warps at 128 registers.
template <int LD, bool GRAD> constexpr int run_kernel_regs()
{
    return (GRAD && LD == 64) ? 128 : (GRAD || LD == 64) ? 96 : 80;
}

template <int LD, bool EXPO, bool GRAD, bool CLUSTER>
__global__ void __maxnreg__((run_kernel_regs<LD, GRAD>())) run_kernel(const RunParams P)
{
    using G = Geo<LD>;
    using row_t = typename G::row_t;
    using mem_t = typename G::mem_t;
    constexpr int TB = G::TILE_BYTES;
    constexpr int SB = slot_bytes<LD>();
    constexpr int OFF_EDGE = TB, OFF_CTR = TB + 64, OFF_META = TB + 120, OFF_OBS = TB + 152;
    // stamped words a halo read needs per neighbour: one half for LD <= 32, two for 64
    constexpr int HALVES = (LD > 32) ? 2 : 1;

    extern __shared__ __align__(16) uint8_t smem[];
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
            reinterpret_cast<int64_t *>(t + RT_GB)[lane] = (lane < 10) ? P.rep_gfix[(size_t)r * GFIX_WORDS + lane] : 0;
        }
        if (lane < 10) {
            reinterpret_cast<int64_t *>(t + RT_GH)[lane] = P.rep_gfix[(size_t)r * GFIX_WORDS + 10 + lane];
            const int32_t *lo = reinterpret_cast<const int32_t *>(P.rep_gfix + (size_t)r * GFIX_WORDS);
            reinterpret_cast<int32_t *>(t + RT_YB)[lane] = lo[2 * GFIX_YB + lane];
            reinterpret_cast<int32_t *>(t + RT_YH)[lane] = lo[2 * GFIX_YH + lane];
        }
        if (lane == 10) *reinterpret_cast<int64_t *>(t + RT_GSCALE) = P.rep_gfix[(size_t)r * GFIX_WORDS + 20];
        reinterpret_cast<double *>(t + 256)[lane] = P.rep_grad[(size_t)r * 32 + lane];
        if (lane == 0) {
            *reinterpret_cast<uint64_t *>(t + RT_SEED) = P.rep_seed[r];
            *reinterpret_cast<uint32_t *>(t + RT_DOMOFF) = P.rep_dom_off[r];
            *reinterpret_cast<int32_t *>(t + RT_DX) = P.rep_Dx[r];
            *reinterpret_cast<int32_t *>(t + RT_K) = P.rep_k[r];
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
        if (lane < 6) {
            // observation accumulators: no record yet, changes zero, clock product 1
            uint64_t *ob = reinterpret_cast<uint64_t *>(sl + OFF_OBS);
            ob[lane] = (lane == 0) ? (uint64_t)NO_RECORD : (lane == 2) ? (1ull << 63) : 0ull;
        }
        if (lane == 0) {
            meta[META_G] = g;
            meta[META_R] = r;
            meta[META_D] = g - P.rep_dom_off[r];
            meta[META_RT] = rt;
        }
        if (lane < 4) {
            const uint32_t nb = P.slot_nb[(size_t)s * 4 + lane];
            if (CLUSTER) {
                // address of the neighbour's slot in the cluster's shared memory
                const uint32_t nrank = nb >> 24, nslot_ = nb & 0xFFFFFFu;
                meta[META_NB + lane] = map_rank(smem_addr(slots + (size_t)nslot_ * SB), nrank);
            } else if (nb & 0x80000000u) {
                // neighbour in this CTA: shared-memory address of its slot, flagged
                meta[META_NB + lane] = 0x80000000u | smem_addr(slots + (size_t)(nb & 0x7FFFFFFFu) * SB);
            } else {
                meta[META_NB + lane] = nb;
            }
        }
        {
            // edges of the staged tile, stamped with visit count 0 (the slot's
            // copy; in GRID mode the global copy is the one neighbours read)
            row_t S[G::RPL];
            const mem_t *trow = reinterpret_cast<const mem_t *>(sl);
#pragma unroll
            for (int t = 0; t < G::RPL; ++t) S[t] = (lane < G::NACT) ? (row_t)trow[lane * G::RPL + t] : (row_t)0;
            const Edges ew = all_edges<LD>(S);
            if (lane < EDGE_WORDS) reinterpret_cast<uint64_t *>(sl + OFF_EDGE)[lane] = stamped_word(ew, lane, 0u);
        }
    }
    if (CLUSTER) cluster_sync();
    else __syncthreads();

    // Halo of a slot once its neighbours are ready.  Lane i (< 4*HALVES)
    // reads half (i / 4) of the edge word that borders on neighbour i % 4
    // (the N neighbour's S row, the S neighbour's N row, the W neighbour's E
    // column, the E neighbour's W column) until its stamp shows that the
    // neighbour has completed `need` visits, i.e. all its visits of earlier
    // phases (bounded spin).  A neighbour cannot complete another visit before
    // this one, so the stamp then equals `need`.
    unsigned long long warp_polls = 0; // poll iterations of this warp (profiling)
    auto wait_halo = [&](const uint32_t *meta, uint32_t needNS, uint32_t needWE, uint64_t &hN, uint64_t &hS,
                         uint64_t &hW, uint64_t &hE) -> bool {
        uint32_t half = 0;
        int good = 1;
        unsigned spins = 0;
        if (lane < 4 * HALVES) {
            const int dir = lane & 3, hf = lane >> 2;
            const uint32_t need = ((dir < 2) ? needNS : needWE) + (uint32_t)P.debug_extra;
            const int want = (dir == EDGE_N) ? EDGE_S : (dir == EDGE_S) ? EDGE_N : (dir == EDGE_W) ? EDGE_E : EDGE_W;
            const uint32_t nb = meta[META_NB + dir];
            const int word = 2 * want + hf;
            auto load = [&]() -> uint64_t {
                if (CLUSTER) return ld_dsmem(nb + OFF_EDGE + 8 * word);
                if (nb & 0x80000000u) return ld_volatile_shared((nb & 0x7FFFFFFFu) + OFF_EDGE + 8 * word);
                return ld_volatile_global(&P.edges[(size_t)nb * EDGE_WORDS + word]);
            };
            uint64_t v = load();
            if ((uint32_t)(v >> 32) < need) {
                const uint64_t t0 = global_ns();
                while (true) {
                    v = load();
                    if ((uint32_t)(v >> 32) >= need) break;
                    if ((++spins & 63u) == 0) {
                        if (*(volatile int *)P.err != 0) { good = 0; break; }
                        if (global_ns() - t0 > P.bar_limit_ns) {
                            atomicCAS(P.err, 0, ERR_TIMEOUT);
                            good = 0;
                            break;
                        }
                    }
                }
            }
            half = (uint32_t)v;
        }
        const bool all = __all_sync(FULL_WARP, good != 0);
        // the warp runs the loop as long as its slowest lane
        if (P.polls) warp_polls += __reduce_max_sync(FULL_WARP, spins);
        uint64_t h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint64_t lo = __shfl_sync(FULL_WARP, half, q);
            const uint64_t hi = (HALVES == 2) ? (uint64_t)__shfl_sync(FULL_WARP, half, 4 + q) : 0ull;
            h[q] = lo | (hi << 32);
        }
        hN = h[EDGE_N];
        hS = h[EDGE_S];
        hW = h[EDGE_W];
        hE = h[EDGE_E];
        return all;
    };

    // One visit; publishes the slot's edges, then (release) its visit count.
    const int nph = (P.schedule == SCHED_PALINDROME) ? 8 : 4; // colour passes per schedule

    // A slot's summed changes of one record go to the replica's record (lane
    // 0 of the warp; records past the launch's last one are dropped).
    auto flush_record = [&](const uint8_t *sl, uint32_t rep) {
        const uint32_t *ob = reinterpret_cast<const uint32_t *>(sl + OFF_OBS);
        const double *obd = reinterpret_cast<const double *>(sl + OFF_OBS + 32);
        const uint64_t *obm = reinterpret_cast<const uint64_t *>(sl + OFF_OBS + 16);
        const uint32_t o = ob[0];
        if (o == NO_RECORD || (int64_t)o >= P.n_obs) return;
        unsigned long long *acc = P.obs_acc + ((size_t)o * P.n_rep + rep) * OBS_WORDS;
        if (ob[1] != 0) atomicAdd(&acc[0], (unsigned long long)(long long)(int)ob[1]);
        if (ob[2] != 0) atomicAdd(&acc[1], (unsigned long long)(long long)(int)ob[2]);
        // the record's clock advance of this domain: one logarithm per record
        const double dt = EXPO ? domain_time(true, obm[0], (int64_t)obm[1], 0, P.lambda)
                               : P.horizon ? __dmul_rn((double)ob[3], P.dtau) : __ddiv_rn((double)ob[3], P.lambda);
        atomicAdd(reinterpret_cast<double *>(&acc[2]), dt);
        if (GRAD) {
            atomicAdd(reinterpret_cast<double *>(&acc[3]), obd[0]);
            atomicAdd(reinterpret_cast<double *>(&acc[4]), obd[1]);
        }
    };

    // Everything of a visit that does not depend on the halo, done before the
    // warp waits for its neighbours: the domain's rows and their interior
    // neighbour counts, its counters, the rate table and the first 32 steps'
    // random numbers.
    struct Prep {
        Planes<LD> pl;
        Counters cn;
        RateRegs rr;
        uint2 key;
        Chunk first;
        int k;
    };
    auto prepare = [&](const uint8_t *sl, uint64_t np0, int nf) -> Prep {
        Prep pp;
        const uint32_t *meta = reinterpret_cast<const uint32_t *>(sl + OFF_META);
        const uint8_t *rt = tables + (size_t)meta[META_RT] * RT_BYTES;
        const uint64_t seed = *reinterpret_cast<const uint64_t *>(rt + RT_SEED);
        pp.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
        pp.k = P.horizon ? horizon_steps(pp.key, meta[META_D], np0, P.htab, P.hkmax, lane)
                         : *reinterpret_cast<const int32_t *>(rt + RT_K);
        pp.rr = load_rates<GRAD>(rt, lane);
        pp.pl.valid = (lane < G::NACT) ? G::FULL : (row_t)0;
        const mem_t *trow = reinterpret_cast<const mem_t *>(sl);
#pragma unroll
        for (int t = 0; t < G::RPL; ++t) pp.pl.S[t] = (lane < G::NACT) ? (row_t)trow[lane * G::RPL + t] : (row_t)0;
        pp.pl.build_interior(lane);
        const uint64_t *ctr = reinterpret_cast<const uint64_t *>(sl + OFF_CTR);
        pp.cn.H = ctr[DCTR_HASH];
        pp.cn.flips = 0;
        pp.cn.clkM = ctr[DCTR_CLKM];
        pp.cn.clkE = (int64_t)ctr[DCTR_CLKE];
        pp.cn.sb = 0.0;
        pp.cn.sh = 0.0;
        pp.cn.dbonds = 0;
        pp.cn.dmag = 0;
        pp.cn.vM = 1ull << 63;
        pp.cn.vE = 0;
        pp.first = draw_chunk<EXPO>(pp.key, meta[META_D], np0, 0, nf * pp.k, max(pp.k, 1), lane);
        return pp;
    };

    // The visit once the halo is here.  The edges (with the new visit count)
    // are published first, since neighbours wait for them; then the tile, the
    // counters and the observation sums are stored in the slot.
    auto visit = [&](uint8_t *sl, Prep &pp, uint64_t np0, int nf, uint64_t hN, uint64_t hS, uint64_t hW,
                     uint64_t hE, uint32_t count_after, int64_t pass) {
        const uint32_t *meta = reinterpret_cast<const uint32_t *>(sl + OFF_META);
        Counters &cn = pp.cn;
        const int k = pp.k;
        visit_core<LD, EXPO, GRAD>(pp.pl, cn, pp.rr, pp.key, (row_t)hN, (row_t)hS, hW, hE, meta[META_D], np0,
                                   max(k, 1), lane, P.err, pp.first, nf * k);
        uint64_t *es = reinterpret_cast<uint64_t *>(sl + OFF_EDGE);
        const bool changed = cn.flips != 0; // warp-uniform
        uint64_t wv = 0;
        if (changed) {
            const Edges ew = all_edges<LD>(pp.pl.S);
            wv = stamped_word(ew, lane & 7, count_after);
        } else if (lane < EDGE_WORDS) {
            wv = (es[lane] & 0xFFFFFFFFull) | ((uint64_t)count_after << 32); // same edges, new count
        }
        if (lane < EDGE_WORDS) {
            // the slot's copy (read by this CTA's and, in CLUSTER mode, the
            // cluster's other warps) and, in GRID mode, the global copy
            reinterpret_cast<volatile uint64_t *>(es)[lane] = wv;
            if (!CLUSTER) st_cg(&P.edges[(size_t)meta[META_G] * EDGE_WORDS + lane], wv);
        }
        if (changed) {
            mem_t *wrow = reinterpret_cast<mem_t *>(sl);
            if (lane < G::NACT) {
#pragma unroll
                for (int t = 0; t < G::RPL; ++t) wrow[lane * G::RPL + t] = (mem_t)pp.pl.S[t];
            }
        }
        if (lane == 0) {
            uint64_t *ctr = reinterpret_cast<uint64_t *>(sl + OFF_CTR);
            ctr[DCTR_HASH] = cn.H;
            ctr[DCTR_FLIPS] += cn.flips;
            ctr[DCTR_STEPS] += (uint64_t)(nf * k);
            ctr[DCTR_CLKM] = cn.clkM;
            ctr[DCTR_CLKE] = (uint64_t)cn.clkE;
            if (GRAD) {
                reinterpret_cast<double *>(ctr)[DCTR_SB] += cn.sb;
                reinterpret_cast<double *>(ctr)[DCTR_SH] += cn.sh;
            }
            // observation: the visit's changes belong to the first record at or
            // after its pass (the finalize kernel adds the records up); they are
            // summed per slot and leave the CTA once per record
            if (P.n_obs > 0) {
                const int64_t o = (P.obs_pass ? pass : pass / nph) / P.obs_every;
                uint32_t *ob = reinterpret_cast<uint32_t *>(sl + OFF_OBS);
                uint64_t *obm = reinterpret_cast<uint64_t *>(sl + OFF_OBS + 16);
                double *obd = reinterpret_cast<double *>(sl + OFF_OBS + 32);
                if ((int64_t)ob[0] != o) {
                    flush_record(sl, meta[META_R]);
                    ob[0] = (uint32_t)o;
                    ob[1] = 0;
                    ob[2] = 0;
                    ob[3] = 0;
                    obm[0] = 1ull << 63;
                    obm[1] = 0;
                    obd[0] = 0.0;
                    obd[1] = 0.0;
                }
                ob[1] = (uint32_t)((int)ob[1] + cn.dbonds);
                ob[2] = (uint32_t)((int)ob[2] + cn.dmag);
                if (EXPO) {
                    uint64_t m = obm[0];
                    int64_t e = (int64_t)obm[1];
                    mant_mul(m, e, cn.vM, cn.vE);
                    obm[0] = m;
                    obm[1] = (uint64_t)e;
                } else {
                    ob[3] += P.horizon ? 1u : (uint32_t)(nf * k); // visits (fixed time) or steps
                }
                if (GRAD) {
                    obd[0] += cn.sb;
                    obd[1] += cn.sh;
                }
            }
        }
        __syncwarp();
    };

    // completed visit groups per colour in this launch (PALINDROME, FIXED)
    uint32_t gc0 = 0, gc1 = 0, gc2 = 0, gc3 = 0;
    auto gcount = [&](int c) { return c == 0 ? gc0 : c == 1 ? gc1 : c == 2 ? gc2 : gc3; };

    const uint64_t gp_begin = (uint64_t)P.sched_begin * nph;
    const uint64_t gp_end = (uint64_t)(P.sched_begin + P.n_sched) * nph;
    bool ok = true; // uniform within the warp; a warp that failed skips work but keeps every barrier
    uint64_t gp = gp_begin;
    while (gp < gp_end) {
        const uint64_t n = gp / nph;
        const int p = (int)(gp % nph);
        // global phase index of the Philox counter: 8 slots per schedule for every
        // schedule kind; the palindrome's fused phases (3,4) and seam (7 | next 0)
        // have consecutive indices
        const uint64_t np0 = n * 8 + (uint64_t)p;
        int nf = 1;
        if (P.schedule != SCHED_RANDOM_PERM) {
            const int colour = fixed_colour(P.schedule, p);
            // fuse following phases of the same colour unless an observation
            // intervenes (pass observation: every pass ends on its own)
            while (!P.obs_pass && !P.horizon && gp + nf < gp_end) {
                const uint64_t g2 = gp + nf;
                const int p2 = (int)(g2 % nph);
                if (fixed_colour(P.schedule, p2) != colour) break;
                if (p2 == 0) {
                    const int64_t nl_prev = (int64_t)(g2 / nph - 1 - (uint64_t)P.sched_begin);
                    if (P.obs_every > 0 && ((nl_prev + 1) % P.obs_every) == 0) break;
                }
                ++nf;
            }
            // a neighbour across a row has colour ^ 2, across a column colour ^ 1
            const uint32_t needNS = gcount(colour ^ 2), needWE = gcount(colour ^ 1);
            const uint32_t after = gcount(colour) + 1;
            if (ok) {
                const int i0 = (int)col_off[colour], i1 = (int)col_off[colour + 1];
                for (int i = i0 + wib; i < i1; i += nwarps) {
                    uint8_t *sl = slots + (size_t)i * SB;
                    Prep pp = prepare(sl, np0, nf);
                    uint64_t hN, hS, hW, hE;
                    if (!wait_halo(reinterpret_cast<const uint32_t *>(sl + OFF_META), needNS, needWE, hN, hS, hW, hE)) {
                        ok = false;
                        break;
                    }
                    visit(sl, pp, np0, nf, hN, hS, hW, hE, after, (int64_t)(gp - gp_begin));
                }
            }
            if (colour == 0) ++gc0;
            else if (colour == 1) ++gc1;
            else if (colour == 2) ++gc2;
            else ++gc3;
        } else if (ok) {
            // RANDOM_PERM: every replica draws its own colour order per schedule
            const uint32_t done_before = (uint32_t)(n - (uint64_t)P.sched_begin);
            for (int i = wib; i < nslot; i += nwarps) {
                uint8_t *sl = slots + (size_t)i * SB;
                const uint32_t *meta = reinterpret_cast<const uint32_t *>(sl + OFF_META);
                const uint32_t d = meta[META_D];
                const uint8_t *rt = tables + (size_t)meta[META_RT] * RT_BYTES;
                const uint64_t seed = *reinterpret_cast<const uint64_t *>(rt + RT_SEED);
                const int Dx = *reinterpret_cast<const int32_t *>(rt + RT_DX);
                const int c = (int)((d % (uint32_t)Dx) & 1u) | (int)(((d / (uint32_t)Dx) & 1u) << 1);
                if (perm_colour(seed, n, p) != c) continue;
                // neighbours' colours c^2 (rows) and c^1 (columns): done in this
                // schedule iff they came earlier in its order
                int posNS = 0, posWE = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int cq = perm_colour(seed, n, q);
                    if (cq == (c ^ 2)) posNS = q;
                    if (cq == (c ^ 1)) posWE = q;
                }
                Prep pp = prepare(sl, np0, 1);
                uint64_t hN, hS, hW, hE;
                if (!wait_halo(meta, done_before + (posNS < p ? 1u : 0u), done_before + (posWE < p ? 1u : 0u), hN, hS,
                               hW, hE)) {
                    ok = false;
                    break;
                }
                visit(sl, pp, np0, 1, hN, hS, hW, hE, done_before + 1u, (int64_t)(gp - gp_begin));
            }
        }
        gp += (uint64_t)nf;
    }
    if (P.polls && lane == 0 && warp_polls != 0) atomicAdd(P.polls, warp_polls);
    // every warp of the CTA must have finished its visits before any warp
    // writes a slot back; in CLUSTER mode, also no CTA may leave while another
    // still reads its shared memory
    if (CLUSTER) cluster_sync();
    else __syncthreads();
    if (*(volatile int *)P.err != 0) return;
    // write owned tiles and counters back (and edges, for the observables
    // kernel), and each slot's open record
    for (int i = wib; i < nslot; i += nwarps) {
        const uint8_t *sl = slots + (size_t)i * SB;
        const uint32_t g = reinterpret_cast<const uint32_t *>(sl + OFF_META)[META_G];
        if (lane == 0 && P.n_obs > 0) flush_record(sl, reinterpret_cast<const uint32_t *>(sl + OFF_META)[META_R]);
        for (int q = lane * 4; q < TB; q += 128)
            *reinterpret_cast<uint32_t *>(P.tiles + (size_t)g * TB + q) = *reinterpret_cast<const uint32_t *>(sl + q);
        if (lane < DCTR_WORDS)
            P.dctr[(size_t)g * DCTR_WORDS + lane] = reinterpret_cast<const uint64_t *>(sl + OFF_CTR)[lane];
        if (CLUSTER && lane < EDGE_WORDS)
            P.edges[(size_t)g * EDGE_WORDS + lane] = reinterpret_cast<const uint64_t *>(sl + OFF_EDGE)[lane];
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
    const int32_t *rep_init; // per-replica start (init mode INIT_PER_REPLICA)
    const uint32_t *dom_rep;
    int8_t *spins;
    uint8_t *tiles;
    uint64_t *edges;
    uint64_t *dctr;
    int *err;
};

// iid +-1 from Philox (block b of 128 sites: counter {b_lo, b_hi, 0, TAG_INIT<<24}) or all up;
// init = INIT_PER_REPLICA takes each replica's mode from rep_init (INIT_KEEP leaves it alone).
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
        const int mode = (init == INIT_PER_REPLICA) ? P.rep_init[r] : init;
        if (mode == INIT_KEEP) continue;
        const uint64_t b = t - P.rep_blk_off[r];
        uint4 w = make_uint4(~0u, ~0u, ~0u, ~0u);
        if (mode == 0) {
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
        const Edges ew = all_edges<LD>(S);
        if (lane < EDGE_WORDS) P.edges[(uint64_t)g * EDGE_WORDS + lane] = stamped_word(ew, lane, 0u);
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
        const uint64_t *eS = P.edges + (gbase + (uint32_t)(((by + 1) % Dx) * Dx + bx)) * EDGE_WORDS;
        const uint64_t *eE = P.edges + (gbase + (uint32_t)(by * Dx + (bx + 1) % Dx)) * EDGE_WORDS;
        const uint64_t hS = (eS[2 * EDGE_N] & 0xFFFFFFFFull) | (eS[2 * EDGE_N + 1] << 32);
        const uint64_t hE = (eE[2 * EDGE_W] & 0xFFFFFFFFull) | (eE[2 * EDGE_W + 1] << 32);
        row_t S[G::RPL];
        const mem_t *trow = reinterpret_cast<const mem_t *>(P.tiles + (uint64_t)g * G::TILE_BYTES);
#pragma unroll
        for (int t = 0; t < G::RPL; ++t) S[t] = (lane < G::NACT) ? (row_t)trow[lane * G::RPL + t] : (row_t)0;
        int bonds, mag;
        domain_bonds_mag<LD>(S, hE, hS, lane, bonds, mag);
        if (lane == 0) {
            const uint64_t *ctr = P.dctr + (uint64_t)g * DCTR_WORDS;
            const double t = P.horizon ? __dmul_rn((double)visits, P.dtau)
                                       : domain_time(EXPO, ctr[DCTR_CLKM], (int64_t)ctr[DCTR_CLKE],
                                                     visits * (int64_t)P.rep_k[r], P.lambda);
            unsigned long long *a = acc + (size_t)r * OBS_WORDS;
            atomicAdd(&a[0], (unsigned long long)(long long)bonds);
            atomicAdd(&a[1], (unsigned long long)(long long)mag);
            atomicAdd(reinterpret_cast<double *>(&a[2]), t);
            atomicAdd(reinterpret_cast<double *>(&a[3]), __longlong_as_double((long long)ctr[DCTR_SB]));
            atomicAdd(reinterpret_cast<double *>(&a[4]), __longlong_as_double((long long)ctr[DCTR_SH]));
        }
    }
}

// Records {e, m, e*m, T (, score beta, score h)}: record o = base (the state
// before the launch) + the changes of every record up to o.  One thread per
// replica walks its records in order; the integer sums are exact and e, m
// follow the oracle's FP64 formula.
__global__ void finalize_obs_kernel(const unsigned long long *base /* [n_rep][OBS_WORDS] */,
                                         const unsigned long long *acc, int64_t n_obs, int n_rep,
                                         const int32_t *rep_L, const int32_t *rep_Dx, double J,
                                         const double *rep_h, double *out, int stride)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rep) return;
    const unsigned long long *b0 = base + (size_t)r * OBS_WORDS;
    long long bonds = (long long)b0[0], mag = (long long)b0[1];
    double tsum = __longlong_as_double((long long)b0[2]);
    double sb = __longlong_as_double((long long)b0[3]), sh = __longlong_as_double((long long)b0[4]);
    const double N = (double)rep_L[r] * (double)rep_L[r];
    const double nD = (double)rep_Dx[r] * (double)rep_Dx[r];
    for (int64_t o = 0; o < n_obs; ++o) {
        const unsigned long long *a = acc + ((size_t)o * n_rep + r) * OBS_WORDS;
        bonds += (long long)a[0];
        mag += (long long)a[1];
        tsum = __dadd_rn(tsum, __longlong_as_double((long long)a[2]));
        sb = __dadd_rn(sb, __longlong_as_double((long long)a[3]));
        sh = __dadd_rn(sh, __longlong_as_double((long long)a[4]));
        const double b = (double)bonds, m = (double)mag;
        const double e = __ddiv_rn(__dsub_rn(__dmul_rn(-J, b), __dmul_rn(rep_h[r], m)), N);
        const double mm = __ddiv_rn(m, N);
        double *w = out + ((size_t)o * n_rep + r) * stride;
        w[0] = e;
        w[1] = mm;
        w[2] = __dmul_rn(e, mm);
        w[3] = __ddiv_rn(tsum, nD);
        if (stride >= 6) {
            w[4] = sb;
            w[5] = sh;
        }
    }
}

// per-domain counters -> host-facing arrays (hash, flips, clock)
// dtau > 0: fixed-time visits, the clock is visits * dtau.
template <bool EXPO>
__global__ void domain_state_kernel(const uint64_t *dctr, int n_dom, int64_t visits, const uint32_t *dom_rep,
                                    const int32_t *rep_k, double lambda, double dtau, uint64_t *hash,
                                    int64_t *flips, double *t, int64_t *steps)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_dom) return;
    const uint64_t *c = dctr + (uint64_t)g * DCTR_WORDS;
    hash[g] = c[DCTR_HASH];
    flips[g] = (int64_t)c[DCTR_FLIPS];
    steps[g] = (int64_t)c[DCTR_STEPS];
    t[g] = dtau > 0.0 ? __dmul_rn((double)visits, dtau)
                      : domain_time(EXPO, c[DCTR_CLKM], (int64_t)c[DCTR_CLKE], visits * (int64_t)rep_k[dom_rep[g]],
                                    lambda);
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
    c[DCTR_STEPS] = 0;
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

// Likelihood-ratio estimate of d E[A]/d theta over the replicas, with A_r
// = A[r * stride]: out[0] = mean A, out[1 + j] = (1/(R - 1)) sum_r (A_r -
// mean A) S_r,j + mean X_j (j = beta, h), where X_r,j = xsel-dependent
// explicit derivative of A_r (xsel 0: none; 1: -m_r; 2: -m_r^2, m_r =
// M[r * stride], for j = h only).  The 1/(R - 1) makes the estimate unbiased
// with the replica mean as baseline (E[S] = 0).  One block of 256 threads,
// sums in a fixed order.
__global__ void lr_estimate_kernel(const double *A, const double *M, int stride, int xsel, const uint64_t *dctr,
                                   const uint32_t *rep_dom_off, int n_rep, double *out)
{
    __shared__ double red[3][256];
    const int t = threadIdx.x;
    double a = 0.0, x = 0.0;
    for (int r = t; r < n_rep; r += blockDim.x) {
        a += A[(size_t)r * stride];
        if (xsel != 0) {
            const double m = M[(size_t)r * stride];
            x -= (xsel == 1) ? m : m * m;
        }
    }
    red[0][t] = a;
    red[1][t] = x;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w) {
            red[0][t] += red[0][t + w];
            red[1][t] += red[1][t + w];
        }
        __syncthreads();
    }
    const double mean = red[0][0] / (double)n_rep;
    const double xmean = red[1][0] / (double)n_rep;
    __syncthreads();
    double sb = 0.0, sh = 0.0;
    for (int r = t; r < n_rep; r += blockDim.x) {
        double xb = 0.0, xh = 0.0;
        for (uint32_t g = rep_dom_off[r]; g < rep_dom_off[r + 1]; ++g) {
            xb += __longlong_as_double((long long)dctr[(uint64_t)g * DCTR_WORDS + DCTR_SB]);
            xh += __longlong_as_double((long long)dctr[(uint64_t)g * DCTR_WORDS + DCTR_SH]);
        }
        const double c = A[(size_t)r * stride] - mean;
        sb += c * xb;
        sh += c * xh;
    }
    red[1][t] = sb;
    red[2][t] = sh;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w) {
            red[1][t] += red[1][t + w];
            red[2][t] += red[2][t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        out[0] = mean;
        out[1] = red[1][0] / (double)(n_rep - 1);
        out[2] = red[2][0] / (double)(n_rep - 1) + xmean;
    }
}

} // namespace kmcdev
