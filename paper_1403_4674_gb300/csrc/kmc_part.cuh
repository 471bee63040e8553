// kmc_part.cuh -- sm_103a device code for small periodic lattices (L <= 128)
// under the partitions of Sec. 3.2: a Dx x Dx grid of square blocks or N_D
// vertical stripes of width L/N_D and full height (Fig. 1 caption), with any
// domain size n_d (the paper's 12^2 and 100^2 lattices).
//
// Data parallelism is over trajectories (the paper's N_TRAJ runs per
// setting): one warp owns one trajectory for the whole launch and runs its
// domain processes in schedule order, so the halo of a visit is the live
// state -- no other domain of the trajectory moves meanwhile.  The lattice
// lives in shared memory as bit rows (row y: two 64-bit words, bit x =
// column x, 1 = up).  Lane l holds domain rows l*RPL .. l*RPL+RPL-1
// (RPL = ceil(H/32)), so a warp scan over lanes runs in row-major order.
//
// Step target (n_d not a power of two): P = 63 - ceil(log2 n_d),
// M = n_d 2^P, target = floor(X M / 2^64) for X = w0 | w1<<32; with n_d a
// power of two this is X >> 1, the lattice path's target.
#pragma once

#include <cstdint>

#include "kmc_kernels.cuh"

namespace kmcpart {

using kmcdev::FULL_WARP;
using kmcdev::HASH_PRIME;
using u128 = unsigned __int128;

constexpr int PART_WARPS = 4;        // trajectories per CTA
constexpr int PART_MAX_L = 128;
constexpr int PART_PHASE_SLOTS = 64; // Philox phase index np = n*64 + p
constexpr int PART_BLOCKS = 0, PART_STRIPES = 1;
constexpr uint32_t PART_TAG_PERM = 2u;
// shared memory per warp (64-bit words): bit rows, the domain order, the
// class counts of every domain (int [64][10]), the rate sum R' of every
// domain (u64 [64]), the fixed-point rates (u64 [16]) and, when the lattice
// has at most PART_RC_ROWS domain rows (N_D x domain height), the class
// counts of every domain row (u8 [rows][10], in 32-bit words)
constexpr int PART_RC_ROWS = 512;
constexpr int PART_OFF_ORDER = 2 * PART_MAX_L, PART_OFF_DCOUNT = PART_OFF_ORDER + 8,
              PART_OFF_DR = PART_OFF_DCOUNT + 64 * 10 / 2, PART_OFF_ATAB = PART_OFF_DR + 64,
              PART_OFF_RC = PART_OFF_ATAB + 16;
constexpr int PART_WARP_WORDS = PART_OFF_RC + PART_RC_ROWS * 10 / 8;

struct PartParams {
    int n_traj, L, kind, ND, k;
    int Dx;              // blocks per side (blocks), else 0
    int W, H;            // domain width and height
    int ncol;            // colours (1, 2 or 4)
    int schedule, obs_every;
    int64_t sched_begin, n_sched;
    uint64_t M;          // n_d 2^P
    double J, nu;
    const uint64_t *seed; // [n_traj]
    const uint64_t *A;    // [n_traj][10]
    const double *h;      // [n_traj]
    int8_t *spins;        // [n_traj][L][L], +-1
    uint64_t *hash, *clkM;
    int64_t *clkE, *flips, *steps;
    double *t;            // [n_traj] clock after the launch
    double *obs;          // [n_rec][n_traj][4] or null
    int *err;
};

__device__ __forceinline__ u128 row_ld(const uint64_t *rows, int y)
{
    return ((u128)rows[2 * y + 1] << 64) | rows[2 * y];
}

// bit x <- bit x-1 (mod L) / bit x <- bit x+1 (mod L) of an L-bit row
__device__ __forceinline__ u128 rot_w(u128 c, int L, u128 Lm) { return ((c << 1) | (c >> (L - 1))) & Lm; }
__device__ __forceinline__ u128 rot_e(u128 c, int L) { return (c >> 1) | ((c & (u128)1) << (L - 1)); }

__device__ __forceinline__ int popc128(u128 v) { return __popcll((uint64_t)v) + __popcll((uint64_t)(v >> 64)); }

// Up-neighbour count planes (bit-sliced b2 b1 b0) of row y, restricted to the
// domain columns DM, and its up / down spins there.
struct RowPlanes {
    u128 up, dn, b0, b1, b2;
};

__device__ __forceinline__ RowPlanes row_planes(const uint64_t *rows, int y, int L, u128 Lm, u128 DM)
{
    const u128 c = row_ld(rows, y);
    const u128 n = row_ld(rows, (y == 0) ? L - 1 : y - 1);
    const u128 s = row_ld(rows, (y == L - 1) ? 0 : y + 1);
    const u128 w = rot_w(c, L, Lm), e = rot_e(c, L);
    const u128 s1 = n ^ s, c1 = n & s, s2 = w ^ e, c2 = w & e, t0 = s1 & s2;
    RowPlanes p;
    p.b0 = s1 ^ s2;
    p.b1 = c1 ^ c2 ^ t0;
    p.b2 = (c1 & c2) | (c1 & t0) | (c2 & t0);
    p.up = c & DM;
    p.dn = ~c & DM;
    return p;
}

// Sites of class c = 5 up + q in a row.
__device__ __forceinline__ u128 class_mask(const RowPlanes &p, int c)
{
    const int q = (c >= 5) ? c - 5 : c;
    const u128 ones = ~(u128)0;
    const u128 diff = (p.b2 ^ ((q & 4) ? ones : 0)) | (p.b1 ^ ((q & 2) ? ones : 0)) | (p.b0 ^ ((q & 1) ? ones : 0));
    return ((c >= 5) ? p.up : p.dn) & ~diff;
}

// Lane c (< 10) receives n_c of the domain (rows y0 .. y0+H-1).
__device__ __forceinline__ uint32_t part_counts(const uint64_t *rows, int lane, int y0, int H, int RPL, int L,
                                                u128 Lm, u128 DM)
{
    uint32_t w[5] = {0, 0, 0, 0, 0};
    for (int t = 0; t < RPL; ++t) {
        const int yy = lane * RPL + t;
        if (yy >= H) break;
        const RowPlanes p = row_planes(rows, y0 + yy, L, Lm, DM);
        const u128 n2 = ~p.b2;
        const u128 e[5] = {n2 & ~p.b1 & ~p.b0, n2 & ~p.b1 & p.b0, n2 & p.b1 & ~p.b0, n2 & p.b1 & p.b0, p.b2};
#pragma unroll
        for (int q = 0; q < 5; ++q)
            w[q] += (uint32_t)popc128(p.dn & e[q]) | ((uint32_t)popc128(p.up & e[q]) << 16);
    }
    uint32_t tw = 0;
    const int q = (lane < 5) ? lane : lane - 5;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const uint32_t s = __reduce_add_sync(FULL_WARP, w[i]);
        if (q == i) tw = s;
    }
    const uint32_t n = (lane < 5) ? (tw & 0xFFFFu) : (tw >> 16);
    return (lane < 10) ? n : 0u;
}

// The rr-th (0-based) set bit of a 128-bit mask; rr < popc(m).
__device__ __forceinline__ int select128(u128 m, uint32_t rr)
{
    const uint64_t lo = (uint64_t)m;
    const uint32_t pl = (uint32_t)__popcll(lo);
    if (rr < pl) return kmcdev::select_bit(lo, rr);
    return 64 + kmcdev::select_bit((uint64_t)(m >> 64), rr - pl);
}

// Class 5 up + (number of up neighbours) of site (x, y), from the live rows.
__device__ __forceinline__ int site_class(const uint64_t *rows, int x, int y, int L)
{
    const int xm = (x == 0) ? L - 1 : x - 1, xp = (x == L - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? L - 1 : y - 1, yp = (y == L - 1) ? 0 : y + 1;
    auto bit = [&](int xx, int yy) { return (int)((rows[2 * yy + (xx >> 6)] >> (xx & 63)) & 1ull); };
    return 5 * bit(x, y) + bit(xm, y) + bit(xp, y) + bit(x, ym) + bit(x, yp);
}

template <bool EXPO>
__global__ void __launch_bounds__(PART_WARPS * 32) part_kernel(const PartParams P)
{
    extern __shared__ uint64_t part_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tr = blockIdx.x * PART_WARPS + warp;
    if (tr >= P.n_traj) return; // whole warps only; no CTA-wide barrier below
    const int L = P.L;
    uint64_t *rows = part_smem + (size_t)warp * PART_WARP_WORDS;
    uint8_t *order = reinterpret_cast<uint8_t *>(rows + PART_OFF_ORDER);
    int *dcount = reinterpret_cast<int *>(rows + PART_OFF_DCOUNT);              // [N_D][10] class counts
    unsigned long long *dR = reinterpret_cast<unsigned long long *>(rows + PART_OFF_DR); // [N_D] R'
    uint64_t *Atab = rows + PART_OFF_ATAB;                                       // [10] A_c
    uint8_t *rc = reinterpret_cast<uint8_t *>(rows + PART_OFF_RC);               // [N_D * H][10]
    const u128 Lm = (L == 128) ? ~(u128)0 : (((u128)1 << L) - 1);
    const int8_t *sp = P.spins + (size_t)tr * L * L;

    // load the lattice into bit rows (ballots over 32-column chunks)
    int bad = 0;
    for (int y = 0; y < L; ++y) {
        uint64_t wd[2] = {0, 0};
        for (int x0 = 0; x0 < L; x0 += 32) {
            const int x = x0 + lane;
            const int8_t v = (x < L) ? sp[(size_t)y * L + x] : (int8_t)-1;
            bad |= (v != 1 && v != -1);
            const uint32_t b = __ballot_sync(FULL_WARP, v == 1);
            wd[x0 >> 6] |= (uint64_t)b << (x0 & 63);
        }
        if (lane == 0) {
            rows[2 * y] = wd[0];
            rows[2 * y + 1] = wd[1];
        }
    }
    if (__any_sync(FULL_WARP, bad) && lane == 0) atomicOr(P.err, 1);
    __syncwarp();

    uint64_t A = 0;
    if (lane < 10) A = P.A[(size_t)tr * 10 + lane];
    // 1/A_c from below (A_c rounded up, its reciprocal rounded down)
    const float invAf = (lane < 10) ? __frcp_rd(kmcdev::u64_to_float_ru(A)) : 0.0f;
    const uint64_t seed = P.seed[tr];
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const double hr = P.h[tr];
    uint64_t H = P.hash[tr], clkM = P.clkM[tr];
    int64_t clkE = P.clkE[tr], flips = P.flips[tr], steps = P.steps[tr];
    const int W = P.W, Hd = P.H, RPL = (Hd + 31) / 32, k = P.k;
    const u128 DM0 = (W == 128) ? ~(u128)0 : (((u128)1 << W) - 1);
    const uint64_t M = P.M;

    auto domain_origin = [&](int d, int &x0, int &y0) {
        if (P.kind == PART_STRIPES) {
            x0 = d * W;
            y0 = 0;
        } else {
            x0 = (d % P.Dx) * W;
            y0 = (d / P.Dx) * W;
        }
    };
    // class counts of every domain (and of every domain row, when they
    // fit) and every domain's rate sum, kept up to date flip by flip
    const bool use_rc = P.ND * Hd <= PART_RC_ROWS;
    if (lane < 10) Atab[lane] = A;
    for (int d = 0; d < P.ND; ++d) {
        int x0, y0;
        domain_origin(d, x0, y0);
        const uint32_t n = part_counts(rows, lane, y0, Hd, RPL, L, Lm, DM0 << x0);
        if (lane < 10) dcount[d * 10 + lane] = (int)n;
        const uint64_t R0 = __shfl_sync(FULL_WARP, kmcdev::prefix16((uint64_t)n * A, lane), 9);
        if (lane == 0) dR[d] = R0;
        if (use_rc) {
            for (int yy = lane; yy < Hd; yy += 32) {
                const RowPlanes pr = row_planes(rows, y0 + yy, L, Lm, DM0 << x0);
                for (int c = 0; c < 10; ++c) rc[(d * Hd + yy) * 10 + c] = (uint8_t)popc128(class_mask(pr, c));
            }
        }
    }
    __syncwarp();
    // a domain row's count byte: the 32-bit word holding it and its shift
    auto rc_word = [&](int d, int yy, int c, int &sh) {
        const int b = (d * Hd + yy) * 10 + c;
        sh = 8 * (b & 3);
        return reinterpret_cast<unsigned *>(rc) + (b >> 2);
    };

    // The real events among the steps held by lanes [lo, hi): lane i holds
    // step j = i - lo + jbase of the visit (target tgt, ~0 for no step).
    // Null runs are skipped by one ballot; each real event selects its class
    // and member, flips, and updates the class counts of the domains the five
    // touched sites belong to.
    auto events = [&](int d, uint64_t np, int x0, int y0, u128 DM, uint64_t tgt, int lo, int hi, int jbase) {
        // a visit without real events needs only the domain's rate sum
        uint64_t R = dR[d];
        if (!__any_sync(FULL_WARP, lane >= lo && lane < hi && tgt < R)) return;
        uint32_t n_c = (lane < 10) ? (uint32_t)dcount[d * 10 + lane] : 0u;
        uint64_t Wc = (uint64_t)n_c * A;
        uint64_t Cinc = kmcdev::prefix16(Wc, lane);
        int pos = lo;
        while (true) {
            const unsigned real = __ballot_sync(FULL_WARP, lane >= pos && lane < hi && tgt < R);
            if (!real) break;
            const int jx = __ffs(real) - 1;
            const uint64_t t = __shfl_sync(FULL_WARP, tgt, jx);
            const unsigned sel = __ballot_sync(FULL_WARP, lane < 10 && t < Cinc);
            const int c = __ffs(sel) - 1;
            // exact q = floor((t - C_{c-1}) / A_c) < n_c <= 16384 from an FP32
            // estimate with every rounding toward the lower side (so it is q or
            // q - 1) and one integer comparison, instead of a 64-bit division
            const uint64_t xq = t - (Cinc - Wc);
            uint32_t q = (uint32_t)__fmul_rz(kmcdev::u64_to_float_rz(xq), invAf);
            q = (xq - (uint64_t)q * A >= A) ? q + 1u : q;
            const uint32_t jj = __shfl_sync(FULL_WARP, q, c);
            // jj-th member of class c in row-major order
            uint32_t cl = 0;
            for (int tt = 0; tt < RPL; ++tt) {
                const int yy = lane * RPL + tt;
                if (yy >= Hd) break;
                cl += use_rc ? (uint32_t)rc[(d * Hd + yy) * 10 + c]
                             : (uint32_t)popc128(class_mask(row_planes(rows, y0 + yy, L, Lm, DM), c));
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
                if (lane == 0) atomicOr(P.err, 2);
                break;
            }
            const int wl = __ffs(win) - 1;
            uint32_t yx = 0;
            if (lane == wl) {
                uint32_t rr = jj - excl;
                for (int tt = 0; tt < RPL; ++tt) {
                    const int yy = lane * RPL + tt;
                    if (use_rc) {
                        // the row from its count, then that row's class mask alone
                        const uint32_t pc = rc[(d * Hd + yy) * 10 + c];
                        if (rr < pc) {
                            const u128 mk = class_mask(row_planes(rows, y0 + yy, L, Lm, DM), c);
                            yx = ((uint32_t)yy << 8) | (uint32_t)select128(mk, rr);
                            break;
                        }
                        rr -= pc;
                        continue;
                    }
                    const u128 mk = class_mask(row_planes(rows, y0 + yy, L, Lm, DM), c);
                    const uint32_t pc = (uint32_t)popc128(mk);
                    if (rr < pc) {
                        yx = ((uint32_t)yy << 8) | (uint32_t)select128(mk, rr);
                        break;
                    }
                    rr -= pc;
                }
            }
            yx = __shfl_sync(FULL_WARP, yx, wl);
            const int yy = (int)(yx >> 8), x = (int)(yx & 255u);
            // the flip changes the classes of the site and its four
            // neighbours (lanes 0..4); their domains' counts follow
            const int y = y0 + yy;
            int sx = x, sy = y;
            if (lane == 1) sx = (x == 0) ? L - 1 : x - 1;
            if (lane == 2) sx = (x == L - 1) ? 0 : x + 1;
            if (lane == 3) sy = (y == 0) ? L - 1 : y - 1;
            if (lane == 4) sy = (y == L - 1) ? 0 : y + 1;
            const bool mine = lane < 5 && !(L == 2 && (lane == 2 || lane == 4)); // L = 2: x-1 = x+1
            const int sd = (P.kind == PART_STRIPES) ? sx / W : (sy / W) * P.Dx + sx / W;
            __syncwarp();
            const int old_c = mine ? site_class(rows, sx, sy, L) : 0;
            __syncwarp();
            if (lane == 0) rows[2 * y + (x >> 6)] ^= 1ull << (x & 63);
            __syncwarp();
            if (mine) {
                const int new_c = site_class(rows, sx, sy, L);
                if (new_c != old_c) {
                    atomicAdd(&dcount[sd * 10 + old_c], -1);
                    atomicAdd(&dcount[sd * 10 + new_c], 1);
                    atomicAdd(&dR[sd], (unsigned long long)(Atab[new_c] - Atab[old_c])); // mod 2^64
                    if (use_rc) {
                        const int syy = (P.kind == PART_STRIPES) ? sy : sy - (sd / P.Dx) * W;
                        int sh0, sh1;
                        unsigned *w0 = rc_word(sd, syy, old_c, sh0);
                        unsigned *w1 = rc_word(sd, syy, new_c, sh1);
                        atomicSub(w0, 1u << sh0); // the byte holds at least this site
                        atomicAdd(w1, 1u << sh1);
                    }
                }
            }
            __syncwarp();
            const uint64_t ev = (np << 32) | ((uint64_t)(jx - lo + jbase) << 16) | (uint64_t)(yy * W + (x - x0));
            H = (H ^ ev) * HASH_PRIME;
            ++flips;
            pos = jx + 1;
            // the classes are needed again only if a step of this visit remains
            if (pos >= hi) break;
            n_c = (lane < 10) ? (uint32_t)dcount[d * 10 + lane] : 0u;
            Wc = (uint64_t)n_c * A;
            Cinc = kmcdev::prefix16(Wc, lane);
            R = dR[d];
        }
    };

    // Step draw of lane `lane` for step j of domain d in phase np:
    // target = floor(X M / 2^64) (tgt) and the clock variate (V).
    auto draw = [&](uint32_t j, uint32_t d, uint64_t np, uint64_t &tgt, uint64_t &V) {
        const uint4 w = kmcdev::philox4x32_10(make_uint4(j, d, (uint32_t)np, (uint32_t)(np >> 32) & 0xFFFFFFu), key);
        tgt = __umul64hi(((uint64_t)w.y << 32) | w.x, M);
        V = ((((uint64_t)w.w << 32) | w.z) >> 11) + 1ull;
    };
    // Product of the variates of aligned groups of `span` lanes (a power of
    // two; lanes without a step hold 1): lane 0 of each group receives it.
    auto variate_product = [&](uint64_t V, int span, uint64_t &m, int &e) {
        const int z = __clzll((long long)V);
        m = V << z;
        e = 10 - z;
        for (int off = 1; off < span; off <<= 1) {
            const uint64_t m2 = __shfl_xor_sync(FULL_WARP, m, off);
            const int e2 = __shfl_xor_sync(FULL_WARP, e, off);
            kmcdev::mant_mul32(m, e, m2, e2);
        }
    };

    // One visit with its own draws, 32 steps at a time.
    auto visit = [&](int d, uint64_t np) {
        int x0, y0;
        domain_origin(d, x0, y0);
        const u128 DM = DM0 << x0;
        for (int base = 0; base < k; base += 32) {
            uint64_t tgt = ~0ull, V = 1ull << 53;
            if (base + lane < k) draw((uint32_t)(base + lane), (uint32_t)d, np, tgt, V);
            const int chunk_end = min(32, k - base);
            if (EXPO) {
                uint64_t m;
                int e;
                variate_product(V, 32, m, e);
                kmcdev::mant_mul(clkM, clkE, __shfl_sync(FULL_WARP, m, 0), (int64_t)__shfl_sync(FULL_WARP, e, 0));
            }
            steps += chunk_end;
            events(d, np, x0, y0, DM, tgt, 0, chunk_end, base);
        }
    };

    const bool perm = P.schedule == kmcdev::SCHED_RANDOM_PERM;
    const int nph = perm ? P.ND : (P.schedule == kmcdev::SCHED_PALINDROME ? 2 * P.ncol : P.ncol);
    const int dpp = (perm || P.ND == 1) ? 1 : P.ND / P.ncol; // visits per phase
    const int Vs = nph * dpp;                                // visits per schedule
    const double N = (double)L * (double)L;
    int64_t passes = 0;

    // colour of phase p: 0 1 .. [.. 1 0]; the i-th domain of colour col in
    // ascending order (blocks: by = col>>1 + 2 (i / (Dx/2)), bx = col&1 + 2 (i % (Dx/2)))
    auto phase_colour = [&](int p) { return (p < P.ncol) ? p : (2 * P.ncol - 1 - p); };
    auto domain_of_colour = [&](int col, int i) {
        if (P.ND == 1) return 0;
        if (P.kind == PART_STRIPES) return col + 2 * i;
        const int half = P.Dx / 2;
        return ((col >> 1) + 2 * (i / half)) * P.Dx + (col & 1) + 2 * (i % half);
    };
    // the paper's random order of all domains of schedule n (Fisher-Yates over Philox)
    auto shuffle = [&](uint8_t *ord, uint64_t n) {
        for (int i = 0; i < P.ND; ++i) ord[i] = (uint8_t)i;
        for (int i = P.ND - 1; i >= 1; --i) {
            const uint4 w = kmcdev::philox4x32_10(
                make_uint4((uint32_t)i, 0u, (uint32_t)n, ((uint32_t)(n >> 32) & 0xFFFFFFu) | (PART_TAG_PERM << 24)),
                key);
            const int jx = (int)__umul64hi(((uint64_t)w.y << 32) | w.x, (uint64_t)(i + 1));
            const uint8_t tmp = ord[i];
            ord[i] = ord[jx];
            ord[jx] = tmp;
        }
    };
    auto pass_done = [&]() {
        ++passes;
        if (P.obs != nullptr && P.obs_every > 0 && passes % P.obs_every == 0) {
            // bonds = 2 L^2 - 2 (unlike neighbour pairs), mag = 2 (up spins) - L^2
            int unlike = 0, up = 0;
            for (int y = lane; y < L; y += 32) {
                const u128 c = row_ld(rows, y);
                const u128 s = row_ld(rows, (y == L - 1) ? 0 : y + 1);
                unlike += popc128((c ^ rot_e(c, L)) & Lm) + popc128(c ^ s);
                up += popc128(c);
            }
            unlike = __reduce_add_sync(FULL_WARP, unlike);
            up = __reduce_add_sync(FULL_WARP, up);
            if (lane == 0) {
                const int64_t bonds = 2ll * L * L - 2ll * unlike;
                const int64_t mag = 2ll * up - (int64_t)L * L;
                const double e = __ddiv_rn(__dsub_rn(__dmul_rn(-P.J, (double)bonds), __dmul_rn(hr, (double)mag)), N);
                const double m = __ddiv_rn((double)mag, N);
                double4_32a v;
                v.x = e;
                v.y = m;
                v.z = __dmul_rn(e, m);
                v.w = kmcdev::domain_time(EXPO, clkM, clkE, steps, __dmul_rn(N, P.nu));
                const int64_t rec = passes / P.obs_every - 1;
                reinterpret_cast<double4_32a *>(P.obs)[(size_t)rec * P.n_traj + tr] = v;
            }
        }
    };

    // Short visits: the steps of the visits of Sw consecutive schedules are
    // drawn together, lane i holding step i % kp of visit i / kp (kp = k
    // rounded up to a power of two), when Sw Vs kp <= 32; the schedules'
    // domain orders are shuffled one per lane first.
    int kp = 1;
    while (kp < k) kp <<= 1;
    const int Sw = (k >= 1 && kp * Vs <= 32) ? 32 / (kp * Vs) : 0;
    if (Sw > 0) {
        for (int64_t nl = 0; nl < P.n_sched; nl += Sw) {
            const int sw = (int)((P.n_sched - nl < Sw) ? (P.n_sched - nl) : Sw);
            const uint64_t n0 = (uint64_t)(P.sched_begin + nl);
            if (perm) {
                __syncwarp();
                if (lane < sw) shuffle(order + lane * P.ND, n0 + lane);
                __syncwarp();
            }
            uint64_t tgt = ~0ull, V = 1ull << 53;
            {
                const int t = lane / kp, j = lane % kp;
                if (t < sw * Vs && j < k) {
                    const int sv = t / Vs, r = t % Vs;
                    const int p = perm ? r : r / dpp;
                    const int d = perm ? order[sv * P.ND + r] : domain_of_colour(phase_colour(p), r % dpp);
                    draw((uint32_t)j, (uint32_t)d, (n0 + sv) * PART_PHASE_SLOTS + (uint64_t)p, tgt, V);
                }
            }
            uint64_t pm = 0;
            int pe = 0;
            if (EXPO) variate_product(V, kp, pm, pe);
            int t = 0;
            for (int sv = 0; sv < sw; ++sv) {
                for (int p = 0; p < nph; ++p) {
                    const uint64_t np = (n0 + sv) * PART_PHASE_SLOTS + (uint64_t)p;
                    for (int i = 0; i < dpp; ++i, ++t) {
                        const int d = perm ? order[sv * P.ND + p] : domain_of_colour(phase_colour(p), i);
                        int x0, y0;
                        domain_origin(d, x0, y0);
                        if (EXPO)
                            kmcdev::mant_mul(clkM, clkE, __shfl_sync(FULL_WARP, pm, t * kp),
                                             (int64_t)__shfl_sync(FULL_WARP, pe, t * kp));
                        steps += k;
                        events(d, np, x0, y0, DM0 << x0, tgt, t * kp, t * kp + k, 0);
                    }
                    pass_done();
                }
            }
        }
    } else {
        for (int64_t nl = 0; nl < P.n_sched; ++nl) {
            const uint64_t n = (uint64_t)(P.sched_begin + nl);
            if (perm) {
                __syncwarp();
                if (lane == 0) shuffle(order, n);
                __syncwarp();
            }
            for (int p = 0; p < nph; ++p) {
                const uint64_t np = n * PART_PHASE_SLOTS + (uint64_t)p;
                for (int i = 0; i < dpp; ++i) visit(perm ? order[p] : domain_of_colour(phase_colour(p), i), np);
                pass_done();
            }
        }
    }

    // write the lattice back
    int8_t *out = P.spins + (size_t)tr * L * L;
    for (int y = 0; y < L; ++y) {
        const u128 c = row_ld(rows, y);
        for (int x = lane; x < L; x += 32) out[(size_t)y * L + x] = ((c >> x) & 1) ? (int8_t)1 : (int8_t)-1;
    }
    if (lane == 0) {
        P.hash[tr] = H;
        P.clkM[tr] = clkM;
        P.clkE[tr] = clkE;
        P.flips[tr] = flips;
        P.steps[tr] = steps;
        P.t[tr] = kmcdev::domain_time(EXPO, clkM, clkE, steps, __dmul_rn(N, P.nu));
    }
}

} // namespace kmcpart
