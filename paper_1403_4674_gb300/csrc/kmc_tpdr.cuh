// kmc_tpdr.cuh -- one thread per 16x16 or 32x32 domain, state in shared
// memory for the whole launch.
//
// A warp holds 32 domains of one colour, one per lane, and runs their domain
// processes (Sec. 2.2) side by side with no warp-collective operation on the
// step path.  What a lane keeps of its domain, in the warp's shared-memory
// region (word i of lane l at index i*32 + l, so that the 32 lanes' accesses
// to the same word index never share a bank, whatever rows they touch):
//   * the spins, one 32-bit word per row (bit x = column x);
//   * the class counts of every row (App. A: class 5 s + q, q the number of
//     up neighbours), as two words of five 12-bit fields: lo for down spins
//     (q = 0..4), hi for up spins; the same two-word form for blocks of 8
//     rows and for the whole domain;
//   * the halo those counts were built with, the W and E edge columns,
//     counters, the open observation record and the neighbours' ids.
// A step that is a real event finds its class from the cumulative rates, its
// member's block from the block counts, its row from the 8 row counts of the
// block and its column by a bit selection in the row's class mask; the flip
// moves the site and its in-domain neighbours between classes, which changes
// the counts of at most three rows, two blocks and the domain by word-wide
// additions.  A visit first re-counts the rows whose halo bits changed since
// the domain's last visit.
//
// The trajectory is the warp kernel's, decision for decision: step j of
// global phase np draws Philox {j, d, np_lo, np_hi} with the replica seed,
// target = (w0 | w1<<32) >> 1 against R' = sum_c n_c A_c, class = first c
// with target < C_c, member jj = (target - C_{c-1}) / A_c in row-major order.
// Halos come from the neighbours' stamped edge words in global memory (L2),
// as in the other plans.
//
// Scope: palindromic and fixed colour schedules, exponential and expected
// clocks, per-replica k, records at schedule endpoints or every colour pass,
// path scores (GRAD: every lane forms its own domain's FP64 score terms, so
// one FP64 instruction serves up to 32 domains).  Fixed-time visits and
// random colour orders use the warp kernel.
#pragma once

#include "kmc_kernels.cuh"

namespace kmcdev {

template <int LD> struct TpdrLayout {
    static_assert(LD == 16 || LD == 32, "rows of at most 32 sites");
    static constexpr int NB = LD / 8;  // blocks of 8 rows
    static constexpr int CHUNK = 32;   // steps drawn at a time
    static constexpr uint32_t FULL = (LD == 32) ? 0xFFFFFFFFu : ((1u << LD) - 1u);
    // 64-bit words per lane: row counts lo / hi, block counts lo / hi (one
    // spare block each, the target of updates that have no second block),
    // domain counts lo / hi, event hash, real flips, steps, clock mantissa and
    // exponent, open record (record | steps << 32, bonds | mag << 32, clock
    // product mantissa, exponent), the domain's scores d/dbeta, d/dh and
    // those of the open record (FP64 bits), 0 and the cumulative class rates
    // C_c, acceptances A_c, their reciprocals floor((2^64 - 1) / A_c), the
    // step targets of the current chunk (eight spare words past its end hold
    // ~0, a target no rate sum reaches, so that a scan of eight never reads
    // past them)
    static constexpr int ROWLO = 0, ROWHI = LD, BLKLO = 2 * LD, BLKHI = BLKLO + NB + 1, TOTLO = BLKHI + NB + 1,
                         TOTHI = TOTLO + 1, CH = TOTLO + 2, CFL = CH + 1, CST = CH + 2, CCM = CH + 3, CCE = CH + 4,
                         OB0 = CH + 5, OB1 = OB0 + 1, OBM = OB0 + 2, OBE = OB0 + 3, CSB = OB0 + 4, CSH = CSB + 1,
                         OSB = CSB + 2, OSH = CSB + 3, CC = CSB + 4, AT = CC + 11, MR = AT + 10, TG = MR + 10,
                         N64 = TG + CHUNK + 8;
    // 32-bit words per lane: spin rows, the halo the counts hold (N row, S
    // row, W column, E column), the domain's W and E columns, neighbour ids,
    // phase offset f << 16 | step j of each step of the chunk
    static constexpr int SP = 0, HN = LD, HS = LD + 1, HW = LD + 2, HE = LD + 3, CW = LD + 4, CE = LD + 5,
                         NBN = LD + 6, NBS = LD + 7, NBW = LD + 8, NBE = LD + 9, EB = LD + 10, N32 = EB + CHUNK;
    static constexpr int WARP_BYTES = 32 * (8 * N64 + 4 * N32);
};

template <int LD> __host__ __device__ constexpr int tpdr_warp_bytes() { return TpdrLayout<LD>::WARP_BYTES; }

// Bit-sliced count (b2 b1 b0) of the up neighbours of every site of row S,
// with U and D the rows above and below and wb, eb the spins left of column 0
// and right of column LD-1 (halo bits).
template <int LD>
__device__ __forceinline__ void tpdr_planes(uint32_t S, uint32_t U, uint32_t D, uint32_t wb, uint32_t eb,
                                            uint32_t &b0, uint32_t &b1, uint32_t &b2)
{
    constexpr uint32_t FULL = TpdrLayout<LD>::FULL;
    const uint32_t Wn = ((S << 1) | wb) & FULL;       // bit x: the spin at x - 1
    const uint32_t En = (S >> 1) | (eb << (LD - 1));  // bit x: the spin at x + 1
    const uint32_t s1 = U ^ D, c1 = U & D, s2 = Wn ^ En, c2 = Wn & En, t0 = s1 & s2;
    b0 = s1 ^ s2;
    b1 = c1 ^ c2 ^ t0;
    b2 = (c1 & c2) | (c1 & t0) | (c2 & t0);
}

// Sites with exactly q up neighbours.
__device__ __forceinline__ uint32_t tpdr_eq(uint32_t b0, uint32_t b1, uint32_t b2, int q)
{
    return ((q & 4) ? b2 : ~b2) & ((q & 2) ? b1 : ~b1) & ((q & 1) ? b0 : ~b0);
}

// Class counts of one row as two words of five 12-bit fields.
template <int LD>
__device__ __forceinline__ void tpdr_row_counts(uint32_t S, uint32_t U, uint32_t D, uint32_t wb, uint32_t eb,
                                                uint64_t &lo, uint64_t &hi)
{
    constexpr uint32_t FULL = TpdrLayout<LD>::FULL;
    uint32_t b0, b1, b2;
    tpdr_planes<LD>(S, U, D, wb, eb, b0, b1, b2);
    lo = 0;
    hi = 0;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const uint32_t m = tpdr_eq(b0, b1, b2, q) & FULL;
        lo |= (uint64_t)__popc(m & ~S) << (12 * q);
        hi |= (uint64_t)__popc(m & S) << (12 * q);
    }
}

__device__ __forceinline__ uint32_t tpdr_field(uint64_t w, int sh) { return (uint32_t)(w >> sh) & 0xFFFu; }

// Position of the rr-th (0-based) set bit of w; rr < popc(w).  Bit counts
// of 2-bit pairs, nibbles and bytes side by side in one word (the classic
// SWAR popcount steps), byte prefix sums by one multiplication; the byte that
// holds the member is the number of bytes whose prefix is <= rr (a borrow-free
// subtraction per byte, as every prefix is <= 32), then one nibble and one
// pair decide the bit.  Integer ALU only.
__device__ __forceinline__ int tpdr_select(uint32_t w, uint32_t rr)
{
    const uint32_t p1 = w - ((w >> 1) & 0x55555555u);                 // per pair
    const uint32_t p2 = (p1 & 0x33333333u) + ((p1 >> 2) & 0x33333333u); // per nibble
    const uint32_t p4 = (p2 + (p2 >> 4)) & 0x0F0F0F0Fu;                 // per byte
    const uint32_t pre = p4 * 0x01010101u;                              // inclusive byte prefixes
    const uint32_t le = ((((rr * 0x01010101u) | 0x80808080u) - pre) >> 7) & 0x01010101u;
    const int sh = 8 * (int)((le * 0x01010101u) >> 24);                 // 8 x bytes before the member
    rr -= ((pre << 8) >> sh) & 0xFFu;
    int pos = sh;
    const uint32_t cn = (p2 >> pos) & 0xFu;
    if (rr >= cn) { rr -= cn; pos += 4; }
    const uint32_t cp = (p1 >> pos) & 0x3u;
    if (rr >= cp) { rr -= cp; pos += 2; }
    if (rr >= ((w >> pos) & 1u)) pos += 1;
    return pos;
}

// Persistent kernel.  P.slot_g holds 32 domain ids per warp of the grid (one
// colour per warp, 0xFFFFFFFF for an empty lane); the dynamic shared memory
// holds a TpdrLayout region per warp.
template <int LD, bool EXPO, bool GRAD>
__global__ void __launch_bounds__(128) tpdr_kernel(const RunParams P)
{
    using Lay = TpdrLayout<LD>;
    constexpr int NB = Lay::NB;
    constexpr int CHUNK = Lay::CHUNK;
    constexpr uint32_t FULL = Lay::FULL;
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wg = blockIdx.x * (blockDim.x >> 5) + wib;
    uint64_t *w64 = reinterpret_cast<uint64_t *>(smem + (size_t)wib * Lay::WARP_BYTES);
    uint32_t *w32 = reinterpret_cast<uint32_t *>(w64 + 32 * Lay::N64);
    auto at = [&](int i) -> uint64_t & { return w64[i * 32 + lane]; };
    auto at32 = [&](int i) -> uint32_t & { return w32[i * 32 + lane]; };

    const uint32_t g = P.slot_g[(size_t)wg * 32 + lane];
    const bool has = g != 0xFFFFFFFFu;
    const uint32_t g0 = P.slot_g[(size_t)wg * 32];
    if (g0 == 0xFFFFFFFFu) return; // a warp past the plan's last (no barrier below)
    const uint32_t gl = has ? g : g0;
    const uint32_t r = P.dom_rep[gl];
    const uint32_t rbase = P.rep_dom_off[r];
    const uint32_t d = gl - rbase;
    const int k = P.rep_k[r];
    const uint64_t seed = P.rep_seed[r];
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    int wcol;
    {
        // the warp's colour: that of its first domain
        const uint32_t r0 = P.dom_rep[g0];
        const uint32_t d0 = g0 - P.rep_dom_off[r0];
        const uint32_t Dx0 = (uint32_t)P.rep_Dx[r0];
        wcol = (int)((d0 % Dx0) & 1u) | (int)(((d0 / Dx0) & 1u) << 1);
    }
    // the replica's fixed-point acceptances A_c, and M_c = floor((2^64 - 1) /
    // A_c) for the member index (a class of rate 0 is never chosen)
    uint64_t A[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) {
        A[c] = __ldg(&P.rep_A[(size_t)r * 16 + c]);
        at(Lay::AT + c) = A[c];
        at(Lay::MR + c) = A[c] ? ~0ull / A[c] : 0ull;
    }
#pragma unroll
    for (int i = CHUNK; i < CHUNK + 8; ++i) at(Lay::TG + i) = ~0ull;
    at(Lay::CC) = 0;
    // Score constants of the lane's replica (scores only; registers): the
    // two fixed-point words X_c (2^-Q) and Y_c (2^-(Q+18)) of a_c dlog a_c /
    // d(beta, h), and 2^-(Q+4) 2^P, the scale of a state's rounded sum over
    // 2^P (n_d - R).  The per-event terms dlog a_c are read where an event
    // needs them.
    constexpr int PBITS = 63 - 2 * (LD == 16 ? 4 : 5);
    int64_t Xb[10], Xh[10];
    int32_t Yb[10], Yh[10];
    double scaleP = 0.0;
    const double *gr = P.rep_grad + (size_t)r * 32;
    if (GRAD) {
        const int64_t *gf = P.rep_gfix + (size_t)r * GFIX_WORDS;
        const int32_t *gl32 = reinterpret_cast<const int32_t *>(gf);
#pragma unroll
        for (int c = 0; c < 10; ++c) {
            Xb[c] = __ldg(gf + c);
            Xh[c] = __ldg(gf + 10 + c);
            Yb[c] = __ldg(gl32 + 2 * GFIX_YB + c);
            Yh[c] = __ldg(gl32 + 2 * GFIX_YH + c);
        }
        scaleP = __longlong_as_double(__ldg(gf + 20)) * (double)(1ull << PBITS);
    }

    // ---- stage the domain: spins, row / block / domain counts with an all-down halo ----
    if (has) {
        const int Dx = P.rep_Dx[r];
        const int bx = (int)(d % (uint32_t)Dx), by = (int)(d / (uint32_t)Dx);
        at32(Lay::NBN) = rbase + (uint32_t)(((by + Dx - 1) % Dx) * Dx + bx);
        at32(Lay::NBS) = rbase + (uint32_t)(((by + 1) % Dx) * Dx + bx);
        at32(Lay::NBW) = rbase + (uint32_t)(by * Dx + (bx + Dx - 1) % Dx);
        at32(Lay::NBE) = rbase + (uint32_t)(by * Dx + (bx + 1) % Dx);
        uint32_t colW = 0, colE = 0;
        for (int y = 0; y < LD; ++y) {
            const uint32_t Sy = (LD == 32)
                                    ? reinterpret_cast<const uint32_t *>(P.tiles + (size_t)g * (LD * LD / 8))[y]
                                    : (uint32_t)reinterpret_cast<const uint16_t *>(P.tiles + (size_t)g * (LD * LD / 8))[y];
            at32(Lay::SP + y) = Sy;
            colW |= (Sy & 1u) << y;
            colE |= ((Sy >> (LD - 1)) & 1u) << y;
        }
        at32(Lay::CW) = colW;
        at32(Lay::CE) = colE;
        at32(Lay::HN) = 0;
        at32(Lay::HS) = 0;
        at32(Lay::HW) = 0;
        at32(Lay::HE) = 0;
        uint64_t tlo = 0, thi = 0;
        for (int b = 0; b <= NB; ++b) {
            uint64_t blo = 0, bhi = 0;
            for (int i = 0; i < 8 && b < NB; ++i) {
                const int y = 8 * b + i;
                uint64_t lo, hi;
                tpdr_row_counts<LD>(at32(Lay::SP + y), y > 0 ? at32(Lay::SP + (y > 0 ? y - 1 : 0)) : 0u,
                                    y < LD - 1 ? at32(Lay::SP + (y < LD - 1 ? y + 1 : 0)) : 0u, 0u, 0u, lo, hi);
                at(Lay::ROWLO + y) = lo;
                at(Lay::ROWHI + y) = hi;
                blo += lo;
                bhi += hi;
            }
            at(Lay::BLKLO + b) = blo;
            at(Lay::BLKHI + b) = bhi;
            tlo += blo;
            thi += bhi;
        }
        at(Lay::TOTLO) = tlo;
        at(Lay::TOTHI) = thi;
        const uint64_t *ctr = P.dctr + (size_t)g * DCTR_WORDS;
        at(Lay::CH) = ctr[DCTR_HASH];
        at(Lay::CFL) = ctr[DCTR_FLIPS];
        at(Lay::CST) = ctr[DCTR_STEPS];
        at(Lay::CCM) = ctr[DCTR_CLKM];
        at(Lay::CCE) = ctr[DCTR_CLKE];
        at(Lay::OB0) = (uint64_t)NO_RECORD;
        at(Lay::OB1) = 0;
        at(Lay::OBM) = 1ull << 63;
        at(Lay::OBE) = 0;
        at(Lay::CSB) = ctr[DCTR_SB];
        at(Lay::CSH) = ctr[DCTR_SH];
        at(Lay::OSB) = 0; // +0.0
        at(Lay::OSH) = 0;
    }

    // the open record of this lane's domain to its replica's record (records
    // past the launch's last one are dropped)
    auto flush = [&]() {
        const uint64_t o0 = at(Lay::OB0), o1 = at(Lay::OB1);
        const uint32_t o = (uint32_t)o0;
        if (o == NO_RECORD || (int64_t)o >= P.n_obs) return;
        unsigned long long *acc = P.obs_acc + ((size_t)o * P.n_rep + r) * OBS_WORDS;
        const int bonds = (int)(uint32_t)o1, mag = (int)(uint32_t)(o1 >> 32);
        if (bonds != 0) atomicAdd(&acc[0], (unsigned long long)(long long)bonds);
        if (mag != 0) atomicAdd(&acc[1], (unsigned long long)(long long)mag);
        const uint32_t steps = (uint32_t)(o0 >> 32);
        const double dt = EXPO ? domain_time(true, at(Lay::OBM), (int64_t)at(Lay::OBE), 0, P.lambda)
                               : __ddiv_rn((double)steps, P.lambda);
        atomicAdd(reinterpret_cast<double *>(&acc[2]), dt);
        if (GRAD) {
            atomicAdd(reinterpret_cast<double *>(&acc[3]), __longlong_as_double((long long)at(Lay::OSB)));
            atomicAdd(reinterpret_cast<double *>(&acc[4]), __longlong_as_double((long long)at(Lay::OSH)));
        }
    };

    const int nph = (P.schedule == SCHED_PALINDROME) ? 8 : 4;
    unsigned long long polls = 0; // halo re-reads of the warp (profiling)
    bool ok = true;
    uint32_t gc0 = 0, gc1 = 0, gc2 = 0, gc3 = 0; // completed visit groups per colour in this launch
    const uint64_t gp_begin = (uint64_t)P.sched_begin * nph;
    const uint64_t gp_end = (uint64_t)(P.sched_begin + P.n_sched) * nph;
    uint64_t gp = gp_begin;
    while (gp < gp_end) {
        const uint64_t n = gp / nph;
        const int p = (int)(gp % nph);
        const uint64_t np0 = n * 8 + (uint64_t)p;
        const int colour = fixed_colour(P.schedule, p);
        // fuse following phases of the same colour unless an observation intervenes
        int nf = 1;
        while (!P.obs_pass && gp + nf < gp_end) {
            const uint64_t g2 = gp + nf;
            const int p2 = (int)(g2 % nph);
            if (fixed_colour(P.schedule, p2) != colour) break;
            if (p2 == 0) {
                const int64_t nl_prev = (int64_t)(g2 / nph - 1 - (uint64_t)P.sched_begin);
                if (P.obs_every > 0 && ((nl_prev + 1) % P.obs_every) == 0) break;
            }
            ++nf;
        }
        auto gcount = [&](int c) { return c == 0 ? gc0 : c == 1 ? gc1 : c == 2 ? gc2 : gc3; };
        if (colour == wcol && ok) {
            // a neighbour across a row has colour ^ 2, across a column colour ^ 1
            const uint32_t needNS = gcount(colour ^ 2) + (uint32_t)P.debug_extra;
            const uint32_t needWE = gcount(colour ^ 1) + (uint32_t)P.debug_extra;
            const uint32_t after = gcount(colour) + 1;
            const int64_t pass = (int64_t)(gp - gp_begin);
            const int total = has ? nf * k : 0;
            const int smax = (int)__reduce_max_sync(FULL_WARP, (unsigned)total);

            // The draws of the next CHUNK steps (they depend only on the
            // seed, the domain and the step counters): targets and step
            // counters to shared memory, clock variates into the visit's
            // product.  Step s = f k + j of the visit is step j of global
            // phase np0 + f.
            uint32_t jcur = 0, fcur = 0;
            uint64_t vM = 1ull << 63;
            int64_t vE = 0;
            auto draw = [&](int base) {
#pragma unroll 4
                for (int i = 0; i < CHUNK; ++i) {
                    uint64_t t = ~0ull;
                    if (base + i < total) {
                        const uint64_t np = np0 + fcur;
                        const uint4 w = philox4x32_10(
                            make_uint4(jcur, d, (uint32_t)np, (uint32_t)(np >> 32) & 0xFFFFFFu), key);
                        t = (((uint64_t)w.y << 32) | w.x) >> 1;
                        if (EXPO) {
                            // clock variate v = V 2^-53 as a normalised mantissa
                            // m / 2^63 times 2^(10 - z)
                            const uint64_t V = ((((uint64_t)w.w << 32) | w.z) >> 11) + 1ull;
                            const int z = __clzll((long long)V);
                            mant_mul(vM, vE, V << z, (int64_t)(10 - z));
                        }
                        at32(Lay::EB + i) = (fcur << 16) | jcur;
                        if (++jcur == (uint32_t)k) {
                            jcur = 0;
                            ++fcur;
                        }
                    }
                    at(Lay::TG + i) = t;
                }
            };
            draw(0); // before the halo wait

            const uint64_t *pN = P.edges + (size_t)at32(Lay::NBN) * EDGE_WORDS + 2 * EDGE_S;
            const uint64_t *pS = P.edges + (size_t)at32(Lay::NBS) * EDGE_WORDS + 2 * EDGE_N;
            const uint64_t *pW = P.edges + (size_t)at32(Lay::NBW) * EDGE_WORDS + 2 * EDGE_E;
            const uint64_t *pE = P.edges + (size_t)at32(Lay::NBE) * EDGE_WORDS + 2 * EDGE_W;
            uint64_t wN = 0, wS = 0, wW = 0, wE = 0;
            auto current = [&]() {
                return !has || ((uint32_t)(wN >> 32) >= needNS && (uint32_t)(wS >> 32) >= needNS &&
                                (uint32_t)(wW >> 32) >= needWE && (uint32_t)(wE >> 32) >= needWE);
            };
            if (has) {
                wN = ld_volatile_global(pN);
                wS = ld_volatile_global(pS);
                wW = ld_volatile_global(pW);
                wE = ld_volatile_global(pE);
            }
            bool ready = current();
            if (!__all_sync(FULL_WARP, ready)) {
                const uint64_t t0 = global_ns();
                unsigned it = 0;
                while (true) {
                    if (!ready) {
                        wN = ld_volatile_global(pN);
                        wS = ld_volatile_global(pS);
                        wW = ld_volatile_global(pW);
                        wE = ld_volatile_global(pE);
                        ready = current();
                    }
                    ++polls;
                    if (__all_sync(FULL_WARP, ready)) break;
                    if ((++it & 63u) == 0) {
                        const bool late = global_ns() - t0 > P.bar_limit_ns;
                        const bool quit = late || *(volatile int *)P.err != 0;
                        if (__any_sync(FULL_WARP, quit)) {
                            if (late) atomicCAS(P.err, 0, ERR_TIMEOUT);
                            ok = false;
                            break;
                        }
                    }
                }
            }
            if (ok) {
                const uint32_t hN = (uint32_t)wN & FULL, hS = (uint32_t)wS & FULL;
                const uint32_t hW = (uint32_t)wW & FULL, hE = (uint32_t)wE & FULL;
                uint64_t tlo = at(Lay::TOTLO), thi = at(Lay::TOTHI);
                // rows whose halo bits changed since the counts were built
                uint32_t todo = 0;
                if (has) {
                    todo = ((hN != at32(Lay::HN)) ? 1u : 0u) | ((hS != at32(Lay::HS)) ? (1u << (LD - 1)) : 0u) |
                           (hW ^ at32(Lay::HW)) | (hE ^ at32(Lay::HE));
                    at32(Lay::HN) = hN;
                    at32(Lay::HS) = hS;
                    at32(Lay::HW) = hW;
                    at32(Lay::HE) = hE;
                }
                // two rows per round; re-counting a row is idempotent (its counts
                // follow from the current spins and halo), so a lane with one row
                // or none left re-counts row 0 in the free place
                while (__any_sync(FULL_WARP, todo != 0)) {
                    int yy[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        yy[u] = todo ? __ffs(todo) - 1 : 0;
                        todo &= todo - 1;
                    }
                    uint64_t lo[2], hi[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int y = yy[u];
                        const uint32_t Sy = at32(Lay::SP + y);
                        const uint32_t U = (y > 0) ? at32(Lay::SP + (y > 0 ? y - 1 : 0)) : hN;
                        const uint32_t D = (y < LD - 1) ? at32(Lay::SP + (y < LD - 1 ? y + 1 : 0)) : hS;
                        tpdr_row_counts<LD>(Sy, U, D, (hW >> y) & 1u, (hE >> y) & 1u, lo[u], hi[u]);
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int y = yy[u];
                        // differences of packed counts: exact once added to words that hold the old row
                        const uint64_t dlo = lo[u] - at(Lay::ROWLO + y), dhi = hi[u] - at(Lay::ROWHI + y);
                        at(Lay::ROWLO + y) = lo[u];
                        at(Lay::ROWHI + y) = hi[u];
                        at(Lay::BLKLO + (y >> 3)) += dlo;
                        at(Lay::BLKHI + (y >> 3)) += dhi;
                        tlo += dlo;
                        thi += dhi;
                    }
                }
                // cumulative class rates C_c = sum_{c' <= c} n_c' A_c' (registers
                // and, for indexed reads, shared memory); C[9] = R'
                uint64_t C[10];
                auto rates = [&]() {
                    uint64_t W[10];
#pragma unroll
                    for (int c = 0; c < 10; ++c) W[c] = (uint64_t)tpdr_field(c < 5 ? tlo : thi, 12 * (c % 5)) * A[c];
                    // prefix sums in a shallow tree (pairs, then a chain over pairs)
                    const uint64_t s01 = W[0] + W[1], s23 = W[2] + W[3], s45 = W[4] + W[5], s67 = W[6] + W[7],
                                   s89 = W[8] + W[9];
                    C[0] = W[0];
                    C[1] = s01;
                    C[2] = s01 + W[2];
                    C[3] = s01 + s23;
                    C[4] = C[3] + W[4];
                    C[5] = C[3] + s45;
                    C[6] = C[5] + W[6];
                    C[7] = C[5] + s67;
                    C[8] = C[7] + W[8];
                    C[9] = C[7] + s89;
#pragma unroll
                    for (int c = 0; c < 10; ++c) at(Lay::CC + 1 + c) = C[c];
                };
                rates();
                uint64_t H = at(Lay::CH);
                uint32_t colW = at32(Lay::CW), colE = at32(Lay::CE);
                uint64_t flips = 0;
                int dbonds = 0, dmag = 0;

                // Path score of the visit (scores only): a real event of class c
                // adds dlog a_c, a null step dlog(1 - R/n_d) = -sum_c n_c a_c
                // dlog a_c / (n_d - R) (App. A, Eq. Glauber_TM), one value per
                // state, formed only for states that have null steps.  The
                // numerator is an exact integer sum of the two fixed-point words
                // of every class, rounded once to 2^-(Q+4); n_d - R comes from
                // the exact rate sum as (2^63 - R') 2^-P; its reciprocal from the
                // FP32 one x0 = (1 - e)/g by x0 (1 + e + e^2) = (1 - e^3)/g
                // (|e| < 2^-21: truncation 2^-63).  Terms are added in step
                // order, a null run split at the 32-step chunk boundaries.
                double sb = 0.0, sh = 0.0, nbo = 0.0, nho = 0.0;
                bool scored = false;
                auto grad_state = [&]() {
                    int64_t xb = 0, xh = 0;
                    int yb = 0, yh = 0;
#pragma unroll
                    for (int c = 0; c < 10; ++c) {
                        const uint32_t n = tpdr_field(c < 5 ? tlo : thi, 12 * (c % 5));
                        xb += (int64_t)n * Xb[c];
                        xh += (int64_t)n * Xh[c];
                        yb += (int)n * Yb[c];
                        yh += (int)n * Yh[c];
                    }
                    constexpr int SH = GFIX_LO_BITS - GFIX_T_BITS;
                    const int64_t tb = xb * (1ll << GFIX_T_BITS) + (int64_t)((yb + (1 << (SH - 1))) >> SH);
                    const int64_t th = xh * (1ll << GFIX_T_BITS) + (int64_t)((yh + (1 << (SH - 1))) >> SH);
                    const uint64_t gap = (1ull << 63) - C[9];
                    const double gd = __ull2double_rn(gap);
                    const double x0 = (double)__frcp_rn(u64_to_float_rz(gap));
                    const double e = __fma_rn(-gd, x0, 1.0);
                    const double inv = gap ? __fma_rn(x0, __fma_rn(e, e, e), x0) : 0.0;
                    const double w = inv * scaleP;
                    nbo = (double)tb * w;
                    nho = (double)th * w;
                    scored = true;
                };

                bool corrupt = false; // counts and spins disagreed at some event
                for (int base = 0; base < smax; base += CHUNK) {
                    if (base > 0) draw(base);
                    // Each lane jumps from real event to real event of its own
                    // domain (the steps between are null: App. A, the diagonal
                    // 1 - R/n_d); the warp runs as many rounds as its busiest lane.
                    int i = 0;   // this lane's next step, relative to the chunk
                    int pos = 0; // first step of the current run of null steps (scores)
                    while (true) {
                        // the lane's next step with target < R' (targets past its
                        // last step are ~0), four at a time
                        uint64_t tgt = 0;
                        while (i < CHUNK) {
                            const uint64_t R = C[9];
                            uint64_t t[8];
                            unsigned m = 0;
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                t[u] = at(Lay::TG + i + u);
                                m |= (t[u] < R ? 1u : 0u) << u;
                            }
                            if (m) {
                                const int f = __ffs(m) - 1;
                                i += f;
                                // t[f] by selection (no indexed registers)
                                uint64_t q[4];
#pragma unroll
                                for (int u = 0; u < 4; ++u) q[u] = (f & 1) ? t[2 * u + 1] : t[2 * u];
#pragma unroll
                                for (int w = 4, bit = 2; w > 1; w >>= 1, bit <<= 1)
#pragma unroll
                                    for (int u = 0; u < w / 2; ++u) q[u] = (f & bit) ? q[2 * u + 1] : q[2 * u];
                                tgt = q[0];
                                break;
                            }
                            i += 8;
                        }
                        const bool ev = i < CHUNK;
                        if (GRAD) {
                            // the null steps before this event, or up to the chunk's
                            // (or the visit's) end, all in the current state
                            const int end = ev ? i : min(CHUNK, total - base);
                            if (end > pos) {
                                if (!scored) grad_state();
                                const double q = (double)(end - pos);
                                sb -= q * nbo;
                                sh -= q * nho;
                            }
                            pos = ev ? i + 1 : CHUNK;
                        }
                        if (!__any_sync(FULL_WARP, ev)) break;
                        if (!ev) continue;
                        const uint32_t eb = at32(Lay::EB + i);
                        ++i;
                        const uint64_t np = np0 + (eb >> 16);
                        const uint32_t j = eb & 0xFFFFu;
                        // class: the first c with tgt < C_c
                        int c = 0;
#pragma unroll
                        for (int cc = 0; cc < 9; ++cc) c += (tgt >= C[cc]) ? 1 : 0;
                        if (GRAD) {
                            // dlog a_c / d(beta, h) of the chosen class
                            sb += __ldg(gr + 10 + c);
                            sh += __ldg(gr + 20 + c);
                        }
                        const uint64_t Cprev = at(Lay::CC + c); // C_{c-1}, 0 for c = 0
                        const uint64_t Ac = at(Lay::AT + c);
                        const uint64_t Mc = at(Lay::MR + c);
                        // exact jj = floor((tgt - C_{c-1}) / A_c) < n_c <= 1024: with
                        // M_c = floor((2^64 - 1) / A_c) and x < 2^63, the high word
                        // of x M_c is jj or jj - 1, and one integer comparison
                        // decides which
                        const uint64_t x = tgt - Cprev;
                        uint32_t jj = (uint32_t)__umul64hi(x, Mc);
                        jj = (x - (uint64_t)jj * Ac >= Ac) ? jj + 1u : jj;
                        const bool up = c >= 5;
                        const int qc = up ? c - 5 : c;
                        const int sh = 12 * qc;
                        // the member's block of 8 rows: the first whose running count exceeds jj
                        const int bw = up ? Lay::BLKHI : Lay::BLKLO;
                        int bsel = 0;
                        uint32_t before = 0;
                        {
                            uint32_t acc = 0;
#pragma unroll
                            for (int b = 0; b < NB - 1; ++b) {
                                acc += tpdr_field(at(bw + b), sh);
                                const bool past = jj >= acc;
                                bsel += past ? 1 : 0;
                                before = past ? acc : before;
                            }
                        }
                        // its row among the block's 8
                        const int rw = (up ? Lay::ROWHI : Lay::ROWLO) + 8 * bsel;
                        const uint32_t rem = jj - before;
                        int yi = 0;
                        uint32_t rbefore = 0;
                        {
                            uint32_t f[7], pf[7];
#pragma unroll
                            for (int q = 0; q < 7; ++q) f[q] = tpdr_field(at(rw + q), sh);
                            // inclusive prefix sums in a shallow tree
                            pf[0] = f[0];
                            pf[1] = f[0] + f[1];
                            pf[2] = pf[1] + f[2];
                            pf[3] = pf[1] + (f[2] + f[3]);
                            pf[4] = pf[3] + f[4];
                            pf[5] = pf[3] + (f[4] + f[5]);
                            pf[6] = pf[5] + f[6];
#pragma unroll
                            for (int q = 0; q < 7; ++q) {
                                const bool past = rem >= pf[q];
                                yi += past ? 1 : 0;
                                rbefore = max(rbefore, past ? pf[q] : 0u);
                            }
                        }
                        const int y = 8 * bsel + yi;
                        const uint32_t rr = rem - rbefore;
                        const bool hasN = y > 0, hasS = y < LD - 1;
                        const int yN = hasN ? y - 1 : y, yS = hasS ? y + 1 : y;
                        const uint32_t Sy = at32(Lay::SP + y);
                        const uint32_t Su = hasN ? at32(Lay::SP + yN) : hN;
                        const uint32_t Sd = hasS ? at32(Lay::SP + yS) : hS;
                        const uint32_t Suu = (y > 1) ? at32(Lay::SP + (y > 1 ? y - 2 : 0)) : hN;
                        const uint32_t Sdd = (y < LD - 2) ? at32(Lay::SP + (y < LD - 2 ? y + 2 : 0)) : hS;
                        const uint64_t rYlo = at(Lay::ROWLO + y), rYhi = at(Lay::ROWHI + y);
                        const uint64_t rNlo = at(Lay::ROWLO + yN), rNhi = at(Lay::ROWHI + yN);
                        const uint64_t rSlo = at(Lay::ROWLO + yS), rShi = at(Lay::ROWHI + yS);
                        uint32_t b0, b1, b2;
                        tpdr_planes<LD>(Sy, Su, Sd, (hW >> y) & 1u, (hE >> y) & 1u, b0, b1, b2);
                        const uint32_t mask = tpdr_eq(b0, b1, b2, qc) & (up ? Sy : ~Sy) & FULL;
                        // counts and spins disagree (never, unless the state is
                        // corrupt): recorded, reported after the visit; every
                        // index below stays within the domain's rows
                        const bool bad = rr >= (uint32_t)__popc(mask);
                        const int col = tpdr_select(mask, rr) & 31;
                        const uint32_t bit = 1u << col;
                        // the site moves from (s, q) to (1 - s, q); each in-domain
                        // neighbour from (s', q') to (s', q' + delta)
                        const bool hasW = col > 0, hasE = col < LD - 1;
                        const int xw = hasW ? col - 1 : col, xe = hasE ? col + 1 : col;
                        auto qat = [&](int xx) {
                            return (int)((b0 >> xx) & 1u) + 2 * (int)((b1 >> xx) & 1u) + 4 * (int)((b2 >> xx) & 1u);
                        };
                        const int qW = qat(xw), qE = qat(xe);
                        const int sW = (int)((Sy >> xw) & 1u), sE = (int)((Sy >> xe) & 1u);
                        const int qN = (int)((Suu >> col) & 1u) + (int)((Sy >> col) & 1u) +
                                       (int)(hasW ? (Su >> xw) & 1u : (hW >> yN) & 1u) +
                                       (int)(hasE ? (Su >> xe) & 1u : (hE >> yN) & 1u);
                        const int qS = (int)((Sdd >> col) & 1u) + (int)((Sy >> col) & 1u) +
                                       (int)(hasW ? (Sd >> xw) & 1u : (hW >> yS) & 1u) +
                                       (int)(hasE ? (Sd >> xe) & 1u : (hE >> yS) & 1u);
                        const int sN = (int)((Su >> col) & 1u), sS = (int)((Sd >> col) & 1u);
                        const bool gain = !up; // the neighbours gain an up neighbour
                        uint64_t dYlo, dYhi, dNlo = 0, dNhi = 0, dSlo = 0, dShi = 0;
                        {
                            const uint64_t v = 1ull << sh;
                            dYlo = up ? v : 0ull - v;
                            dYhi = up ? 0ull - v : v;
                        }
                        auto move = [&](uint64_t &lo, uint64_t &hi, bool in, int sn, int qn) {
                            const int qq = gain ? qn : max(qn - 1, 0);
                            const uint64_t m0 = in ? (0xFFFull << (12 * qq)) : 0ull;
                            const uint64_t mv = gain ? m0 : 0ull - m0;
                            lo += sn ? 0ull : mv;
                            hi += sn ? mv : 0ull;
                        };
                        move(dYlo, dYhi, hasW, sW, qW);
                        move(dYlo, dYhi, hasE, sE, qE);
                        move(dNlo, dNhi, hasN, sN, qN);
                        move(dSlo, dShi, hasS, sS, qS);
                        // the block of row y, and the other block a neighbour row
                        // may lie in (the spare block when there is none)
                        const int by = y >> 3;
                        const bool crossN = (yN >> 3) != by, crossS = (yS >> 3) != by;
                        const int bo = crossN ? (yN >> 3) : crossS ? (yS >> 3) : NB;
                        const uint64_t bYlo = dYlo + (crossN ? 0ull : dNlo) + (crossS ? 0ull : dSlo);
                        const uint64_t bYhi = dYhi + (crossN ? 0ull : dNhi) + (crossS ? 0ull : dShi);
                        const uint64_t bOlo = (crossN ? dNlo : 0ull) + (crossS ? dSlo : 0ull);
                        const uint64_t bOhi = (crossN ? dNhi : 0ull) + (crossS ? dShi : 0ull);
                        const uint64_t kYlo = at(Lay::BLKLO + by), kYhi = at(Lay::BLKHI + by);
                        const uint64_t kOlo = at(Lay::BLKLO + bo), kOhi = at(Lay::BLKHI + bo);
                        at32(Lay::SP + y) = Sy ^ bit;
                        // the neighbour rows first: without one (yN or yS = y) its
                        // store writes row y's old words, which row y's store then
                        // replaces
                        at(Lay::ROWLO + yN) = rNlo + dNlo;
                        at(Lay::ROWHI + yN) = rNhi + dNhi;
                        at(Lay::ROWLO + yS) = rSlo + dSlo;
                        at(Lay::ROWHI + yS) = rShi + dShi;
                        at(Lay::ROWLO + y) = rYlo + dYlo;
                        at(Lay::ROWHI + y) = rYhi + dYhi;
                        at(Lay::BLKLO + by) = kYlo + bYlo;
                        at(Lay::BLKHI + by) = kYhi + bYhi;
                        at(Lay::BLKLO + bo) = kOlo + bOlo;
                        at(Lay::BLKHI + bo) = kOhi + bOhi;
                        tlo += dYlo + dNlo + dSlo;
                        thi += dYhi + dNhi + dShi;
                        colW ^= (col == 0) ? (1u << y) : 0u;
                        colE ^= (col == LD - 1) ? (1u << y) : 0u;
                        H = (H ^ ((np << 32) | ((uint64_t)j << 16) | (uint64_t)(y * LD + col))) * HASH_PRIME;
                        ++flips;
                        // flipping spin s with neighbour sum 2 qc - 4 changes the bond
                        // sum by -2 s (2 qc - 4) and the magnetisation by -2 s
                        const int sgn = up ? 1 : -1;
                        dbonds -= 2 * sgn * (2 * qc - 4);
                        dmag -= 2 * sgn;
                        rates();
                        scored = false;
                        corrupt |= bad;
                    }
                }
                if (corrupt) atomicCAS(P.err, 0, ERR_INTERNAL);
                if (has) {
                    // edges first (neighbours wait for them), then counters and record
                    uint64_t *ew = P.edges + (size_t)gl * EDGE_WORDS;
                    const uint64_t cnt = (uint64_t)after << 32;
                    st_cg(ew + 2 * EDGE_N, cnt | at32(Lay::SP + 0));
                    st_cg(ew + 2 * EDGE_S, cnt | at32(Lay::SP + LD - 1));
                    st_cg(ew + 2 * EDGE_W, cnt | colW);
                    st_cg(ew + 2 * EDGE_E, cnt | colE);
                    at(Lay::TOTLO) = tlo;
                    at(Lay::TOTHI) = thi;
                    at32(Lay::CW) = colW;
                    at32(Lay::CE) = colE;
                    at(Lay::CH) = H;
                    at(Lay::CFL) += flips;
                    at(Lay::CST) += (uint64_t)total;
                    if (GRAD) {
                        at(Lay::CSB) = (uint64_t)__double_as_longlong(__longlong_as_double((long long)at(Lay::CSB)) + sb);
                        at(Lay::CSH) = (uint64_t)__double_as_longlong(__longlong_as_double((long long)at(Lay::CSH)) + sh);
                    }
                    if (EXPO) {
                        // the domain clock takes the visit's product
                        uint64_t m = at(Lay::CCM);
                        int64_t e = (int64_t)at(Lay::CCE);
                        mant_mul(m, e, vM, vE);
                        at(Lay::CCM) = m;
                        at(Lay::CCE) = (uint64_t)e;
                    }
                    if (P.n_obs > 0) {
                        // the visit's changes belong to the first record at or after its pass
                        const int64_t o = (P.obs_pass ? pass : pass / nph) / P.obs_every;
                        if ((int64_t)(uint32_t)at(Lay::OB0) != o) {
                            flush();
                            at(Lay::OB0) = (uint64_t)(uint32_t)o;
                            at(Lay::OB1) = 0;
                            at(Lay::OBM) = 1ull << 63;
                            at(Lay::OBE) = 0;
                            at(Lay::OSB) = 0;
                            at(Lay::OSH) = 0;
                        }
                        const uint64_t o0 = at(Lay::OB0), o1 = at(Lay::OB1);
                        const uint32_t steps = (uint32_t)(o0 >> 32) + (uint32_t)total;
                        const int bonds = (int)(uint32_t)o1 + dbonds, mag = (int)(uint32_t)(o1 >> 32) + dmag;
                        at(Lay::OB0) = (uint64_t)(uint32_t)o0 | ((uint64_t)steps << 32);
                        at(Lay::OB1) = (uint64_t)(uint32_t)bonds | ((uint64_t)(uint32_t)mag << 32);
                        if (EXPO) {
                            uint64_t m = at(Lay::OBM);
                            int64_t e = (int64_t)at(Lay::OBE);
                            mant_mul(m, e, vM, vE);
                            at(Lay::OBM) = m;
                            at(Lay::OBE) = (uint64_t)e;
                        }
                        if (GRAD) {
                            at(Lay::OSB) = (uint64_t)__double_as_longlong(__longlong_as_double((long long)at(Lay::OSB)) + sb);
                            at(Lay::OSH) = (uint64_t)__double_as_longlong(__longlong_as_double((long long)at(Lay::OSH)) + sh);
                        }
                    }
                }
            }
        }
        if (colour == 0) ++gc0;
        else if (colour == 1) ++gc1;
        else if (colour == 2) ++gc2;
        else ++gc3;
        gp += (uint64_t)nf;
    }
    if (P.polls && lane == 0 && polls != 0) atomicAdd(P.polls, polls);
    if (!ok || *(volatile int *)P.err != 0) return;
    // write the domain back: tile, counters, open record
    if (has) {
        for (int y = 0; y < LD; ++y) {
            if (LD == 32) reinterpret_cast<uint32_t *>(P.tiles + (size_t)g * (LD * LD / 8))[y] = at32(Lay::SP + y);
            else reinterpret_cast<uint16_t *>(P.tiles + (size_t)g * (LD * LD / 8))[y] = (uint16_t)at32(Lay::SP + y);
        }
        uint64_t *ctr = P.dctr + (size_t)g * DCTR_WORDS;
        ctr[DCTR_HASH] = at(Lay::CH);
        ctr[DCTR_FLIPS] = at(Lay::CFL);
        ctr[DCTR_STEPS] = at(Lay::CST);
        ctr[DCTR_CLKM] = at(Lay::CCM);
        ctr[DCTR_CLKE] = at(Lay::CCE);
        if (GRAD) {
            ctr[DCTR_SB] = at(Lay::CSB);
            ctr[DCTR_SH] = at(Lay::CSH);
        }
        if (P.n_obs > 0) flush();
    }
}

} // namespace kmcdev
