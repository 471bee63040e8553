// kmc_tpdr64.cuh -- one thread per 64x64 domain, state in shared memory for
// the whole launch.
//
// The 64x64 form of the shared-memory thread kernel (kmc_tpdr.cuh): a warp
// holds 32 domains of one colour, one per lane, and runs their domain
// processes (Sec. 2.2) side by side with no warp-collective operation on the
// step path.  A 64x64 domain's per-row class counts would not leave room for
// the 16,384 domains of an 8192^2 lattice in the GPU's shared memory, so a
// lane keeps only (word i of lane l at index i*32 + l, conflict-free):
//   * the spins, one 64-bit word per row (bit x = column x);
//   * the class counts (App. A: class 5 s + q, q the number of up
//     neighbours) of every block of 8 rows and of each half of the domain
//     (blocks 0-3 and 4-7), as two words of five 12-bit fields, lo for down
//     spins and hi for up spins (a block holds at most 512 sites, a half
//     2048; the domain's 4096 would not fit a field, so the rates add the
//     two halves);
//   * the halo those counts were built with, the W and E edge columns,
//     counters, the open observation record and the neighbours' ids.
// A real event finds its class from the cumulative rates, its member's half
// and block from the half and block counts, and its row by counting the
// class in the block's 8 rows from their spins (the count planes of a row
// are a dozen bit operations); the flip moves the site and its in-domain
// neighbours between classes, which changes at most two blocks' and two
// halves' counts by word-wide additions.  A visit first re-counts, for the
// rows whose halo bits changed since the domain's last visit, the difference
// between their counts under the new and the old halo.
//
// The trajectory is the warp kernel's, decision for decision (same draws,
// classes, member order and event hash).  Edge words follow the lattice
// layout: rows as plain 64-bit masks, columns with row y at bit
// (y % 2) * 32 + y / 2, split into two stamped 32-bit halves.
//
// Scope: palindromic and fixed colour schedules, exponential and expected
// clocks, per-replica k, records at schedule endpoints or every colour pass;
// no scores.  Other runs use the warp kernel.
#pragma once

#include "kmc_tpdr.cuh"

namespace kmcdev {

struct Tpdr64Layout {
    static constexpr int LD = 64, NB = 8, CHUNK = 32;
    // 64-bit words per lane: spin rows, block counts lo / hi (one spare block
    // each, the target of updates that have no second block), half counts lo
    // / hi (one spare each), the halo the counts hold (N row, S row, W and E
    // columns, bit y = row y), the domain's W and E columns (bit y = row y),
    // event hash, real flips, steps, clock mantissa and exponent, open record
    // (record | steps << 32, bonds | mag << 32, clock product mantissa,
    // exponent), 0 and the cumulative class rates C_c, acceptances A_c, their
    // reciprocals floor((2^64 - 1) / A_c), the step targets of the current
    // chunk (eight spare words past its end hold ~0, a target no rate sum
    // reaches)
    static constexpr int SP = 0, BLKLO = 64, BLKHI = BLKLO + NB + 1, HFLO = BLKHI + NB + 1, HFHI = HFLO + 3,
                         HN = HFHI + 3, HS = HN + 1, HW = HN + 2, HE = HN + 3, CW = HN + 4, CE = HN + 5,
                         CH = CE + 1, CFL = CH + 1, CST = CH + 2, CCM = CH + 3, CCE = CH + 4, OB0 = CH + 5,
                         OB1 = OB0 + 1, OBM = OB0 + 2, OBE = OB0 + 3, CC = OB0 + 4, AT = CC + 11, MR = AT + 10,
                         TG = MR + 10, N64 = TG + CHUNK + 8;
    // 32-bit words per lane: neighbour ids, phase offset f << 16 | step j of
    // each step of the chunk
    static constexpr int NBN = 0, NBS = 1, NBW = 2, NBE = 3, EB = 4, N32 = EB + CHUNK;
    static constexpr int WARP_BYTES = 32 * (8 * N64 + 4 * N32);
};

__host__ __device__ constexpr int tpdr64_warp_bytes() { return Tpdr64Layout::WARP_BYTES; }

// Bit-sliced count (b2 b1 b0) of the up neighbours of every site of row S,
// with U and D the rows above and below and wb, eb the spins left of column
// 0 and right of column 63 (halo bits, 0 or 1).
__device__ __forceinline__ void t64_planes(uint64_t S, uint64_t U, uint64_t D, uint64_t wb, uint64_t eb,
                                           uint64_t &b0, uint64_t &b1, uint64_t &b2)
{
    const uint64_t Wn = (S << 1) | wb;         // bit x: the spin at x - 1
    const uint64_t En = (S >> 1) | (eb << 63); // bit x: the spin at x + 1
    const uint64_t s1 = U ^ D, c1 = U & D, s2 = Wn ^ En, c2 = Wn & En, t0 = s1 & s2;
    b0 = s1 ^ s2;
    b1 = c1 ^ c2 ^ t0;
    b2 = (c1 & c2) | (c1 & t0) | (c2 & t0);
}

__device__ __forceinline__ uint64_t t64_eq(uint64_t b0, uint64_t b1, uint64_t b2, int q)
{
    return ((q & 4) ? b2 : ~b2) & ((q & 2) ? b1 : ~b1) & ((q & 1) ? b0 : ~b0);
}

// Class counts of one row as two words of five 12-bit fields.
__device__ __forceinline__ void t64_row_counts(uint64_t S, uint64_t U, uint64_t D, uint64_t wb, uint64_t eb,
                                               uint64_t &lo, uint64_t &hi)
{
    uint64_t b0, b1, b2;
    t64_planes(S, U, D, wb, eb, b0, b1, b2);
    lo = 0;
    hi = 0;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const uint64_t m = t64_eq(b0, b1, b2, q);
        lo |= (uint64_t)__popcll(m & ~S) << (12 * q);
        hi |= (uint64_t)__popcll(m & S) << (12 * q);
    }
}

// Bits of a 32-bit word to the even bits of a 64-bit word, and back.
__device__ __forceinline__ uint64_t t64_spread(uint32_t v)
{
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}
__device__ __forceinline__ uint32_t t64_compact(uint64_t x)
{
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
    x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
    x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
    return (uint32_t)x;
}
// A column from the edge layout (row y at bit (y % 2) * 32 + y / 2) to bit y
// = row y, and back.
__device__ __forceinline__ uint64_t t64_col_from_edge(uint64_t w)
{
    return t64_spread((uint32_t)w) | (t64_spread((uint32_t)(w >> 32)) << 1);
}
__device__ __forceinline__ uint64_t t64_col_to_edge(uint64_t c)
{
    return (uint64_t)t64_compact(c) | ((uint64_t)t64_compact(c >> 1) << 32);
}

// Persistent kernel.  P.slot_g holds 32 domain ids per warp of the grid (one
// colour per warp, 0xFFFFFFFF for an empty lane); the dynamic shared memory
// holds a Tpdr64Layout region per warp.
template <bool EXPO>
__global__ void __launch_bounds__(128) tpdr64_kernel(const RunParams P)
{
    using Lay = Tpdr64Layout;
    constexpr int LD = 64;
    constexpr int NB = Lay::NB;
    constexpr int CHUNK = Lay::CHUNK;
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

    // ---- stage the domain: spins, block / half counts with an all-down halo ----
    if (has) {
        const int Dx = P.rep_Dx[r];
        const int bx = (int)(d % (uint32_t)Dx), by = (int)(d / (uint32_t)Dx);
        at32(Lay::NBN) = rbase + (uint32_t)(((by + Dx - 1) % Dx) * Dx + bx);
        at32(Lay::NBS) = rbase + (uint32_t)(((by + 1) % Dx) * Dx + bx);
        at32(Lay::NBW) = rbase + (uint32_t)(by * Dx + (bx + Dx - 1) % Dx);
        at32(Lay::NBE) = rbase + (uint32_t)(by * Dx + (bx + 1) % Dx);
        const uint64_t *tile = reinterpret_cast<const uint64_t *>(P.tiles + (size_t)g * (LD * LD / 8));
        uint64_t colW = 0, colE = 0;
        for (int y = 0; y < LD; ++y) {
            const uint64_t Sy = tile[y];
            at(Lay::SP + y) = Sy;
            colW |= (Sy & 1ull) << y;
            colE |= (Sy >> 63) << y;
        }
        at(Lay::CW) = colW;
        at(Lay::CE) = colE;
        at(Lay::HN) = 0;
        at(Lay::HS) = 0;
        at(Lay::HW) = 0;
        at(Lay::HE) = 0;
        uint64_t hlo[2] = {0, 0}, hhi[2] = {0, 0};
        for (int b = 0; b < NB; ++b) {
            uint64_t blo = 0, bhi = 0;
            for (int i = 0; i < 8; ++i) {
                const int y = 8 * b + i;
                uint64_t lo, hi;
                t64_row_counts(at(Lay::SP + y), y > 0 ? at(Lay::SP + (y > 0 ? y - 1 : 0)) : 0ull,
                               y < LD - 1 ? at(Lay::SP + (y < LD - 1 ? y + 1 : 0)) : 0ull, 0ull, 0ull, lo, hi);
                blo += lo;
                bhi += hi;
            }
            at(Lay::BLKLO + b) = blo;
            at(Lay::BLKHI + b) = bhi;
            hlo[b >> 2] += blo;
            hhi[b >> 2] += bhi;
        }
        at(Lay::BLKLO + NB) = 0;
        at(Lay::BLKHI + NB) = 0;
        for (int hf = 0; hf < 2; ++hf) {
            at(Lay::HFLO + hf) = hlo[hf];
            at(Lay::HFHI + hf) = hhi[hf];
        }
        at(Lay::HFLO + 2) = 0;
        at(Lay::HFHI + 2) = 0;
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

            // the neighbours' edges: two stamped words (halves) each
            const uint64_t *pN = P.edges + (size_t)at32(Lay::NBN) * EDGE_WORDS + 2 * EDGE_S;
            const uint64_t *pS = P.edges + (size_t)at32(Lay::NBS) * EDGE_WORDS + 2 * EDGE_N;
            const uint64_t *pW = P.edges + (size_t)at32(Lay::NBW) * EDGE_WORDS + 2 * EDGE_E;
            const uint64_t *pE = P.edges + (size_t)at32(Lay::NBE) * EDGE_WORDS + 2 * EDGE_W;
            uint64_t e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            auto reread = [&]() {
                e[0] = ld_volatile_global(pN);
                e[1] = ld_volatile_global(pN + 1);
                e[2] = ld_volatile_global(pS);
                e[3] = ld_volatile_global(pS + 1);
                e[4] = ld_volatile_global(pW);
                e[5] = ld_volatile_global(pW + 1);
                e[6] = ld_volatile_global(pE);
                e[7] = ld_volatile_global(pE + 1);
            };
            auto current = [&]() {
                if (!has) return true;
                bool c = true;
#pragma unroll
                for (int i = 0; i < 8; ++i) c = c && (uint32_t)(e[i] >> 32) >= (i < 4 ? needNS : needWE);
                return c;
            };
            if (has) reread();
            bool ready = current();
            if (!__all_sync(FULL_WARP, ready)) {
                const uint64_t t0 = global_ns();
                unsigned it = 0;
                while (true) {
                    if (!ready) {
                        reread();
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
                auto join = [&](int i) { return (uint64_t)(uint32_t)e[i] | ((uint64_t)(uint32_t)e[i + 1] << 32); };
                const uint64_t hN = join(0), hS = join(2);
                const uint64_t hW = t64_col_from_edge(join(4)), hE = t64_col_from_edge(join(6));
                uint64_t h0lo = at(Lay::HFLO), h0hi = at(Lay::HFHI), h1lo = at(Lay::HFLO + 1), h1hi = at(Lay::HFHI + 1);
                // rows whose halo bits changed since the counts were built: each
                // row's counts under the new halo less those under the old one
                uint64_t todo = 0;
                const uint64_t oN = at(Lay::HN), oS = at(Lay::HS), oW = at(Lay::HW), oE = at(Lay::HE);
                if (has) {
                    todo = ((hN != oN) ? 1ull : 0ull) | ((hS != oS) ? (1ull << (LD - 1)) : 0ull) | (hW ^ oW) | (hE ^ oE);
                    at(Lay::HN) = hN;
                    at(Lay::HS) = hS;
                    at(Lay::HW) = hW;
                    at(Lay::HE) = hE;
                }
                while (__any_sync(FULL_WARP, todo != 0)) {
                    if (todo) {
                        const int y = __ffsll((long long)todo) - 1;
                        todo &= todo - 1;
                        const uint64_t Sy = at(Lay::SP + y);
                        const uint64_t U = (y > 0) ? at(Lay::SP + (y > 0 ? y - 1 : 0)) : hN;
                        const uint64_t D = (y < LD - 1) ? at(Lay::SP + (y < LD - 1 ? y + 1 : 0)) : hS;
                        const uint64_t Uo = (y > 0) ? U : oN, Do = (y < LD - 1) ? D : oS;
                        uint64_t lo, hi, olo, ohi;
                        t64_row_counts(Sy, U, D, (hW >> y) & 1ull, (hE >> y) & 1ull, lo, hi);
                        t64_row_counts(Sy, Uo, Do, (oW >> y) & 1ull, (oE >> y) & 1ull, olo, ohi);
                        // differences of packed counts: exact once added to words that hold the old row
                        const uint64_t dlo = lo - olo, dhi = hi - ohi;
                        at(Lay::BLKLO + (y >> 3)) += dlo;
                        at(Lay::BLKHI + (y >> 3)) += dhi;
                        const bool second = y >= 32;
                        h0lo += second ? 0ull : dlo;
                        h0hi += second ? 0ull : dhi;
                        h1lo += second ? dlo : 0ull;
                        h1hi += second ? dhi : 0ull;
                    }
                }
                // cumulative class rates C_c = sum_{c' <= c} n_c' A_c' (registers
                // and, for indexed reads, shared memory); C[9] = R'.  A class's
                // count is the sum of the two halves' fields.
                uint64_t C[10];
                auto rates = [&]() {
                    uint64_t W[10];
#pragma unroll
                    for (int c = 0; c < 10; ++c) {
                        const int sh = 12 * (c % 5);
                        const uint32_t nc = tpdr_field(c < 5 ? h0lo : h0hi, sh) + tpdr_field(c < 5 ? h1lo : h1hi, sh);
                        W[c] = (uint64_t)nc * A[c];
                    }
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
                uint64_t colW = at(Lay::CW), colE = at(Lay::CE);
                uint64_t flips = 0;
                int dbonds = 0, dmag = 0;
                bool corrupt = false; // counts and spins disagreed at some event

                for (int base = 0; base < smax; base += CHUNK) {
                    if (base > 0) draw(base);
                    // Each lane jumps from real event to real event of its own
                    // domain (the steps between are null: App. A, the diagonal
                    // 1 - R/n_d); the warp runs as many rounds as its busiest lane.
                    int i = 0; // this lane's next step, relative to the chunk
                    while (true) {
                        // the lane's next step with target < R' (targets past its
                        // last step are ~0), eight at a time
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
                                const uint64_t q0 = (f & 1) ? t[1] : t[0], q1 = (f & 1) ? t[3] : t[2];
                                const uint64_t q2 = (f & 1) ? t[5] : t[4], q3 = (f & 1) ? t[7] : t[6];
                                const uint64_t r0 = (f & 2) ? q1 : q0, r1 = (f & 2) ? q3 : q2;
                                tgt = (f & 4) ? r1 : r0;
                                break;
                            }
                            i += 8;
                        }
                        const bool ev = i < CHUNK;
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
                        const uint64_t Cprev = at(Lay::CC + c); // C_{c-1}, 0 for c = 0
                        const uint64_t Ac = at(Lay::AT + c);
                        const uint64_t Mc = at(Lay::MR + c);
                        // exact jj = floor((tgt - C_{c-1}) / A_c) < n_c <= 4096: with
                        // M_c = floor((2^64 - 1) / A_c) and x < 2^63, the high word
                        // of x M_c is jj or jj - 1, and one integer comparison
                        // decides which
                        const uint64_t x = tgt - Cprev;
                        uint32_t jj = (uint32_t)__umul64hi(x, Mc);
                        jj = (x - (uint64_t)jj * Ac >= Ac) ? jj + 1u : jj;
                        const bool up = c >= 5;
                        const int qc = up ? c - 5 : c;
                        const int sh = 12 * qc;
                        // the member's half, then its block of 8 rows among the half's 4
                        const uint32_t n0 = tpdr_field(up ? h0hi : h0lo, sh);
                        const bool second = jj >= n0;
                        const uint32_t rem0 = second ? jj - n0 : jj;
                        const int bw = (up ? Lay::BLKHI : Lay::BLKLO) + (second ? 4 : 0);
                        int bsel = 0;
                        uint32_t before = 0;
                        {
                            uint32_t acc = 0;
#pragma unroll
                            for (int b = 0; b < 3; ++b) {
                                acc += tpdr_field(at(bw + b), sh);
                                const bool past = rem0 >= acc;
                                bsel += past ? 1 : 0;
                                before = past ? acc : before;
                            }
                        }
                        const int blk = (second ? 4 : 0) + bsel;
                        const uint32_t rem = rem0 - before;
                        // its row among the block's 8: the class counted in each row
                        // from the spins (rows y0 - 1 .. y0 + 8, the halo rows at the
                        // domain's edges)
                        const int y0 = 8 * blk;
                        uint64_t Rw[10];
                        Rw[0] = (y0 > 0) ? at(Lay::SP + (y0 > 0 ? y0 - 1 : 0)) : hN;
#pragma unroll
                        for (int u = 0; u < 8; ++u) Rw[1 + u] = at(Lay::SP + y0 + u);
                        Rw[9] = (y0 + 8 < LD) ? at(Lay::SP + (y0 + 8 < LD ? y0 + 8 : 0)) : hS;
                        uint64_t mk[8];
                        uint32_t f[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int yy = y0 + u;
                            uint64_t b0, b1, b2;
                            t64_planes(Rw[1 + u], Rw[u], Rw[2 + u], (hW >> yy) & 1ull, (hE >> yy) & 1ull, b0, b1, b2);
                            mk[u] = t64_eq(b0, b1, b2, qc) & (up ? Rw[1 + u] : ~Rw[1 + u]);
                            f[u] = (uint32_t)__popcll(mk[u]);
                        }
                        uint32_t pf[7];
                        pf[0] = f[0];
                        pf[1] = f[0] + f[1];
                        pf[2] = pf[1] + f[2];
                        pf[3] = pf[1] + (f[2] + f[3]);
                        pf[4] = pf[3] + f[4];
                        pf[5] = pf[3] + (f[4] + f[5]);
                        pf[6] = pf[5] + f[6];
                        int yi = 0;
                        uint32_t rbefore = 0;
#pragma unroll
                        for (int q = 0; q < 7; ++q) {
                            const bool past = rem >= pf[q];
                            yi += past ? 1 : 0;
                            rbefore = max(rbefore, past ? pf[q] : 0u);
                        }
                        const int y = y0 + yi;
                        const uint32_t rr = rem - rbefore;
                        // the row's class mask and its neighbours, by selection
                        auto pick8 = [&](const uint64_t *v) {
                            const uint64_t a0 = (yi & 1) ? v[1] : v[0], a1 = (yi & 1) ? v[3] : v[2];
                            const uint64_t a2 = (yi & 1) ? v[5] : v[4], a3 = (yi & 1) ? v[7] : v[6];
                            const uint64_t b0 = (yi & 2) ? a1 : a0, b1 = (yi & 2) ? a3 : a2;
                            return (yi & 4) ? b1 : b0;
                        };
                        const uint64_t mask = pick8(mk);
                        const uint64_t Su = pick8(Rw), Sy = pick8(Rw + 1), Sd = pick8(Rw + 2);
                        const bool hasN = y > 0, hasS = y < LD - 1;
                        const int yN = hasN ? y - 1 : y, yS = hasS ? y + 1 : y;
                        const uint64_t Suu = (y > 1) ? at(Lay::SP + (y > 1 ? y - 2 : 0)) : hN;
                        const uint64_t Sdd = (y < LD - 2) ? at(Lay::SP + (y < LD - 2 ? y + 2 : 0)) : hS;
                        // counts and spins disagree (never, unless the state is
                        // corrupt): recorded, and every index below stays in range
                        const bool bad = rr >= (uint32_t)__popcll(mask);
                        const int col = select_bit(mask, rr) & 63;
                        const uint64_t bit = 1ull << col;
                        uint64_t b0, b1, b2;
                        t64_planes(Sy, Su, Sd, (hW >> y) & 1ull, (hE >> y) & 1ull, b0, b1, b2);
                        // the site moves from (s, q) to (1 - s, q); each in-domain
                        // neighbour from (s', q') to (s', q' + delta)
                        const bool hasW = col > 0, hasE = col < LD - 1;
                        const int xw = hasW ? col - 1 : col, xe = hasE ? col + 1 : col;
                        auto qat = [&](int xx) {
                            return (int)((b0 >> xx) & 1ull) + 2 * (int)((b1 >> xx) & 1ull) + 4 * (int)((b2 >> xx) & 1ull);
                        };
                        const int qW = qat(xw), qE = qat(xe);
                        const int sW = (int)((Sy >> xw) & 1ull), sE = (int)((Sy >> xe) & 1ull);
                        const int qN = (int)((Suu >> col) & 1ull) + (int)((Sy >> col) & 1ull) +
                                       (int)(hasW ? (Su >> xw) & 1ull : (hW >> yN) & 1ull) +
                                       (int)(hasE ? (Su >> xe) & 1ull : (hE >> yN) & 1ull);
                        const int qS = (int)((Sdd >> col) & 1ull) + (int)((Sy >> col) & 1ull) +
                                       (int)(hasW ? (Sd >> xw) & 1ull : (hW >> yS) & 1ull) +
                                       (int)(hasE ? (Sd >> xe) & 1ull : (hE >> yS) & 1ull);
                        const int sN = (int)((Su >> col) & 1ull), sS = (int)((Sd >> col) & 1ull);
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
                        // may lie in (the spare block when there is none); blocks
                        // 0-3 form half 0, 4-7 half 1, the spare block half 2
                        const int by = y >> 3;
                        const bool crossN = (yN >> 3) != by, crossS = (yS >> 3) != by;
                        const int bo = crossN ? (yN >> 3) : crossS ? (yS >> 3) : NB;
                        const uint64_t bYlo = dYlo + (crossN ? 0ull : dNlo) + (crossS ? 0ull : dSlo);
                        const uint64_t bYhi = dYhi + (crossN ? 0ull : dNhi) + (crossS ? 0ull : dShi);
                        const uint64_t bOlo = (crossN ? dNlo : 0ull) + (crossS ? dSlo : 0ull);
                        const uint64_t bOhi = (crossN ? dNhi : 0ull) + (crossS ? dShi : 0ull);
                        const uint64_t kYlo = at(Lay::BLKLO + by), kYhi = at(Lay::BLKHI + by);
                        const uint64_t kOlo = at(Lay::BLKLO + bo), kOhi = at(Lay::BLKHI + bo);
                        at(Lay::SP + y) = Sy ^ bit;
                        at(Lay::BLKLO + by) = kYlo + bYlo;
                        at(Lay::BLKHI + by) = kYhi + bYhi;
                        at(Lay::BLKLO + bo) = kOlo + bOlo;
                        at(Lay::BLKHI + bo) = kOhi + bOhi;
                        const int hy = by >> 2, ho = bo >> 2;
                        h0lo += (hy == 0 ? bYlo : 0ull) + (ho == 0 ? bOlo : 0ull);
                        h0hi += (hy == 0 ? bYhi : 0ull) + (ho == 0 ? bOhi : 0ull);
                        h1lo += (hy == 1 ? bYlo : 0ull) + (ho == 1 ? bOlo : 0ull);
                        h1hi += (hy == 1 ? bYhi : 0ull) + (ho == 1 ? bOhi : 0ull);
                        colW ^= (col == 0) ? (1ull << y) : 0ull;
                        colE ^= (col == LD - 1) ? (1ull << y) : 0ull;
                        H = (H ^ ((np << 32) | ((uint64_t)j << 16) | (uint64_t)(y * LD + col))) * HASH_PRIME;
                        ++flips;
                        // flipping spin s with neighbour sum 2 qc - 4 changes the bond
                        // sum by -2 s (2 qc - 4) and the magnetisation by -2 s
                        const int sgn = up ? 1 : -1;
                        dbonds -= 2 * sgn * (2 * qc - 4);
                        dmag -= 2 * sgn;
                        rates();
                        corrupt |= bad;
                    }
                }
                if (corrupt) atomicCAS(P.err, 0, ERR_INTERNAL);
                if (has) {
                    // edges first (neighbours wait for them), then counters and record
                    uint64_t *ew = P.edges + (size_t)gl * EDGE_WORDS;
                    const uint64_t cnt = (uint64_t)after << 32;
                    const uint64_t S0 = at(Lay::SP + 0), S63 = at(Lay::SP + LD - 1);
                    const uint64_t eW = t64_col_to_edge(colW), eE = t64_col_to_edge(colE);
                    st_cg(ew + 2 * EDGE_N, cnt | (uint32_t)S0);
                    st_cg(ew + 2 * EDGE_N + 1, cnt | (uint32_t)(S0 >> 32));
                    st_cg(ew + 2 * EDGE_S, cnt | (uint32_t)S63);
                    st_cg(ew + 2 * EDGE_S + 1, cnt | (uint32_t)(S63 >> 32));
                    st_cg(ew + 2 * EDGE_W, cnt | (uint32_t)eW);
                    st_cg(ew + 2 * EDGE_W + 1, cnt | (uint32_t)(eW >> 32));
                    st_cg(ew + 2 * EDGE_E, cnt | (uint32_t)eE);
                    st_cg(ew + 2 * EDGE_E + 1, cnt | (uint32_t)(eE >> 32));
                    at(Lay::HFLO) = h0lo;
                    at(Lay::HFHI) = h0hi;
                    at(Lay::HFLO + 1) = h1lo;
                    at(Lay::HFHI + 1) = h1hi;
                    at(Lay::CW) = colW;
                    at(Lay::CE) = colE;
                    at(Lay::CH) = H;
                    at(Lay::CFL) += flips;
                    at(Lay::CST) += (uint64_t)total;
                    if (EXPO) {
                        // the domain clock takes the visit's product
                        uint64_t m = at(Lay::CCM);
                        int64_t e2 = (int64_t)at(Lay::CCE);
                        mant_mul(m, e2, vM, vE);
                        at(Lay::CCM) = m;
                        at(Lay::CCE) = (uint64_t)e2;
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
                        }
                        const uint64_t o0 = at(Lay::OB0), o1 = at(Lay::OB1);
                        const uint32_t steps = (uint32_t)(o0 >> 32) + (uint32_t)total;
                        const int bonds = (int)(uint32_t)o1 + dbonds, mag = (int)(uint32_t)(o1 >> 32) + dmag;
                        at(Lay::OB0) = (uint64_t)(uint32_t)o0 | ((uint64_t)steps << 32);
                        at(Lay::OB1) = (uint64_t)(uint32_t)bonds | ((uint64_t)(uint32_t)mag << 32);
                        if (EXPO) {
                            uint64_t m = at(Lay::OBM);
                            int64_t e2 = (int64_t)at(Lay::OBE);
                            mant_mul(m, e2, vM, vE);
                            at(Lay::OBM) = m;
                            at(Lay::OBE) = (uint64_t)e2;
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
        uint64_t *tile = reinterpret_cast<uint64_t *>(P.tiles + (size_t)g * (LD * LD / 8));
        for (int y = 0; y < LD; ++y) tile[y] = at(Lay::SP + y);
        uint64_t *ctr = P.dctr + (size_t)g * DCTR_WORDS;
        ctr[DCTR_HASH] = at(Lay::CH);
        ctr[DCTR_FLIPS] = at(Lay::CFL);
        ctr[DCTR_STEPS] = at(Lay::CST);
        ctr[DCTR_CLKM] = at(Lay::CCM);
        ctr[DCTR_CLKE] = at(Lay::CCE);
        if (P.n_obs > 0) flush();
    }
}

} // namespace kmcdev
