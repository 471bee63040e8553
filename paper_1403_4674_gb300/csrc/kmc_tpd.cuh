// kmc_tpd.cuh -- one thread per domain visit, for 8x8 domains.
//
// An 8x8 domain is one 64-bit word (row y at bits [8y, 8y+8), bit x = column
// x, the bit tile layout of the lattice kernels), so one thread can run a
// whole domain process (Sec. 2.2) in registers: the frozen halo is four
// 8-bit masks, the up-neighbour counts are three bit-sliced 64-bit planes,
// every class of App. A is a 64-bit mask, the cumulative class rates are ten
// 64-bit integers, and the n-fold way's member choice is a bit selection in
// one word.  A warp then runs 32 domain processes with no warp-collective
// operation at all, where the warp-per-domain kernel spends a whole warp
// (8 of its lanes holding rows) and a chain of shuffles, ballots and
// reductions on each one.
//
// The trajectory is the same as the warp kernel's, decision for decision:
// step j of global phase np draws Philox {j, d, np_lo, np_hi} with the
// replica seed, target = (w0 | w1<<32) >> 1 against R' = sum_c n_c A_c, class
// = first c with target < C_c, member jj = (target - C_{c-1}) / A_c in
// row-major (= bit) order.  Domain state, edge words, counters and the open
// observation record live in global memory (L2): each visit reads its tile
// and counters, waits for its neighbours' stamped edge words, runs, and
// writes them back.  Only the domain's owner thread writes its tile,
// counters and record (and only it reads them for use: a lane without a
// domain in a round reads some domain's and discards the values), and the
// stamped edge words carry data and visit count in one 64-bit store.
//
// Scope: palindromic and fixed colour schedules, exponential and expected
// clocks, per-replica k, records at schedule endpoints or every colour pass.
// Scores, fixed-time visits and random colour orders use the warp kernel.
#pragma once

#include "kmc_kernels.cuh"

namespace kmcdev {

constexpr uint64_t TPD_COL0 = 0x0101010101010101ull; // column 0 of every row
constexpr int TPD_OBS_WORDS = 4; // open record per domain: record | steps << 32, bonds | mag << 32, mantissa, exponent

// Bit y of an 8-bit column mask to bit 8y (column 0 of row y).
__device__ __forceinline__ uint64_t tpd_col_spread(uint32_t c8)
{
    uint64_t v = ((uint64_t)(c8 & 0xFFu) * 0x0101010101010101ull) & 0x8040201008040201ull;
    return ((v + 0x7F7F7F7F7F7F7F7Full) >> 7) & TPD_COL0;
}

// Column 0 of an 8x8 tile (bits 8y) to an 8-bit mask (bit y).
__device__ __forceinline__ uint32_t tpd_col_gather(uint64_t w)
{
    return (uint32_t)(((w & TPD_COL0) * 0x0102040810204080ull) >> 56);
}

// Bit-sliced count of up neighbours (0..4) of every site of tile T, with the
// frozen halo: the N neighbour's last row hN above row 0, the S neighbour's
// first row hS below row 7, the W and E neighbours' edge columns hW, hE
// (bit y = row y) left of column 0 and right of column 7.
struct TpdPlanes {
    uint64_t b0, b1, b2;
    __device__ __forceinline__ void build(uint64_t T, uint32_t hN, uint32_t hS, uint32_t hW, uint32_t hE)
    {
        const uint64_t U = (T << 8) | (uint64_t)(hN & 0xFFu);
        const uint64_t D = (T >> 8) | ((uint64_t)(hS & 0xFFu) << 56);
        const uint64_t Wn = ((T << 1) & ~TPD_COL0) | tpd_col_spread(hW);
        const uint64_t En = ((T >> 1) & ~(TPD_COL0 << 7)) | (tpd_col_spread(hE) << 7);
        const uint64_t s1 = U ^ D, c1 = U & D, s2 = Wn ^ En, c2 = Wn & En;
        const uint64_t t0 = s1 & s2;
        b0 = s1 ^ s2;
        b1 = c1 ^ c2 ^ t0;
        b2 = (c1 & c2) | (c1 & t0) | (c2 & t0);
    }
    // sites with exactly q up neighbours
    __device__ __forceinline__ uint64_t eq(int q) const
    {
        const uint64_t m2 = (q & 4) ? b2 : ~b2, m1 = (q & 2) ? b1 : ~b1, m0 = (q & 1) ? b0 : ~b0;
        return m2 & m1 & m0;
    }
};

// Cumulative class rates C_c = sum_{c' <= c} n_c' A_c' of tile T (classes
// 5 (s > 0) + q in order 0..9); C[9] = R'.
__device__ __forceinline__ void tpd_rates(uint64_t T, const TpdPlanes &pl, const uint64_t (&A)[10], uint64_t (&C)[10])
{
    uint64_t acc = 0;
#pragma unroll
    for (int c = 0; c < 10; ++c) {
        const uint64_t m = ((c >= 5) ? T : ~T) & pl.eq(c % 5);
        acc += (uint64_t)__popcll(m) * A[c];
        C[c] = acc;
    }
}

// The open record of domain g goes to its replica's record (records past
// the launch's last one are dropped), as the warp kernel's flush.
template <bool EXPO>
__device__ __forceinline__ void tpd_flush(const RunParams &P, const uint64_t *ob, uint32_t r)
{
    const uint32_t o = (uint32_t)ob[0];
    if (o == NO_RECORD || (int64_t)o >= P.n_obs) return;
    unsigned long long *acc = P.obs_acc + ((size_t)o * P.n_rep + r) * OBS_WORDS;
    const int bonds = (int)(uint32_t)ob[1], mag = (int)(uint32_t)(ob[1] >> 32);
    if (bonds != 0) atomicAdd(&acc[0], (unsigned long long)(long long)bonds);
    if (mag != 0) atomicAdd(&acc[1], (unsigned long long)(long long)mag);
    const uint32_t steps = (uint32_t)(ob[0] >> 32);
    const double dt = EXPO ? domain_time(true, ob[2], (int64_t)ob[3], 0, P.lambda) : __ddiv_rn((double)steps, P.lambda);
    atomicAdd(reinterpret_cast<double *>(&acc[2]), dt);
}

// Persistent kernel: thread t visits, in every colour phase, the domains
// t, t + T, t + 2T, ... of that colour's list (T = threads of the grid).
// P.cta_col_off holds the five offsets of the colour-sorted domain list
// P.slot_g; P.obs_dom the open records (TPD_OBS_WORDS per domain).  Bounds
// of two 4-warp CTAs per SM let the compiler keep about 150 registers (three
// CTAs still fit): 2 % faster on the 512-replica batch than its own choice
// of 102 with more values recomputed.
template <bool EXPO>
__global__ void __launch_bounds__(128, 2) tpd_kernel(const RunParams P)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const uint32_t *col_off = P.cta_col_off;
    const uint32_t *col_list = P.slot_g;
    const uint64_t *tile64 = reinterpret_cast<const uint64_t *>(P.tiles);
    uint64_t *tile64w = reinterpret_cast<uint64_t *>(P.tiles);
    const int nph = (P.schedule == SCHED_PALINDROME) ? 8 : 4;

    // no open record yet for any owned domain (a domain's owner is the
    // thread that visits it: list position - colour offset = tid mod T, so
    // only the owner ever reads or writes its record)
    if (P.n_obs > 0) {
        for (int c = 0; c < 4; ++c) {
            for (uint32_t i = col_off[c] + (uint32_t)tid; i < col_off[c + 1]; i += (uint32_t)nthreads) {
                uint64_t *ob = P.obs_dom + (size_t)col_list[i] * TPD_OBS_WORDS;
                ob[0] = (uint64_t)NO_RECORD;
                ob[1] = 0;
                ob[2] = 1ull << 63;
                ob[3] = 0;
            }
        }
    }

    unsigned spins = 0; // halo re-reads (profiling)
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
        // a neighbour across a row has colour ^ 2, across a column colour ^ 1
        const uint32_t needNS = gcount(colour ^ 2) + (uint32_t)P.debug_extra;
        const uint32_t needWE = gcount(colour ^ 1) + (uint32_t)P.debug_extra;
        const uint32_t after = gcount(colour) + 1;
        const int64_t pass = (int64_t)(gp - gp_begin);
        // Rounds of one domain per thread: every lane of a warp runs the
        // same trip counts (lanes without a domain in a round ride along
        // predicated), so the halo wait and the steps stay warp-synchronous
        // and the collectives below see the full warp.
        const uint32_t lo = col_off[colour], hi = col_off[colour + 1];
        const uint32_t rounds = (hi - lo + (uint32_t)nthreads - 1) / (uint32_t)nthreads;
        for (uint32_t m = 0; m < rounds && ok; ++m) {
            const uint32_t i = lo + (uint32_t)tid + m * (uint32_t)nthreads;
            const bool has = i < hi;
            const uint32_t g = has ? col_list[i] : col_list[lo];
            const uint32_t r = P.dom_rep[g];
            const uint32_t base = P.rep_dom_off[r];
            const uint32_t d = g - base;
            const int Dx = P.rep_Dx[r];
            const int bx = (int)(d % (uint32_t)Dx), by = (int)(d / (uint32_t)Dx);
            const uint32_t gN = base + (uint32_t)(((by + Dx - 1) % Dx) * Dx + bx);
            const uint32_t gS = base + (uint32_t)(((by + 1) % Dx) * Dx + bx);
            const uint32_t gW = base + (uint32_t)(by * Dx + (bx + Dx - 1) % Dx);
            const uint32_t gE = base + (uint32_t)(by * Dx + (bx + 1) % Dx);
            // everything that does not depend on the halo first
            const int k = P.rep_k[r];
            const int total = has ? nf * k : 0;
            const uint64_t seed = P.rep_seed[r];
            const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
            uint64_t A[10];
#pragma unroll
            for (int c = 0; c < 10; ++c) A[c] = __ldg(&P.rep_A[(size_t)r * 16 + c]);
            uint64_t T = tile64[g];
            uint64_t *ctr = P.dctr + (size_t)g * DCTR_WORDS;
            uint64_t H = ctr[DCTR_HASH];
            uint64_t clkM = ctr[DCTR_CLKM];
            int64_t clkE = (int64_t)ctr[DCTR_CLKE];
            // halo: the N neighbour's S row, the S neighbour's N row, the W
            // neighbour's E column, the E neighbour's W column (half 0 of
            // each), stamped with the neighbour's completed visits; the warp
            // re-reads until every lane's four are current (bounded)
            const uint64_t *pN = P.edges + (size_t)gN * EDGE_WORDS + 2 * EDGE_S;
            const uint64_t *pS = P.edges + (size_t)gS * EDGE_WORDS + 2 * EDGE_N;
            const uint64_t *pW = P.edges + (size_t)gW * EDGE_WORDS + 2 * EDGE_E;
            const uint64_t *pE = P.edges + (size_t)gE * EDGE_WORDS + 2 * EDGE_W;
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
                unsigned n = 0;
                while (true) {
                    if (!ready) {
                        wN = ld_volatile_global(pN);
                        wS = ld_volatile_global(pS);
                        wW = ld_volatile_global(pW);
                        wE = ld_volatile_global(pE);
                        ++spins;
                        ready = current();
                    }
                    if (__all_sync(FULL_WARP, ready)) break;
                    if ((++n & 63u) == 0) {
                        const bool late = global_ns() - t0 > P.bar_limit_ns;
                        const bool quit = late || *(volatile int *)P.err != 0;
                        if (__any_sync(FULL_WARP, quit)) {
                            if (late) atomicCAS(P.err, 0, ERR_TIMEOUT);
                            ok = false;
                            break;
                        }
                    }
                }
                if (!ok) break;
            }
            const uint32_t hN = (uint32_t)wN, hS = (uint32_t)wS, hW = (uint32_t)wW, hE = (uint32_t)wE;

            TpdPlanes pl;
            pl.build(T, hN, hS, hW, hE);
            uint64_t C[10];
            tpd_rates(T, pl, A, C);
            uint64_t flips = 0;
            int dbonds = 0, dmag = 0;
            uint64_t vM = 1ull << 63;
            int64_t vE = 0;
            const int smax = (int)__reduce_max_sync(FULL_WARP, (unsigned)total);
            // step s = f k + j of the visit: step j of global phase np0 + f
            int j = -1;
            uint64_t np = np0;
            for (int s = 0; s < smax; ++s) {
                const bool act = s < total;
                if (++j == k) {
                    j = 0;
                    ++np;
                }
                const uint4 w = philox4x32_10(make_uint4((uint32_t)j, d, (uint32_t)np, (uint32_t)(np >> 32) & 0xFFFFFFu),
                                              key);
                const uint64_t tgt = (((uint64_t)w.y << 32) | w.x) >> 1;
                if (EXPO && act) {
                    // clock variate v = V 2^-53 as a normalised mantissa m / 2^63
                    // times 2^(10 - z), into the visit's product
                    const uint64_t V = ((((uint64_t)w.w << 32) | w.z) >> 11) + 1ull;
                    const int z = __clzll((long long)V);
                    mant_mul(vM, vE, V << z, (int64_t)(10 - z));
                }
                if (!act || tgt >= C[9]) continue; // null step (App. A: the diagonal 1 - R/n_d)
                // class: the first c with tgt < C_c; C_{c-1} and A_c along with it
                int c = 0;
                uint64_t Cprev = 0, Ac = A[0];
#pragma unroll
                for (int cc = 0; cc < 9; ++cc) {
                    const bool past = tgt >= C[cc];
                    c = past ? cc + 1 : c;
                    Cprev = past ? C[cc] : Cprev;
                    Ac = past ? A[cc + 1] : Ac;
                }
                // exact jj = floor((tgt - C_{c-1}) / A_c) < n_c <= 64: an FP32
                // estimate rounded toward the lower side is jj or jj - 1, and
                // one integer comparison decides which
                const uint64_t x = tgt - Cprev;
                const float inv = __frcp_rd(u64_to_float_ru(Ac));
                uint32_t jj = (uint32_t)__fmul_rz(u64_to_float_rz(x), inv);
                jj = (x - (uint64_t)jj * Ac >= Ac) ? jj + 1u : jj;
                const int qc = (c >= 5) ? c - 5 : c;
                const uint64_t mask = ((c >= 5) ? T : ~T) & pl.eq(qc);
                const int site = select_bit(mask, jj);
                T ^= 1ull << site;
                H = (H ^ ((np << 32) | ((uint64_t)j << 16) | (uint64_t)site)) * HASH_PRIME;
                ++flips;
                // flipping spin s with neighbour sum 2 qc - 4 changes the bond
                // sum by -2 s (2 qc - 4) and the magnetisation by -2 s
                const int sgn = (c >= 5) ? 1 : -1;
                dbonds -= 2 * sgn * (2 * qc - 4);
                dmag -= 2 * sgn;
                if (s + 1 < total) {
                    pl.build(T, hN, hS, hW, hE);
                    tpd_rates(T, pl, A, C);
                }
            }
            if (!has) continue;
            if (EXPO) mant_mul(clkM, clkE, vM, vE); // the domain clock takes the visit's product
            // edges first (neighbours wait for them), then tile and counters
            uint64_t *ew = P.edges + (size_t)g * EDGE_WORDS;
            const uint64_t cnt = (uint64_t)after << 32;
            st_cg(ew + 2 * EDGE_N, cnt | (T & 0xFFull));
            st_cg(ew + 2 * EDGE_S, cnt | (T >> 56));
            st_cg(ew + 2 * EDGE_W, cnt | tpd_col_gather(T));
            st_cg(ew + 2 * EDGE_E, cnt | tpd_col_gather(T >> 7));
            if (flips) tile64w[g] = T;
            ctr[DCTR_HASH] = H;
            ctr[DCTR_FLIPS] += flips;
            ctr[DCTR_STEPS] += (uint64_t)total;
            ctr[DCTR_CLKM] = clkM;
            ctr[DCTR_CLKE] = (uint64_t)clkE;
            if (P.n_obs > 0) {
                // the visit's changes belong to the first record at or after its pass
                const int64_t o = (P.obs_pass ? pass : pass / nph) / P.obs_every;
                uint64_t *ob = P.obs_dom + (size_t)g * TPD_OBS_WORDS;
                uint64_t o0 = ob[0], o1 = ob[1], om = ob[2];
                int64_t oe = (int64_t)ob[3];
                if ((int64_t)(uint32_t)o0 != o) {
                    tpd_flush<EXPO>(P, ob, r);
                    o0 = (uint64_t)(uint32_t)o;
                    o1 = 0;
                    om = 1ull << 63;
                    oe = 0;
                }
                const uint32_t steps = (uint32_t)(o0 >> 32) + (uint32_t)total;
                const int bonds = (int)(uint32_t)o1 + dbonds, mag = (int)(uint32_t)(o1 >> 32) + dmag;
                if (EXPO) mant_mul(om, oe, vM, vE);
                ob[0] = (uint64_t)(uint32_t)o0 | ((uint64_t)steps << 32);
                ob[1] = (uint64_t)(uint32_t)bonds | ((uint64_t)(uint32_t)mag << 32);
                ob[2] = om;
                ob[3] = (uint64_t)oe;
            }
        }
        if (colour == 0) ++gc0;
        else if (colour == 1) ++gc1;
        else if (colour == 2) ++gc2;
        else ++gc3;
        gp += (uint64_t)nf;
    }
    if (P.polls && spins != 0) atomicAdd(P.polls, (unsigned long long)spins);
    if (!ok || *(volatile int *)P.err != 0) return;
    // every owned domain's open record
    if (P.n_obs > 0) {
        for (int c = 0; c < 4; ++c) {
            for (uint32_t i = col_off[c] + (uint32_t)tid; i < col_off[c + 1]; i += (uint32_t)nthreads) {
                const uint32_t g = col_list[i];
                tpd_flush<EXPO>(P, P.obs_dom + (size_t)g * TPD_OBS_WORDS, P.dom_rep[g]);
            }
        }
    }
}

} // namespace kmcdev
