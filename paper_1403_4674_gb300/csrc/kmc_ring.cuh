// kmc_ring.cuh -- sm_103a device code of the 1D ring (Sec. 3.1): many
// independent trajectories of an N_S-spin toroidal Ising ring (N_S <= 64),
// cut into N_D contiguous domains of L_d spins (Sec. 3.1, Eq. 1D partitions),
// each domain process k uniformised steps with its two halo spins frozen.
//
// Data parallelism is over trajectories (the paper's N_TRAJ independent
// runs per setting, Eq. time dependent averages): one thread owns one
// trajectory for the whole launch, its configuration a 64-bit register word
// (bit n set iff spin n is up).  Within a thread the domain processes of a
// schedule run in schedule order, so the halo of a visit is the live word:
// no other domain of the trajectory moves while it runs.  Observation records
// per trajectory are coalesced stores; the ensemble sums over trajectories
// (integers, so their order does not matter) are reduced per warp with
// ballots and warp reductions, per CTA in shared memory, and added to global
// memory with one atomic per CTA and quantity.
#pragma once

#include <cstdint>

#include "kmc_kernels.cuh"

namespace kmcring {

using kmcdev::FULL_WARP;
using kmcdev::HASH_PRIME;

constexpr int RING_CLASSES = 6;      // c = 3*up + (number of up neighbours)
constexpr int RING_PHASE_SLOTS = 64; // Philox phase index np = n*64 + p
constexpr int RING_ENS_FIXED = 4;    // sum bonds, sum mag, sum bonds*mag, sum mag^2; then per-site up counts
constexpr int RING_BLOCK = 128;
constexpr uint32_t RING_TAG_PERM = 2u;

struct RingParams {
    int n_traj, NS, Ld, k;
    int schedule;         // KMC_SCHED_*
    int obs_every;        // passes between records (0: none)
    int64_t sched_begin, n_sched;
    double J, nu;
    const uint64_t *seed; // [n_traj]
    const uint64_t *A;    // [n_traj][6] fixed-point acceptance, P = 63 - log2(L_d)
    const double *h;      // [n_traj]
    uint64_t *state, *hash, *clkM;
    int64_t *clkE, *flips, *steps;
    double *t;            // [n_traj] clock after the launch
    double *obs;          // [n_rec][n_traj][4] or null
    uint64_t *obs_state;  // [n_rec][n_traj] or null
    unsigned long long *ens; // [n_rec][4 + NS] or null (added to)
};

// Neighbour words of a ring of NS bits: bit n of lw is spin n-1, of rw spin n+1.
__device__ __forceinline__ uint64_t ring_left(uint64_t S, int NS, uint64_t NM)
{
    return ((S << 1) | (S >> (NS - 1))) & NM;
}
__device__ __forceinline__ uint64_t ring_right(uint64_t S, int NS, uint64_t NM)
{
    return (S >> 1) | ((S & 1ull) << (NS - 1));
}

// Sites of class c = 3 up + q of one domain (DM: its sites).
__device__ __forceinline__ uint64_t ring_class_mask(uint64_t S, uint64_t DM, int NS, uint64_t NM, int c)
{
    const uint64_t lw = ring_left(S, NS, NM), rw = ring_right(S, NS, NM);
    const int q = (c >= 3) ? c - 3 : c;
    const uint64_t qm = (q == 0) ? ~(lw | rw) : ((q == 1) ? (lw ^ rw) : (lw & rw));
    return ((c >= 3) ? S : ~S) & qm & DM;
}

// Inclusive cumulative rates C_c = sum_{c' <= c} n_c' A_c' in class order 0..5.
__device__ __forceinline__ void ring_cumulative(uint64_t (&C)[RING_CLASSES], uint64_t S, uint64_t DM, int NS,
                                                uint64_t NM, const uint64_t (&A)[RING_CLASSES])
{
    const uint64_t lw = ring_left(S, NS, NM), rw = ring_right(S, NS, NM);
    const uint64_t q0 = ~(lw | rw), q1 = lw ^ rw, q2 = lw & rw;
    const uint64_t up = S & DM, dn = ~S & DM;
    const uint64_t M[RING_CLASSES] = {dn & q0, dn & q1, dn & q2, up & q0, up & q1, up & q2};
    uint64_t acc = 0;
#pragma unroll
    for (int c = 0; c < RING_CLASSES; ++c) {
        acc += (uint64_t)__popcll(M[c]) * A[c];
        C[c] = acc;
    }
}

// One domain process: domain d, k steps of global phase np.  Step j draws
// Philox {j, d, np_lo, np_hi} with the trajectory seed: target = (w0 |
// w1<<32) >> 1 on [0, L_d 2^P); target >= R' is a null step; otherwise the
// class is the first c with target < C_c and the member jj = (target -
// C_{c-1}) / A_c, counted in ascending site order, flips (App. A, the
// n-fold way's cumulative selection of Sec. 2.1).  jj < n_c <= 64: an FP32
// estimate with every rounding toward the lower side (x down, A_c up, the
// reciprocal down, the product toward zero) is jj or jj - 1, and one exact
// integer comparison decides.
template <bool EXPO>
__device__ __forceinline__ void ring_visit(uint64_t &S, uint64_t &H, int64_t &flips, uint64_t &clkM, int64_t &clkE,
                                           int d, int Ld, int k, int NS, uint64_t NM, uint64_t DM0, uint64_t np,
                                           uint2 key, const uint64_t (&A)[RING_CLASSES],
                                           const float (&invA)[RING_CLASSES])
{
    const int first = d * Ld;
    const uint64_t DM = DM0 << first;
    uint64_t C[RING_CLASSES];
    ring_cumulative(C, S, DM, NS, NM, A);
    for (int j = 0; j < k; ++j) {
        const uint4 w = kmcdev::philox4x32_10(
            make_uint4((uint32_t)j, (uint32_t)d, (uint32_t)np, (uint32_t)(np >> 32) & 0xFFFFFFu), key);
        const uint64_t tgt = (((uint64_t)w.y << 32) | w.x) >> 1;
        if (EXPO) {
            const uint64_t V = ((((uint64_t)w.w << 32) | w.z) >> 11) + 1ull;
            const int z = __clzll((long long)V);
            kmcdev::mant_mul(clkM, clkE, V << z, (int64_t)(10 - z));
        }
        if (tgt >= C[RING_CLASSES - 1]) continue; // null step
        uint64_t lo = 0, Ac = A[0];
        float inv = invA[0];
        int c = 0;
#pragma unroll
        for (int cc = 1; cc < RING_CLASSES; ++cc) {
            if (tgt >= C[cc - 1]) {
                lo = C[cc - 1];
                Ac = A[cc];
                inv = invA[cc];
                c = cc;
            }
        }
        const uint64_t x = tgt - lo;
        uint32_t jj = (uint32_t)__fmul_rz(kmcdev::u64_to_float_rz(x), inv);
        jj = (x - (uint64_t)jj * Ac >= Ac) ? jj + 1u : jj;
        const int site = kmcdev::select_bit(ring_class_mask(S, DM, NS, NM, c), jj);
        S ^= 1ull << site;
        ++flips;
        H = (H ^ ((np << 32) | ((uint64_t)j << 16) | (uint64_t)(site - first))) * HASH_PRIME;
        ring_cumulative(C, S, DM, NS, NM, A);
    }
}

// Uniform random order of the n_dom domains of schedule n (the paper's
// random schedule per sweep): Fisher-Yates, draw i (n_dom-1 down to 1) from
// Philox {i, 0, n_lo, n_hi | TAG_PERM << 24}: position i swaps with
// floor(x (i+1) / 2^64), x = w0 | w1 << 32.
__device__ __forceinline__ void ring_perm(uint8_t *order, int n_dom, uint64_t n, uint2 key)
{
    for (int i = 0; i < n_dom; ++i) order[i] = (uint8_t)i;
    for (int i = n_dom - 1; i >= 1; --i) {
        const uint4 w = kmcdev::philox4x32_10(
            make_uint4((uint32_t)i, 0u, (uint32_t)n, ((uint32_t)(n >> 32) & 0xFFFFFFu) | (RING_TAG_PERM << 24)), key);
        const uint64_t x = ((uint64_t)w.y << 32) | w.x;
        const int jx = (int)__umul64hi(x, (uint64_t)(i + 1));
        const uint8_t t = order[i];
        order[i] = order[jx];
        order[jx] = t;
    }
}

// Clock of a trajectory: the mean over domains of t_d (Sec. 2.1), i.e.
// -ln(product of all its variates) / (N_S nu) (exponential) or
// steps / (N_S nu) (expected).
__device__ __forceinline__ double ring_clock(bool expo, uint64_t M, int64_t E, int64_t steps, int NS, double nu)
{
    return kmcdev::domain_time(expo, M, E, steps, __dmul_rn((double)NS, nu));
}

template <bool EXPO>
__global__ void __launch_bounds__(RING_BLOCK, 6) ring_kernel(const RingParams P)
{
    __shared__ int ens_blk[RING_ENS_FIXED + 64];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool active = tid < P.n_traj;
    const int r = active ? tid : 0;
    const int NS = P.NS, Ld = P.Ld, ND = NS / Ld, k = P.k;
    const int n_ens = RING_ENS_FIXED + NS;
    const uint64_t NM = (NS == 64) ? ~0ull : ((1ull << NS) - 1ull);
    const uint64_t DM0 = (Ld == 64) ? ~0ull : ((1ull << Ld) - 1ull);

    uint64_t A[RING_CLASSES];
    float invA[RING_CLASSES]; // 1/A_c from below: A_c rounded up, reciprocal rounded down
#pragma unroll
    for (int c = 0; c < RING_CLASSES; ++c) {
        A[c] = P.A[(size_t)r * RING_CLASSES + c];
        invA[c] = A[c] ? __frcp_rd(kmcdev::u64_to_float_ru(A[c])) : 0.0f;
    }
    const uint64_t seed = P.seed[r];
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const double hr = P.h[r];
    uint64_t S = P.state[r], H = P.hash[r], clkM = P.clkM[r];
    int64_t clkE = P.clkE[r], flips = P.flips[r], steps = P.steps[r];

    if (P.ens != nullptr)
        for (int i = threadIdx.x; i < n_ens; i += blockDim.x) ens_blk[i] = 0;
    __syncthreads();

    const bool perm = P.schedule == kmcdev::SCHED_RANDOM_PERM;
    const int ncol = (ND == 1) ? 1 : 2;
    const int nph = perm ? ND : (P.schedule == kmcdev::SCHED_PALINDROME ? 2 * ncol : ncol);
    uint8_t order[64];
    int64_t passes = 0;
    for (int64_t nl = 0; nl < P.n_sched; ++nl) {
        const uint64_t n = (uint64_t)(P.sched_begin + nl);
        if (perm && active) ring_perm(order, ND, n, key);
        for (int p = 0; p < nph; ++p) {
            const uint64_t np = n * RING_PHASE_SLOTS + (uint64_t)p;
            if (active) {
                if (perm) {
                    ring_visit<EXPO>(S, H, flips, clkM, clkE, order[p], Ld, k, NS, NM, DM0, np, key, A, invA);
                    steps += k;
                } else {
                    // colour of phase p: 0 1 [1 0] (one colour when N_D = 1)
                    const int col = (p < ncol) ? p : (2 * ncol - 1 - p);
                    for (int d = col; d < ND; d += ncol) {
                        ring_visit<EXPO>(S, H, flips, clkM, clkE, d, Ld, k, NS, NM, DM0, np, key, A, invA);
                        steps += k;
                    }
                }
            }
            ++passes;
            if (P.obs_every > 0 && passes % P.obs_every == 0) {
                const int64_t rec = passes / P.obs_every - 1;
                // bonds = sum_n s_n s_{n+1}: NS - 2 * (number of unlike neighbour pairs)
                const int unlike = __popcll((S ^ ring_left(S, NS, NM)) & NM);
                const int bonds = NS - 2 * unlike;
                const int mag = 2 * __popcll(S & NM) - NS;
                if (active) {
                    const size_t o = (size_t)rec * P.n_traj + r;
                    if (P.obs) {
                        const double e = __ddiv_rn(__dsub_rn(__dmul_rn(-P.J, (double)bonds), __dmul_rn(hr, (double)mag)),
                                                   (double)NS);
                        const double m = __ddiv_rn((double)mag, (double)NS);
                        double4_32a v;
                        v.x = e;
                        v.y = m;
                        v.z = __dmul_rn(e, m);
                        v.w = ring_clock(EXPO, clkM, clkE, steps, NS, P.nu);
                        reinterpret_cast<double4_32a *>(P.obs)[o] = v;
                    }
                    if (P.obs_state) P.obs_state[o] = S;
                }
                if (P.ens != nullptr) {
                    // ensemble sums: warp reductions, then one shared atomic per warp
                    const int b = active ? bonds : 0, m = active ? mag : 0;
                    const int s0 = __reduce_add_sync(FULL_WARP, b);
                    const int s1 = __reduce_add_sync(FULL_WARP, m);
                    const int s2 = __reduce_add_sync(FULL_WARP, b * m);
                    const int s3 = __reduce_add_sync(FULL_WARP, m * m);
                    int cnt = 0;
                    for (int i = 0; i < NS; ++i) {
                        const int ci = __popc(__ballot_sync(FULL_WARP, active && ((S >> i) & 1ull)));
                        if (lane == (i & 31)) cnt = ci; // lane i%32 keeps site i's count (two sites when NS > 32)
                        if (i == 31 || i == NS - 1) {
                            if (lane <= (i & 31)) atomicAdd(&ens_blk[RING_ENS_FIXED + (i & ~31) + lane], cnt);
                        }
                    }
                    if (lane == 0) {
                        atomicAdd(&ens_blk[0], s0);
                        atomicAdd(&ens_blk[1], s1);
                        atomicAdd(&ens_blk[2], s2);
                        atomicAdd(&ens_blk[3], s3);
                    }
                    __syncthreads();
                    for (int i = threadIdx.x; i < n_ens; i += blockDim.x) {
                        const int v = ens_blk[i];
                        if (v != 0)
                            atomicAdd(&P.ens[(size_t)rec * n_ens + i], (unsigned long long)(long long)v);
                        ens_blk[i] = 0;
                    }
                    __syncthreads();
                }
            }
        }
    }
    if (active) {
        P.state[r] = S;
        P.hash[r] = H;
        P.clkM[r] = clkM;
        P.clkE[r] = clkE;
        P.flips[r] = flips;
        P.steps[r] = steps;
        P.t[r] = ring_clock(EXPO, clkM, clkE, steps, NS, P.nu);
    }
}

} // namespace kmcring
