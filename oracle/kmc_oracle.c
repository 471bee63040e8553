/*
 * kmc_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * sequential-update parallel kinetic Monte Carlo of Nilmeier & Marian,
 * "A rigorous sequential update strategy for parallel kinetic Monte Carlo
 * simulation" (arXiv:1403.4674).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline / reference arm do.  It shares no code, header,
 * table or constant generator with the CUDA library: every definition below
 * (Philox4x32-10, the rate table, the class index, the step protocol, the
 * event hash) is written out here a second time, on purpose, from its
 * published or stated definition.
 *
 * What it computes, in the paper's order:
 *   - 2D periodic Ising energy, App. A (Eq. for beta*H, 2D line; both
 *     factors read as configuration j), plus a field term -h*sum(sigma);
 *   - the lattice cut into equal square domains (Sec. 2.2), coloured 2x2 so
 *     that same-coloured domains share no halo (Sec. 2.2: domains that do
 *     not interact may be visited in any order, or at once);
 *   - each domain process runs k steps with its halo frozen (Sec. 2.2,
 *     Eqs. 4-5).  One step is the uniformised single-site kernel of App. A
 *     (Eq. Glauber_TM): site i of the domain flips with probability
 *     a_c(i)/n_d, otherwise the step is null (the diagonal T_ii).  The real
 *     event is drawn the n-fold-way way (Sec. 2.1, R = sum of all rates):
 *     classes c, counts n_c, cumulative rates, then a uniform member;
 *   - colours visited in a schedule closed under reversal (Sec. 2.2,
 *     Eqs. 9-10): the palindrome 0 1 2 3 3 2 1 0 by default;
 *   - the clock: Erlang / Poisson variate of Sec. 2.1 (Eq. 2) as a sum of
 *     -log(u), or its expectation N*tau_S;
 *   - observables at schedule endpoints only (Sec. 2.3);
 *   - optionally, a domain process that runs for a fixed time dtau instead
 *     of a fixed number of steps: the continuous-time chain of the domain
 *     over dtau, exp(dtau Q_d) = sum_K Poisson(K; n_d nu dtau) P_d^K, i.e. a
 *     Poisson number of uniformised steps, reversible because P_d is;
 *   - the 1D ring of Sec. 3.1 (N_S <= 64 spins, toroidal, contiguous
 *     domains of Eq. 1D partitions) with the same step protocol, colour
 *     schedules (colours d & 1) and the paper's uniformly random order of
 *     all domains per sweep (Sec. 2.2, Fig. 1).
 *
 * Everything that steers the trajectory is integer: the rate table is held
 * in fixed point, A_c = round(a_c * 2^P) with P = 63 - log2(n_d), so that a
 * step's decision is an exact integer comparison.  Floating point only
 * appears in the clock and in the final observables.
 *
 * Pins (tests/test_oracle_*.py): Philox against PyTorch's engine; the
 * rate table against closed forms; the sampler against exact enumeration of
 * the same chain, the beta = 0 closed form and the Erlang clock law; the
 * long-run energy against Kaufman's exact finite lattice; the score table
 * against finite differences of the rate table, and the likelihood-ratio
 * estimator against the exact derivative of the enumerated distribution;
 * the ring against its transfer-matrix equilibrium, the textbook
 * random-site kernel, its enumerated final-state distribution and
 * time-dependent spin averages, and the beta = 0 closed form.
 * Parity unpinned: the per-domain event hash (a fingerprint this library
 * defines for CPU/GPU event-sequence parity, not a quantity of the paper)
 * and the Philox counter layout (likewise a definition of this library).
 *
 * Build: gcc -O2 -std=gnu11 -ffp-contract=off -fPIC -shared -lm.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Ten rounds of the 4x32 Philox S-box with the
 * published multipliers and Weyl key increments.
 * ---------------------------------------------------------------------- */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += ORC_PHILOX_W0;
        k1 += ORC_PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter-word tags (top byte of counter word 3). */
#define ORC_TAG_STEP 0u
#define ORC_TAG_INIT 1u
#define ORC_TAG_PERM 2u
#define ORC_TAG_HORIZON 3u

/* Rate laws, schedules, time modes, initial states. */
#define ORC_RATE_METROPOLIS 0
#define ORC_RATE_BARKER 1
#define ORC_SCHED_PALINDROME 0
#define ORC_SCHED_FIXED 1
#define ORC_SCHED_RANDOM_PERM 2
#define ORC_TIME_EXPONENTIAL 0
#define ORC_TIME_EXPECTED 1
#define ORC_TIME_HORIZON 2
#define ORC_INIT_RANDOM 0
#define ORC_INIT_ALL_UP 1

/* FNV-1a 64-bit offset basis and prime (Fowler, Noll, Vo), applied to
 * whole 64-bit event words rather than bytes. */
#define ORC_HASH_BASIS 0xcbf29ce484222325ull
#define ORC_HASH_PRIME 0x00000100000001b3ull

static int orc_log2(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return ((1 << r) == v) ? r : -1;
}

/* ------------------------------------------------------------------------
 * Rate table (App. A, Eq. Glauber_TM; Metropolis as the alternative law).
 * Class c = 5*sp + q: sp = 1 for an up spin, q = number of up neighbours
 * (0..4).  sigma = 2*sp - 1, neighbour sum = 2q - 4,
 *   dE_c = 2*sigma*(J*(2q-4) + h),
 *   Metropolis: a_c = 1 if dE_c <= 0 else exp(-beta*dE_c)
 *   Barker:     a_c = 1 / (1 + exp(beta*dE_c))     (App. A, "Barker")
 * a_c is the acceptance of the uniformised step; the physical rate is
 * nu*a_c.  A_c = round-to-nearest-even(a_c * 2^P), P = 63 - log2(n_d).
 * Returns 0, -1 for an invalid argument, or -2 when some a_c rounds to
 * A_c = 0: every a_c is positive, so the quantised chain would then leave
 * class c's reverse but never enter it, which breaks detailed balance
 * (Sec. 2.2, Eq. 4).
 * ---------------------------------------------------------------------- */
int orc_rate_table(double J, double beta, double h, int law, int log2_nd,
                   double a_out[10], uint64_t A_out[10])
{
    if (log2_nd < 0 || log2_nd > 16) return -1;
    if (law != ORC_RATE_METROPOLIS && law != ORC_RATE_BARKER) return -1;
    if (!(beta >= 0.0) || !isfinite(beta) || !isfinite(J) || !isfinite(h))
        return -1;
    int P = 63 - log2_nd;
    for (int sp = 0; sp < 2; ++sp) {
        for (int q = 0; q <= 4; ++q) {
            int c = 5 * sp + q;
            double sigma = sp ? 1.0 : -1.0;
            double nsum = (double)(2 * q - 4);
            double dE = 2.0 * sigma * (J * nsum + h);
            double a;
            if (law == ORC_RATE_METROPOLIS)
                a = (dE <= 0.0) ? 1.0 : exp(-beta * dE);
            else
                a = 1.0 / (1.0 + exp(beta * dE));
            a_out[c] = a;
            A_out[c] = (uint64_t)nearbyint(ldexp(a, P));
        }
    }
    for (int c = 0; c < 10; ++c)
        if (A_out[c] == 0) return -2;
    return 0;
}

/* ------------------------------------------------------------------------
 * Derivatives of log a_c for the likelihood-ratio score (the acceptance
 * table above as a function of beta and h):
 *   Metropolis, dE_c > 0: dlog a/dbeta = -dE_c, dlog a/dh = -2 beta sigma;
 *               dE_c <= 0: both 0 (a = 1);
 *   Barker: dlog a/dbeta = -dE_c (1 - a_c), dlog a/dh = -2 beta sigma (1 - a_c).
 * grad[0..9] = a_c, grad[10..19] = dlog a_c/dbeta, grad[20..29] = dlog a_c/dh.
 * ---------------------------------------------------------------------- */
int orc_score_table(double J, double beta, double h, int law, double grad[30])
{
    if (law != ORC_RATE_METROPOLIS && law != ORC_RATE_BARKER) return -1;
    for (int c = 0; c < 10; ++c) {
        int sp = c / 5, q = c % 5;
        double sigma = sp ? 1.0 : -1.0;
        double dE = 2.0 * sigma * (J * (double)(2 * q - 4) + h);
        double a, db, dh;
        if (law == ORC_RATE_METROPOLIS) {
            if (dE <= 0.0) { a = 1.0; db = 0.0; dh = 0.0; }
            else { a = exp(-beta * dE); db = -dE; dh = -beta * 2.0 * sigma; }
        } else {
            a = 1.0 / (1.0 + exp(beta * dE));
            db = -dE * (1.0 - a);
            dh = -beta * 2.0 * sigma * (1.0 - a);
        }
        grad[c] = a;
        grad[10 + c] = db;
        grad[20 + c] = dh;
    }
    return 0;
}

/* dE of class c, for tests and for the score. */
double orc_class_dE(int c, double J, double h)
{
    int sp = c / 5, q = c % 5;
    double sigma = sp ? 1.0 : -1.0;
    return 2.0 * sigma * (J * (double)(2 * q - 4) + h);
}

/* ------------------------------------------------------------------------
 * Initial state: iid +-1 from Philox, or all up.  Site i = y*L + x; block
 * b = i / 128 uses counter {b_lo, b_hi, 0, TAG_INIT<<24}; the site is up
 * iff bit (i mod 128) of the 128-bit output is set (word (i%128)/32,
 * bit i%32).
 * ---------------------------------------------------------------------- */
void orc_init_spins(int8_t *s, int L, int init, uint64_t seed)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; ++i) {
        if (init == ORC_INIT_ALL_UP) { s[i] = 1; continue; }
        uint64_t b = (uint64_t)i / 128u;
        uint32_t ctr[4] = {(uint32_t)b, (uint32_t)(b >> 32), 0u,
                           ORC_TAG_INIT << 24};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        int bit = (int)((w[(i % 128) / 32] >> (i % 32)) & 1u);
        s[i] = bit ? 1 : -1;
    }
}

/* ------------------------------------------------------------------------
 * Colour of domain (bx, by): (bx & 1) | ((by & 1) << 1).
 * Colour sequence of schedule n (Sec. 2.2, Eqs. 9-10):
 *   PALINDROME: 0 1 2 3 3 2 1 0 (its own reverse, so w(L) = w(reverse L));
 *   FIXED:      0 1 2 3 (not closed under reversal: keeps pi stationary but
 *               not detailed balance; kept as a negative test);
 *   RANDOM_PERM: a uniform random order of the four colours per schedule,
 *               Philox counter {0, 0, n_lo, n_hi | TAG_PERM<<24}; index =
 *               floor(x * 24 / 2^64) with x = w0 | w1<<32, decoded as a
 *               Lehmer code (most significant digit first).
 * Returns the number of phases of one schedule.
 * ---------------------------------------------------------------------- */
int orc_schedule_colours(int schedule, uint64_t n, uint64_t seed, int out[8])
{
    if (schedule == ORC_SCHED_PALINDROME) {
        static const int pal[8] = {0, 1, 2, 3, 3, 2, 1, 0};
        memcpy(out, pal, sizeof pal);
        return 8;
    }
    if (schedule == ORC_SCHED_FIXED) {
        for (int i = 0; i < 4; ++i) out[i] = i;
        return 4;
    }
    if (schedule == ORC_SCHED_RANDOM_PERM) {
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t ctr[4] = {0u, 0u, (uint32_t)n,
                           (uint32_t)((n >> 32) & 0xFFFFFFu) | (ORC_TAG_PERM << 24)};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        uint64_t x = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
        /* floor(x * 24 / 2^64), exact in 128-bit arithmetic */
        unsigned __int128 prod = (unsigned __int128)x * 24u;
        int idx = (int)(prod >> 64);
        int pool[4] = {0, 1, 2, 3};
        int left = 4;
        static const int fact[4] = {6, 2, 1, 1};
        for (int pos = 0; pos < 4; ++pos) {
            int sel = idx / fact[pos];
            idx %= fact[pos];
            out[pos] = pool[sel];
            for (int t = sel; t < left - 1; ++t) pool[t] = pool[t + 1];
            --left;
        }
        return 4;
    }
    return -1;
}

/* ------------------------------------------------------------------------
 * Compensated summation (Neumaier 1974, the improved Kahan-Babuska sum):
 * *sum + *comp carries the running total; each term's rounding error is
 * recovered exactly and added to *comp.  The likelihood-ratio score of a
 * domain is a sum of some 1e5 per-step terms of both signs whose total is
 * much smaller than its partial sums; a plain running FP64 sum would carry
 * an error of order 2^-53 times the partial sums times the square root of
 * the number of terms, this one an error of a few ulp of the total.
 * ---------------------------------------------------------------------- */
static void orc_sum_add(double *sum, double *comp, double x)
{
    double t = *sum + x;
    if (fabs(*sum) >= fabs(x))
        *comp += (*sum - t) + x;
    else
        *comp += (x - t) + *sum;
    *sum = t;
}

/* Compensated sum of x[0..n-1] (for tests of the summation above). */
double orc_sum_compensated(const double *x, int64_t n)
{
    double sum = 0.0, comp = 0.0;
    for (int64_t i = 0; i < n; ++i) orc_sum_add(&sum, &comp, x[i]);
    return sum + comp;
}

/* ------------------------------------------------------------------------
 * One domain process (Sec. 2.2): domain d = by*Dx + bx of a replica, k
 * uniformised steps with the halo frozen.
 *
 * Step j of global phase np uses Philox counter
 *   {j, d, np_lo, (np_hi & 0xFFFFFF) | TAG_STEP<<24}, key = replica seed:
 *   target = (w0 | w1<<32) >> 1, uniform on [0, n_d * 2^P) = [0, 2^63);
 *   V      = ((w2 | w3<<32) >> 11) + 1, so v = V * 2^-53 is in (0, 1].
 * With counts n_c and R' = sum_c n_c A_c (classes taken in order 0..9):
 *   target >= R'  -> null step (the diagonal of Eq. Glauber_TM);
 *   otherwise class c = the smallest c with target < C_c (C_c inclusive
 *   cumulative sums), member index jj = (target - C_{c-1}) / A_c, and the
 *   jj-th site of class c in row-major order flips.
 * So P(site i flips) = A_c(i) / (n_d 2^P) exactly, the same single-site
 * kernel as App. A with a_c quantised to P fractional bits.
 *
 * The event hash of the domain folds every real event as
 *   H <- (H xor e) * FNV_PRIME,  e = np<<32 | j<<16 | i.
 * Exponential clock: esum_d += -log(v) for every step (Sec. 2.1, the
 * Poisson variate as a sum of negative logarithms).
 * Score (grad != NULL): score[0..1] are the domain's running sums of
 * d log P / d(beta, h) and score[2..3] their compensations (orc_sum_add);
 * the domain's score is score[0..1] + score[2..3].
 * ---------------------------------------------------------------------- */
static void orc_visit(int8_t *s, int L, int Ld, int bx, int by, int k,
                      const uint64_t A[10], uint32_t key0, uint32_t key1,
                      uint64_t np, uint32_t d, int time_mode,
                      double *esum, uint64_t *hash, int64_t *flips,
                      int64_t *steps, const double *grad, double *score)
{
    const int x0 = bx * Ld, y0 = by * Ld, nd = Ld * Ld;
    /* frozen halo, collected before the domain process runs */
    int8_t *top = (int8_t *)malloc((size_t)Ld);
    int8_t *bot = (int8_t *)malloc((size_t)Ld);
    int8_t *lft = (int8_t *)malloc((size_t)Ld);
    int8_t *rgt = (int8_t *)malloc((size_t)Ld);
    int *cls = (int *)malloc(sizeof(int) * (size_t)nd);
    for (int x = 0; x < Ld; ++x) {
        top[x] = s[(int64_t)((y0 - 1 + L) % L) * L + x0 + x];
        bot[x] = s[(int64_t)((y0 + Ld) % L) * L + x0 + x];
    }
    for (int y = 0; y < Ld; ++y) {
        lft[y] = s[(int64_t)(y0 + y) * L + (x0 - 1 + L) % L];
        rgt[y] = s[(int64_t)(y0 + y) * L + (x0 + Ld) % L];
    }
#define SITE(xx, yy) s[(int64_t)(y0 + (yy)) * L + x0 + (xx)]
    for (int j = 0; j < k; ++j) {
        /* classes of every domain site, recomputed from scratch */
        uint64_t n[10] = {0};
        for (int y = 0; y < Ld; ++y) {
            for (int x = 0; x < Ld; ++x) {
                int sp = SITE(x, y) > 0;
                int up = (y > 0) ? SITE(x, y - 1) : top[x];
                int dn = (y < Ld - 1) ? SITE(x, y + 1) : bot[x];
                int lf = (x > 0) ? SITE(x - 1, y) : lft[y];
                int rt = (x < Ld - 1) ? SITE(x + 1, y) : rgt[y];
                int q = (up > 0) + (dn > 0) + (lf > 0) + (rt > 0);
                int c = 5 * sp + q;
                cls[y * Ld + x] = c;
                n[c] += 1;
            }
        }
        uint64_t R = 0;
        for (int c = 0; c < 10; ++c) R += n[c] * A[c];
        /* likelihood-ratio score of this step: the step's probability is
         * a_c/n_d for a real flip of a class-c site and 1 - R/n_d for a null
         * step, R = sum_c n_c a_c (real-valued acceptances) */
        double Rr = 0.0, Db = 0.0, Dh = 0.0;
        if (grad) {
            for (int c = 0; c < 10; ++c) {
                double w = (double)n[c] * grad[c];
                Rr += w;
                Db += w * grad[10 + c];
                Dh += w * grad[20 + c];
            }
        }

        uint32_t ctr[4] = {(uint32_t)j, d, (uint32_t)np,
                           (uint32_t)((np >> 32) & 0xFFFFFFu) | (ORC_TAG_STEP << 24)};
        uint32_t key[2] = {key0, key1};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        uint64_t target = ((uint64_t)w[0] | ((uint64_t)w[1] << 32)) >> 1;
        uint64_t V = (((uint64_t)w[2] | ((uint64_t)w[3] << 32)) >> 11) + 1u;
        if (time_mode == ORC_TIME_EXPONENTIAL)
            *esum += -log(ldexp((double)V, -53));
        *steps += 1;
        if (target >= R) { /* null step */
            if (grad) {
                orc_sum_add(&score[0], &score[2], -(Db / ((double)nd - Rr)));
                orc_sum_add(&score[1], &score[3], -(Dh / ((double)nd - Rr)));
            }
            continue;
        }

        uint64_t C = 0;
        int c = 0;
        for (c = 0; c < 10; ++c) {
            uint64_t w_c = n[c] * A[c];
            if (target < C + w_c) break;
            C += w_c;
        }
        if (grad) {
            orc_sum_add(&score[0], &score[2], grad[10 + c]);
            orc_sum_add(&score[1], &score[3], grad[20 + c]);
        }
        uint64_t jj = (target - C) / A[c];
        int site = -1;
        uint64_t seen = 0;
        for (int i = 0; i < nd; ++i) {
            if (cls[i] == c) {
                if (seen == jj) { site = i; break; }
                ++seen;
            }
        }
        /* site >= 0 always: jj < n_c by construction */
        int xs = site % Ld, ys = site / Ld;
        SITE(xs, ys) = (int8_t)(-SITE(xs, ys));
        *flips += 1;
        uint64_t e = (np << 32) | ((uint64_t)j << 16) | (uint64_t)site;
        *hash = (*hash ^ e) * ORC_HASH_PRIME;
    }
#undef SITE
    free(top); free(bot); free(lft); free(rgt); free(cls);
}

/* ------------------------------------------------------------------------
 * Observables at a schedule endpoint (Sec. 2.3; App. A energy):
 *   bonds = sum over sites of s(x,y)*(s(x+1,y) + s(x,y+1)), periodic;
 *   mag = sum s;  e = (-J*bonds - h*mag)/N;  m = mag/N;  A = e*m;
 *   T = mean over domains of t_d, t_d = esum_d/Lambda (exponential) or
 *   steps_d/Lambda (expected), Lambda = n_d*nu.
 * out = {e, m, e*m, T}.
 * ---------------------------------------------------------------------- */
void orc_energy_mag(const int8_t *s, int L, int64_t *bonds, int64_t *mag)
{
    int64_t b = 0, m = 0;
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            int v = s[(int64_t)y * L + x];
            int r = s[(int64_t)y * L + (x + 1) % L];
            int u = s[(int64_t)((y + 1) % L) * L + x];
            b += v * (r + u);
            m += v;
        }
    }
    *bonds = b;
    *mag = m;
}

double orc_domain_time(int time_mode, double esum, int64_t steps, int nd,
                       double nu)
{
    double lambda = (double)nd * nu;
    if (time_mode == ORC_TIME_EXPONENTIAL || time_mode == ORC_TIME_HORIZON) return esum / lambda;
    return (double)steps / lambda;
}

static void orc_observe(const int8_t *s, int L, double J, double h,
                        int time_mode, const double *esum,
                        const int64_t *steps, int ND, int nd, double nu,
                        double out[4])
{
    int64_t bonds, mag;
    orc_energy_mag(s, L, &bonds, &mag);
    double N = (double)L * (double)L;
    double e = (-J * (double)bonds - h * (double)mag) / N;
    double m = (double)mag / N;
    double tsum = 0.0;
    for (int d = 0; d < ND; ++d)
        tsum += orc_domain_time(time_mode, esum[d], steps[d], nd, nu);
    out[0] = e;
    out[1] = m;
    out[2] = e * m;
    out[3] = tsum / (double)ND;
}

/* ------------------------------------------------------------------------
 * Run n_sched schedules of one replica, starting at global schedule index
 * sched_begin.  Per-domain state (esum, steps, hash, flips) is read and
 * updated in place, indexed d = by*Dx + bx.  If obs_every > 0, after each
 * local schedule n with (n+1) % obs_every == 0 the record
 * {e, m, e*m, T} is written to obs[4*((n+1)/obs_every - 1)].
 * Domains of one colour are visited in ascending d; the paper allows any
 * order because they do not interact (Sec. 2.2).
 * Returns 0, or -1 for an invalid configuration.
 * ---------------------------------------------------------------------- */
/* ------------------------------------------------------------------------
 * Fixed-time domain process: the number of uniformised steps in a visit of
 * domain time dtau is Poisson with mean mu = n_d nu dtau (uniformisation,
 * Sec. 2.1: events of a domain arrive at total rate n_d nu).  K is drawn by
 * inversion: thresholds T_k = floor(F(k) 2^64) of the Poisson CDF F, with
 * p_k = exp(-mu + k ln mu - lnGamma(k+1)) summed in k order, for
 * k < kmax = ceil(mu + 12 sqrt(mu) + 30); K = the first k with U < T_k for
 * the uniform U = w0 | w1 << 32 of Philox {0, d, np_lo, np_hi | TAG_HORIZON<<24},
 * or kmax if there is none.
 * ---------------------------------------------------------------------- */
int orc_horizon_kmax(double mu)
{
    return (int)ceil(mu + 12.0 * sqrt(mu) + 30.0);
}

void orc_horizon_table(double mu, int kmax, uint64_t *out)
{
    double logmu = log(mu);
    double F = 0.0;
    for (int k = 0; k < kmax; ++k) {
        double lp = -mu + (double)k * logmu - lgamma((double)k + 1.0);
        F += exp(lp);
        out[k] = (F >= 1.0) ? UINT64_MAX : (uint64_t)ldexp(F, 64);
    }
}

static int orc_horizon_steps(const uint64_t *tab, int kmax, uint32_t key0, uint32_t key1,
                             uint64_t np, uint32_t d)
{
    uint32_t ctr[4] = {0u, d, (uint32_t)np, (uint32_t)((np >> 32) & 0xFFFFFFu) | (ORC_TAG_HORIZON << 24)};
    uint32_t key[2] = {key0, key1};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint64_t U = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    for (int k = 0; k < kmax; ++k)
        if (U < tab[k]) return k;
    return kmax;
}

static void orc_record(const int8_t *s, int L, double J, double h, int time_mode,
                       const double *esum, const int64_t *steps, int ND, int nd,
                       double nu, const double *score, double *rec)
{
    orc_observe(s, L, J, h, time_mode, esum, steps, ND, nd, nu, rec);
    if (score) {
        double sb = 0.0, sh = 0.0;
        for (int d = 0; d < ND; ++d) {
            sb += score[4 * d] + score[4 * d + 2];
            sh += score[4 * d + 1] + score[4 * d + 3];
        }
        rec[4] = sb;
        rec[5] = sh;
    }
}

/* obs_unit 0: a record after every obs_every-th schedule of the call (the
 * schedule endpoints of Sec. 2.3); obs_unit 1: after every obs_every-th
 * colour pass of the call.  Every colour pass ends the domain processes of
 * one colour, so its end is a domain-process endpoint; the schedules read
 * with shifted registers end there (Sec. 2.3), which makes these valid
 * observation points as well. */
int orc_run_replica_ex(int8_t *s, int L, int Ld, int k, const uint64_t A[10],
                       uint64_t seed, int schedule, int time_mode, double nu,
                       double J, double h, int64_t sched_begin, int64_t n_sched,
                       int obs_every, int obs_unit, double dtau, double *esum, int64_t *steps,
                       uint64_t *hash, int64_t *flips, double *obs,
                       const double *grad, double *score)
{
    if (L <= 0 || Ld <= 0 || L % Ld != 0) return -1;
    int Dx = L / Ld;
    if (Dx < 2 || (Dx & 1)) return -1;
    if (orc_log2(Ld * Ld) < 0) return -1;
    if (k < 0 || k > 65535) return -1;
    if (obs_unit != 0 && obs_unit != 1) return -1;
    const int ND = Dx * Dx, nd = Ld * Ld;
    uint64_t *htab = NULL;
    int hkmax = 0;
    if (time_mode == ORC_TIME_HORIZON) {
        if (!(dtau > 0.0)) return -1;
        double mu = (double)nd * nu * dtau;
        hkmax = orc_horizon_kmax(mu);
        if (hkmax > 1024) return -1;
        htab = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)hkmax);
        orc_horizon_table(mu, hkmax, htab);
    }
    const int width = score ? 6 : 4;
    uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    int64_t passes = 0; /* colour passes completed in this call */
    for (int64_t nl = 0; nl < n_sched; ++nl) {
        uint64_t n = (uint64_t)(sched_begin + nl);
        int col[8];
        int nph = orc_schedule_colours(schedule, n, seed, col);
        if (nph < 0) { free(htab); return -1; }
        for (int p = 0; p < nph; ++p) {
            /* eight phase slots per schedule index for every schedule kind,
             * so that no two kinds ever share a Philox counter */
            uint64_t np = n * 8u + (uint64_t)p;
            for (int d = 0; d < ND; ++d) {
                int bx = d % Dx, by = d / Dx;
                int colour = (bx & 1) | ((by & 1) << 1);
                if (colour != col[p]) continue;
                int kv = k;
                if (time_mode == ORC_TIME_HORIZON)
                    kv = orc_horizon_steps(htab, hkmax, key0, key1, np, (uint32_t)d);
                orc_visit(s, L, Ld, bx, by, kv, A, key0, key1, np,
                          (uint32_t)d, time_mode, &esum[d], &hash[d],
                          &flips[d], &steps[d], grad,
                          score ? &score[4 * d] : NULL);
                /* fixed-time visit: the domain clock advances by dtau */
                if (time_mode == ORC_TIME_HORIZON) esum[d] += dtau * (double)nd * nu;
            }
            ++passes;
            if (obs_unit == 1 && obs_every > 0 && obs != NULL && passes % obs_every == 0)
                orc_record(s, L, J, h, time_mode, esum, steps, ND, nd, nu, score,
                           &obs[width * (passes / obs_every - 1)]);
        }
        if (obs_unit == 0 && obs_every > 0 && obs != NULL && (nl + 1) % obs_every == 0)
            orc_record(s, L, J, h, time_mode, esum, steps, ND, nd, nu, score,
                       &obs[width * ((nl + 1) / obs_every - 1)]);
    }
    free(htab);
    return 0;
}

int orc_run_replica_obs(int8_t *s, int L, int Ld, int k, const uint64_t A[10],
                        uint64_t seed, int schedule, int time_mode, double nu,
                        double J, double h, int64_t sched_begin, int64_t n_sched,
                        int obs_every, int obs_unit, double *esum, int64_t *steps,
                        uint64_t *hash, int64_t *flips, double *obs,
                        const double *grad, double *score)
{
    return orc_run_replica_ex(s, L, Ld, k, A, seed, schedule, time_mode, nu, J, h, sched_begin,
                              n_sched, obs_every, obs_unit, 0.0, esum, steps, hash, flips, obs,
                              grad, score);
}

int orc_run_replica_grad(int8_t *s, int L, int Ld, int k, const uint64_t A[10],
                         uint64_t seed, int schedule, int time_mode, double nu,
                         double J, double h, int64_t sched_begin, int64_t n_sched,
                         int obs_every, double *esum, int64_t *steps,
                         uint64_t *hash, int64_t *flips, double *obs,
                         const double *grad, double *score)
{
    return orc_run_replica_obs(s, L, Ld, k, A, seed, schedule, time_mode, nu, J, h,
                               sched_begin, n_sched, obs_every, 0, esum, steps, hash,
                               flips, obs, grad, score);
}

int orc_run_replica(int8_t *s, int L, int Ld, int k, const uint64_t A[10],
                    uint64_t seed, int schedule, int time_mode, double nu,
                    double J, double h, int64_t sched_begin, int64_t n_sched,
                    int obs_every, double *esum, int64_t *steps,
                    uint64_t *hash, int64_t *flips, double *obs)
{
    return orc_run_replica_grad(s, L, Ld, k, A, seed, schedule, time_mode, nu,
                                J, h, sched_begin, n_sched, obs_every, esum,
                                steps, hash, flips, obs, NULL, NULL);
}

uint64_t orc_hash_basis(void) { return ORC_HASH_BASIS; }

/* ------------------------------------------------------------------------
 * Many independent short runs for statistical tests: replica r uses seed
 * seed0 + r, starts from s0 (copied), runs n_sched schedules and writes its
 * final state to out[r*L*L ...].  Plain loop over orc_run_replica.
 * ---------------------------------------------------------------------- */
int orc_sample_final_states_grad(const int8_t *s0, int L, int Ld, int k,
                                 const uint64_t A[10], uint64_t seed0,
                                 int64_t n_runs, int schedule, int64_t n_sched,
                                 int8_t *out, const double *grad,
                                 double *score_out)
{
    int Dx = (Ld > 0) ? L / Ld : 0;
    int ND = Dx * Dx;
    if (ND <= 0) return -1;
    double *esum = (double *)calloc((size_t)ND, sizeof(double));
    int64_t *steps = (int64_t *)calloc((size_t)ND, sizeof(int64_t));
    uint64_t *hash = (uint64_t *)calloc((size_t)ND, sizeof(uint64_t));
    int64_t *flips = (int64_t *)calloc((size_t)ND, sizeof(int64_t));
    double *score = (double *)calloc((size_t)ND * 4, sizeof(double));
    int rc = 0;
    for (int64_t r = 0; r < n_runs && rc == 0; ++r) {
        int8_t *s = out + r * (int64_t)L * L;
        memcpy(s, s0, (size_t)L * L);
        memset(score, 0, sizeof(double) * (size_t)ND * 4);
        rc = orc_run_replica_grad(s, L, Ld, k, A, seed0 + (uint64_t)r,
                                  schedule, ORC_TIME_EXPECTED, 1.0, 1.0, 0.0,
                                  0, n_sched, 0, esum, steps, hash, flips,
                                  NULL, grad, grad ? score : NULL);
        if (grad && score_out) {
            double sb = 0.0, sh = 0.0;
            for (int d = 0; d < ND; ++d) {
                sb += score[4 * d] + score[4 * d + 2];
                sh += score[4 * d + 1] + score[4 * d + 3];
            }
            score_out[2 * r] = sb;
            score_out[2 * r + 1] = sh;
        }
    }
    free(esum); free(steps); free(hash); free(flips); free(score);
    return rc;
}

int orc_sample_final_states(const int8_t *s0, int L, int Ld, int k,
                            const uint64_t A[10], uint64_t seed0,
                            int64_t n_runs, int schedule, int64_t n_sched,
                            int8_t *out)
{
    return orc_sample_final_states_grad(s0, L, Ld, k, A, seed0, n_runs,
                                        schedule, n_sched, out, NULL, NULL);
}

/* ========================================================================
 * The 1D ring of Sec. 3.1: N_S spins with toroidal periodicity, energy
 * beta*H = -beta*J*sum_n s_n s_{n+1} (App. A, Eq. for beta*H, 1D line; here
 * with a field term -h*sum(s) as in 2D).  The ring is cut into N_D
 * contiguous domains of L_d = N_S/N_D spins (Sec. 3.1, Eq. 1D partitions:
 * domain d holds spins d*L_d .. d*L_d + L_d - 1).  A configuration is a
 * 64-bit word, bit n set iff spin n is up (N_S <= 64).
 *
 * Class c = 3*sp + q: sp = 1 for an up spin, q = number of up neighbours
 * (0..2); neighbour sum 2q - 2; dE_c = 2*sigma*(J*(2q-2) + h).  Rates and
 * fixed point as in 2D: A_c = round(a_c 2^P), P = 63 - log2(L_d); -2 when
 * some a_c rounds to 0 (as in 2D).
 * ====================================================================== */
int orc_ring_rate_table(double J, double beta, double h, int law, int log2_nd,
                        double a_out[6], uint64_t A_out[6])
{
    if (log2_nd < 0 || log2_nd > 6) return -1;
    if (law != ORC_RATE_METROPOLIS && law != ORC_RATE_BARKER) return -1;
    if (!(beta >= 0.0) || !isfinite(beta) || !isfinite(J) || !isfinite(h))
        return -1;
    int P = 63 - log2_nd;
    for (int sp = 0; sp < 2; ++sp) {
        for (int q = 0; q <= 2; ++q) {
            int c = 3 * sp + q;
            double sigma = sp ? 1.0 : -1.0;
            double dE = 2.0 * sigma * (J * (double)(2 * q - 2) + h);
            double a;
            if (law == ORC_RATE_METROPOLIS)
                a = (dE <= 0.0) ? 1.0 : exp(-beta * dE);
            else
                a = 1.0 / (1.0 + exp(beta * dE));
            a_out[c] = a;
            A_out[c] = (uint64_t)nearbyint(ldexp(a, P));
        }
    }
    for (int c = 0; c < 6; ++c)
        if (A_out[c] == 0) return -2;
    return 0;
}

static int orc_ring_spin(uint64_t S, int n) { return ((S >> n) & 1u) ? 1 : -1; }

/* bonds = sum_n s_n s_{n+1 mod N_S}, mag = sum_n s_n. */
void orc_ring_energy_mag(uint64_t S, int NS, int64_t *bonds, int64_t *mag)
{
    int64_t b = 0, m = 0;
    for (int n = 0; n < NS; ++n) {
        b += orc_ring_spin(S, n) * orc_ring_spin(S, (n + 1) % NS);
        m += orc_ring_spin(S, n);
    }
    *bonds = b;
    *mag = m;
}

/* ------------------------------------------------------------------------
 * Schedules of the ring.  Colour of domain d: d & 1 (N_D even; with N_D = 1
 * the single domain has colour 0).  One schedule is a list of phases; a
 * phase runs a set of domains that share no halo:
 *   PALINDROME: colours 0 1 1 0 (N_D = 1: 0 0), its own reverse;
 *   FIXED:      colours 0 1 (N_D = 1: 0), a negative test as in 2D;
 *   RANDOM_PERM: the paper's own protocol (Sec. 2.2, Fig. 1: a new random
 *               schedule after every sweep): a uniform random order of the
 *               N_D domains, one domain per phase, from a Fisher-Yates
 *               shuffle; draw i (i = N_D-1 down to 1) uses Philox
 *               {i, 0, n_lo, n_hi | TAG_PERM<<24} and swaps position i with
 *               floor(x (i+1) / 2^64), x = w0 | w1<<32.
 * out[p] is a colour (is_domain = 0) or a domain (is_domain = 1).  Returns
 * the number of phases, or -1.
 * ---------------------------------------------------------------------- */
int orc_ring_schedule(int schedule, uint64_t n, uint64_t seed, int ND, int out[64], int *is_domain)
{
    if (ND < 1 || ND > 64) return -1;
    *is_domain = 0;
    if (schedule == ORC_SCHED_PALINDROME || schedule == ORC_SCHED_FIXED) {
        if (ND != 1 && (ND & 1)) return -1;
        int ncol = (ND == 1) ? 1 : 2;
        int np = 0;
        for (int c = 0; c < ncol; ++c) out[np++] = c;
        if (schedule == ORC_SCHED_PALINDROME)
            for (int c = ncol - 1; c >= 0; --c) out[np++] = c;
        return np;
    }
    if (schedule == ORC_SCHED_RANDOM_PERM) {
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        for (int i = 0; i < ND; ++i) out[i] = i;
        for (int i = ND - 1; i >= 1; --i) {
            uint32_t ctr[4] = {(uint32_t)i, 0u, (uint32_t)n,
                               (uint32_t)((n >> 32) & 0xFFFFFFu) | (ORC_TAG_PERM << 24)};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            uint64_t x = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
            int j = (int)(((unsigned __int128)x * (unsigned)(i + 1)) >> 64);
            int t = out[i]; out[i] = out[j]; out[j] = t;
        }
        *is_domain = 1;
        return ND;
    }
    return -1;
}

/* ------------------------------------------------------------------------
 * One domain process of the ring: domain d, k uniformised steps with the
 * two halo spins (left of the first, right of the last site) frozen.  With
 * N_D = 1 the domain is the whole ring and both neighbours of every spin
 * are its own.  Step j of phase np uses Philox {j, d, np_lo, np_hi |
 * TAG_STEP<<24} exactly as in 2D: target, null step if target >= R',
 * class by cumulative rate, member jj = (target - C_{c-1}) / A_c in
 * ascending site order.  Event word e = np<<32 | j<<16 | (site - d*L_d);
 * the trajectory's hash folds all its events in order.
 * ---------------------------------------------------------------------- */
static void orc_ring_visit(uint64_t *S, int NS, int Ld, int d, int k, const uint64_t A[6],
                           uint32_t key0, uint32_t key1, uint64_t np, int time_mode,
                           double *esum, int64_t *steps, uint64_t *hash, int64_t *flips)
{
    const int ND = NS / Ld, first = d * Ld;
    int cls[64];
    int haloL = 0, haloR = 0;
    if (ND > 1) {
        haloL = orc_ring_spin(*S, (first - 1 + NS) % NS);
        haloR = orc_ring_spin(*S, (first + Ld) % NS);
    }
    for (int j = 0; j < k; ++j) {
        uint64_t n[6] = {0};
        for (int x = 0; x < Ld; ++x) {
            int site = first + x;
            int lf, rt;
            if (ND == 1) {
                lf = orc_ring_spin(*S, (site - 1 + NS) % NS);
                rt = orc_ring_spin(*S, (site + 1) % NS);
            } else {
                lf = (x > 0) ? orc_ring_spin(*S, site - 1) : haloL;
                rt = (x < Ld - 1) ? orc_ring_spin(*S, site + 1) : haloR;
            }
            int c = 3 * (orc_ring_spin(*S, site) > 0) + (lf > 0) + (rt > 0);
            cls[x] = c;
            n[c] += 1;
        }
        uint64_t R = 0;
        for (int c = 0; c < 6; ++c) R += n[c] * A[c];

        uint32_t ctr[4] = {(uint32_t)j, (uint32_t)d, (uint32_t)np,
                           (uint32_t)((np >> 32) & 0xFFFFFFu) | (ORC_TAG_STEP << 24)};
        uint32_t key[2] = {key0, key1};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        uint64_t target = ((uint64_t)w[0] | ((uint64_t)w[1] << 32)) >> 1;
        uint64_t V = (((uint64_t)w[2] | ((uint64_t)w[3] << 32)) >> 11) + 1u;
        if (time_mode == ORC_TIME_EXPONENTIAL)
            esum[d] += -log(ldexp((double)V, -53));
        steps[d] += 1;
        if (target >= R) continue;

        uint64_t C = 0;
        int c;
        for (c = 0; c < 6; ++c) {
            uint64_t wc = n[c] * A[c];
            if (target < C + wc) break;
            C += wc;
        }
        uint64_t jj = (target - C) / A[c];
        int x = -1;
        uint64_t seen = 0;
        for (int i = 0; i < Ld; ++i) {
            if (cls[i] == c) {
                if (seen == jj) { x = i; break; }
                ++seen;
            }
        }
        *S ^= 1ull << (first + x);
        *flips += 1;
        uint64_t e = (np << 32) | ((uint64_t)j << 16) | (uint64_t)x;
        *hash = (*hash ^ e) * ORC_HASH_PRIME;
    }
}

/* ------------------------------------------------------------------------
 * Run n_sched schedules of one ring trajectory from global schedule index
 * sched_begin.  Phase p of schedule n has the Philox phase index
 * np = n*64 + p.  A "pass" is one phase (a colour, or one domain for
 * RANDOM_PERM); its end is a domain-process endpoint (Sec. 2.3), and after
 * every obs_every-th pass of the call the record {e, m, e*m, T} goes to
 * obs[4*i] and the configuration word to obs_state[i] (either may be NULL).
 * e = (-J bonds - h mag)/N_S, m = mag/N_S, T = mean over domains of t_d,
 * t_d = esum_d/(L_d nu) (exponential) or steps_d/(L_d nu) (expected).
 * esum and steps are per domain [N_D]; hash and flips per trajectory.
 * ---------------------------------------------------------------------- */
int orc_ring_run(uint64_t *S, int NS, int Ld, int k, const uint64_t A[6], uint64_t seed,
                 int schedule, int time_mode, double nu, double J, double h,
                 int64_t sched_begin, int64_t n_sched, int obs_every,
                 double *esum, int64_t *steps, uint64_t *hash, int64_t *flips,
                 double *obs, uint64_t *obs_state)
{
    if (NS < 2 || NS > 64 || Ld < 1 || NS % Ld != 0 || orc_log2(Ld) < 0) return -1;
    if (k < 0 || k > 65535) return -1;
    if (time_mode != ORC_TIME_EXPONENTIAL && time_mode != ORC_TIME_EXPECTED) return -1;
    const int ND = NS / Ld;
    uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    int64_t passes = 0;
    for (int64_t nl = 0; nl < n_sched; ++nl) {
        uint64_t n = (uint64_t)(sched_begin + nl);
        int ph[64], is_domain;
        int nph = orc_ring_schedule(schedule, n, seed, ND, ph, &is_domain);
        if (nph < 0) return -1;
        for (int p = 0; p < nph; ++p) {
            uint64_t np = n * 64u + (uint64_t)p;
            for (int d = 0; d < ND; ++d) {
                if (is_domain ? (d != ph[p]) : ((d & 1) != ph[p])) continue;
                orc_ring_visit(S, NS, Ld, d, k, A, key0, key1, np, time_mode, esum, steps, hash, flips);
            }
            ++passes;
            if (obs_every > 0 && passes % obs_every == 0) {
                int64_t i = passes / obs_every - 1;
                if (obs) {
                    int64_t b, m;
                    orc_ring_energy_mag(*S, NS, &b, &m);
                    double e = (-J * (double)b - h * (double)m) / (double)NS;
                    double tsum = 0.0;
                    for (int d = 0; d < ND; ++d)
                        tsum += orc_domain_time(time_mode, esum[d], steps[d], Ld, nu);
                    obs[4 * i] = e;
                    obs[4 * i + 1] = (double)m / (double)NS;
                    obs[4 * i + 2] = e * ((double)m / (double)NS);
                    obs[4 * i + 3] = tsum / (double)ND;
                }
                if (obs_state) obs_state[i] = *S;
            }
        }
    }
    return 0;
}

/* Many independent ring trajectories, one after another: trajectory r
 * starts from S[r] with seed seeds[r] and runs n_sched schedules from
 * schedule 0; S[r] receives its final configuration; obs / obs_state (or
 * NULL) receive its records at [r * n_rec ...]; hash[r], flips[r] its
 * event hash and real-event count.  A plain loop over orc_ring_run. */
int orc_ring_run_many(int64_t n_traj, uint64_t *S, const uint64_t *seeds, int NS, int Ld, int k,
                      const uint64_t A[6], int schedule, int time_mode, double nu, double J, double h,
                      int64_t n_sched, int obs_every, int64_t n_rec, double *obs, uint64_t *obs_state,
                      uint64_t *hash, int64_t *flips)
{
    if (NS < 2 || NS > 64 || Ld < 1 || NS % Ld != 0) return -1;
    const int ND = NS / Ld;
    double *esum = (double *)calloc((size_t)ND, sizeof(double));
    int64_t *steps = (int64_t *)calloc((size_t)ND, sizeof(int64_t));
    int rc = 0;
    for (int64_t r = 0; r < n_traj && rc == 0; ++r) {
        memset(esum, 0, sizeof(double) * (size_t)ND);
        memset(steps, 0, sizeof(int64_t) * (size_t)ND);
        uint64_t hh = ORC_HASH_BASIS;
        int64_t ff = 0;
        rc = orc_ring_run(&S[r], NS, Ld, k, A, seeds[r], schedule, time_mode, nu, J, h, 0, n_sched,
                          obs_every, esum, steps, &hh, &ff, obs ? &obs[4 * r * n_rec] : NULL,
                          obs_state ? &obs_state[r * n_rec] : NULL);
        if (hash) hash[r] = hh;
        if (flips) flips[r] = ff;
    }
    free(esum);
    free(steps);
    return rc;
}

/* ========================================================================
 * Small 2D lattices under the partitions of Sec. 3.2: an L x L periodic
 * lattice cut either into a Dx x Dx grid of square blocks (the checkerboard
 * of Sec. 2.2, Fig. 1) or into N_D vertical stripes of width L/N_D and full
 * height (Fig. 1 caption: the striped partition; Sec. 3.2 uses both).  The
 * domain size n_d need not be a power of two (the paper's 12^2 and 100^2
 * lattices), so the step target is taken as a multiply-high:
 *   P = 63 - ceil(log2 n_d),  M = n_d 2^P <= 2^63,
 *   target = floor(X M / 2^64),  X = w0 | w1<<32,
 * uniform on [0, M) up to one X value per interval boundary (probabilities
 * exact to 2^-64).  With n_d a power of two M = 2^63 and the target is
 * X >> 1, the lattice protocol above.  A_c = round(a_c 2^P); a step is null
 * iff target >= R' = sum_c n_c A_c, so site i flips with probability
 * A_c(i)/M = (A_c/2^P)/n_d (App. A, selection probability 1/n_d).
 *
 * Colours: blocks (bx&1) | ((by&1)<<1) (Dx even), stripes d & 1 (N_D even),
 * a single domain colour 0.  Schedules: PALINDROME = colours ascending then
 * descending, FIXED = ascending, RANDOM_PERM = the paper's uniform random
 * order of all N_D domains per sweep (Fisher-Yates as for the ring, one
 * domain per phase).  Phase p of schedule n has Philox phase index
 * np = 64 n + p.  One trajectory's event hash folds its events in order.
 * ====================================================================== */
#define ORC_PART_BLOCKS 0
#define ORC_PART_STRIPES 1

static int orc_ceil_log2(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

/* Domain d's rectangle: x0, y0, width, height; its colour; -1 if invalid. */
int orc_part_geometry(int L, int kind, int ND, int d, int *x0, int *y0, int *w, int *hgt, int *colour)
{
    if (L < 2 || ND < 1 || d < 0 || d >= ND) return -1;
    if (kind == ORC_PART_BLOCKS) {
        int Dx = 0;
        while ((Dx + 1) * (Dx + 1) <= ND) ++Dx;
        if (Dx * Dx != ND || L % Dx != 0) return -1;
        int side = L / Dx, bx = d % Dx, by = d / Dx;
        *x0 = bx * side; *y0 = by * side; *w = side; *hgt = side;
        *colour = (Dx == 1) ? 0 : ((Dx & 1) ? -1 : ((bx & 1) | ((by & 1) << 1)));
        return 0;
    }
    if (kind == ORC_PART_STRIPES) {
        if (L % ND != 0) return -1;
        *x0 = d * (L / ND); *y0 = 0; *w = L / ND; *hgt = L;
        *colour = (ND == 1) ? 0 : ((ND & 1) ? -1 : (d & 1));
        return 0;
    }
    return -1;
}

static int orc_part_ncolours(int kind, int ND)
{
    if (ND == 1) return 1;
    return kind == ORC_PART_BLOCKS ? 4 : 2;
}

/* Phases of schedule n: colours (is_domain 0) or domains (is_domain 1). */
int orc_part_schedule(int kind, int schedule, uint64_t n, uint64_t seed, int ND, int out[64], int *is_domain)
{
    if (ND < 1 || ND > 64) return -1;
    *is_domain = 0;
    if (schedule == ORC_SCHED_PALINDROME || schedule == ORC_SCHED_FIXED) {
        if (kind == ORC_PART_BLOCKS) {
            int Dx = 0;
            while ((Dx + 1) * (Dx + 1) <= ND) ++Dx;
            if (Dx * Dx != ND || (Dx > 1 && (Dx & 1))) return -1;
        } else if (kind != ORC_PART_STRIPES || (ND > 1 && (ND & 1))) {
            return -1;
        }
        int nc = orc_part_ncolours(kind, ND), np = 0;
        for (int c = 0; c < nc; ++c) out[np++] = c;
        if (schedule == ORC_SCHED_PALINDROME)
            for (int c = nc - 1; c >= 0; --c) out[np++] = c;
        return np;
    }
    if (schedule == ORC_SCHED_RANDOM_PERM) {
        int isd;
        int r = orc_ring_schedule(ORC_SCHED_RANDOM_PERM, n, seed, ND, out, &isd);
        *is_domain = 1;
        return r;
    }
    return -1;
}

static void orc_part_visit(int8_t *s, int L, int x0, int y0, int W, int H, int d, int k, const uint64_t A[10],
                           uint64_t M, uint32_t key0, uint32_t key1, uint64_t np, int time_mode,
                           double *esum, int64_t *steps, uint64_t *hash, int64_t *flips)
{
    const int nd = W * H;
    int8_t *frozen = (int8_t *)malloc((size_t)L * L);
    int *cls = (int *)malloc(sizeof(int) * (size_t)nd);
    /* the halo is frozen: neighbours outside the domain are read from this
     * copy taken before the process runs */
    memcpy(frozen, s, (size_t)L * L);
#define PSITE(xx, yy) s[(int64_t)(yy) * L + (xx)]
#define INDOM(xx, yy) ((xx) >= x0 && (xx) < x0 + W && (yy) >= y0 && (yy) < y0 + H)
#define NB(xx, yy) (INDOM(xx, yy) ? PSITE(xx, yy) : frozen[(int64_t)(yy) * L + (xx)])
    for (int j = 0; j < k; ++j) {
        uint64_t n[10] = {0};
        for (int yy = 0; yy < H; ++yy) {
            for (int xx = 0; xx < W; ++xx) {
                int x = x0 + xx, y = y0 + yy;
                int up = NB(x, (y - 1 + L) % L), dn = NB(x, (y + 1) % L);
                int lf = NB((x - 1 + L) % L, y), rt = NB((x + 1) % L, y);
                int q = (up > 0) + (dn > 0) + (lf > 0) + (rt > 0);
                int c = 5 * (PSITE(x, y) > 0) + q;
                cls[yy * W + xx] = c;
                n[c] += 1;
            }
        }
        uint64_t R = 0;
        for (int c = 0; c < 10; ++c) R += n[c] * A[c];
        uint32_t ctr[4] = {(uint32_t)j, (uint32_t)d, (uint32_t)np,
                           (uint32_t)((np >> 32) & 0xFFFFFFu) | (ORC_TAG_STEP << 24)};
        uint32_t key[2] = {key0, key1};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        uint64_t X = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
        uint64_t target = (uint64_t)(((unsigned __int128)X * M) >> 64);
        uint64_t V = (((uint64_t)w[2] | ((uint64_t)w[3] << 32)) >> 11) + 1u;
        if (time_mode == ORC_TIME_EXPONENTIAL) esum[d] += -log(ldexp((double)V, -53));
        steps[d] += 1;
        if (target >= R) continue;
        uint64_t C = 0;
        int c;
        for (c = 0; c < 10; ++c) {
            uint64_t wc = n[c] * A[c];
            if (target < C + wc) break;
            C += wc;
        }
        uint64_t jj = (target - C) / A[c];
        int site = -1;
        uint64_t seen = 0;
        for (int i = 0; i < nd; ++i) {
            if (cls[i] == c) {
                if (seen == jj) { site = i; break; }
                ++seen;
            }
        }
        int xs = x0 + site % W, ys = y0 + site / W;
        PSITE(xs, ys) = (int8_t)(-PSITE(xs, ys));
        *flips += 1;
        uint64_t e = (np << 32) | ((uint64_t)j << 16) | (uint64_t)site;
        *hash = (*hash ^ e) * ORC_HASH_PRIME;
    }
#undef NB
#undef INDOM
#undef PSITE
    free(frozen);
    free(cls);
}

/* n_d and the fixed-point scale of a partition: returns P and sets *M. */
int orc_part_scale(int L, int kind, int ND, uint64_t *M)
{
    int x0, y0, w, hh, col;
    if (orc_part_geometry(L, kind, ND, 0, &x0, &y0, &w, &hh, &col) != 0) return -1;
    int nd = w * hh;
    if (nd > 16384) return -1;
    int P = 63 - orc_ceil_log2(nd);
    *M = (uint64_t)nd << P;
    return P;
}

/* Run n_sched schedules of one trajectory from schedule sched_begin.
 * esum/steps per domain [N_D]; hash/flips of the trajectory; a record
 * {e, m, e*m, T} after every obs_every-th pass of the call to obs[4 i]. */
int orc_part_run(int8_t *s, int L, int kind, int ND, int k, const uint64_t A[10], uint64_t seed,
                 int schedule, int time_mode, double nu, double J, double h, int64_t sched_begin,
                 int64_t n_sched, int obs_every, double *esum, int64_t *steps, uint64_t *hash,
                 int64_t *flips, double *obs)
{
    if (L < 2 || L > 4096 || ND < 1 || ND > 64 || k < 0 || k > 65535) return -1;
    if (time_mode != ORC_TIME_EXPONENTIAL && time_mode != ORC_TIME_EXPECTED) return -1;
    uint64_t M;
    if (orc_part_scale(L, kind, ND, &M) < 0) return -1;
    int x0, y0, W, H, col0;
    orc_part_geometry(L, kind, ND, 0, &x0, &y0, &W, &H, &col0);
    const int nd = W * H;
    uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    int64_t passes = 0;
    for (int64_t nl = 0; nl < n_sched; ++nl) {
        uint64_t n = (uint64_t)(sched_begin + nl);
        int ph[64], is_domain;
        int nph = orc_part_schedule(kind, schedule, n, seed, ND, ph, &is_domain);
        if (nph < 0) return -1;
        for (int p = 0; p < nph; ++p) {
            uint64_t np = n * 64u + (uint64_t)p;
            for (int d = 0; d < ND; ++d) {
                int dx0, dy0, dw, dh, col;
                orc_part_geometry(L, kind, ND, d, &dx0, &dy0, &dw, &dh, &col);
                if (is_domain ? (d != ph[p]) : (col != ph[p])) continue;
                orc_part_visit(s, L, dx0, dy0, dw, dh, d, k, A, M, key0, key1, np, time_mode, esum, steps,
                               hash, flips);
            }
            ++passes;
            if (obs_every > 0 && obs && passes % obs_every == 0) {
                int64_t i = passes / obs_every - 1;
                orc_observe(s, L, J, h, time_mode, esum, steps, ND, nd, nu, &obs[4 * i]);
            }
        }
    }
    return 0;
}

/* Independent partitioned trajectories: trajectory r starts from s0 with
 * seed seeds[r], runs n_sched schedules from schedule 0; its final spins go
 * to out[r*L*L ...], its records (or nothing if obs is NULL) to
 * obs[4 r n_rec ...], its hash and real flips to hash[r], flips[r]. */
int orc_part_run_many(int64_t n_traj, const int8_t *s0, const uint64_t *seeds, int L, int kind, int ND, int k,
                      const uint64_t A[10], int schedule, int time_mode, double nu, double J, double h,
                      int64_t n_sched, int obs_every, int64_t n_rec, int8_t *out, double *obs, uint64_t *hash,
                      int64_t *flips)
{
    if (ND < 1 || ND > 64) return -1;
    double *esum = (double *)calloc((size_t)ND, sizeof(double));
    int64_t *steps = (int64_t *)calloc((size_t)ND, sizeof(int64_t));
    int rc = 0;
    for (int64_t r = 0; r < n_traj && rc == 0; ++r) {
        int8_t *s = out + r * (int64_t)L * L;
        memcpy(s, s0, (size_t)L * L);
        memset(esum, 0, sizeof(double) * (size_t)ND);
        memset(steps, 0, sizeof(int64_t) * (size_t)ND);
        uint64_t hh = ORC_HASH_BASIS;
        int64_t ff = 0;
        rc = orc_part_run(s, L, kind, ND, k, A, seeds[r], schedule, time_mode, nu, J, h, 0, n_sched, obs_every,
                          esum, steps, &hh, &ff, obs ? &obs[4 * r * n_rec] : NULL);
        if (hash) hash[r] = hh;
        if (flips) flips[r] = ff;
    }
    free(esum);
    free(steps);
    return rc;
}
